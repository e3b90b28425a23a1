// Device bodies of the build kernels (S2-S3, Alg. 1-2), parameterised by a
// virtual CTA index (vb of vg) so the same code runs as a plain grid and as an
// item of the batched persistent kernel.  Scratch written earlier in the same
// launch (per-frame leaf bitsets) is read with ordinary coherent loads, after
// the reader's acquire (counter wait + fence).
#pragma once

#include <cuda.h>

#include <type_traits>

#include "async_copy.cuh"
#include "pixels.cuh"

namespace ocq {

__device__ __forceinline__ void red_add_shared(uint32_t *p, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}

template <int MAXP>
__device__ __forceinline__ void planes_add_reg(uint32_t (&pl)[MAXP], int P, uint32_t x) {
#pragma unroll
  for (int k = 0; k < MAXP; ++k) {
    if (k < P) {
      uint32_t t = pl[k] & x;
      pl[k] ^= x;
      x = t;
    }
  }
}

template <int MAXP>
__device__ __forceinline__ uint32_t planes_ge_reg(const uint32_t (&pl)[MAXP], int P, uint32_t T) {
  uint32_t gt = 0, eq = 0xFFFFFFFFu;
#pragma unroll
  for (int k = MAXP - 1; k >= 0; --k) {
    if (k < P) {
      const uint32_t c = pl[k];
      if ((T >> k) & 1u) {
        eq &= c;
      } else {
        gt |= eq & c;
        eq &= ~c;
      }
    }
  }
  return gt | eq;
}

// ---- dense per-frame occupancy ----------------------------------------------

// Whole-frame regions, depth <= 6: CTA (x, y) marks the leaves of pixel chunk x
// of frame f0 + y in a shared bitset, then ORs it into occ[y / group] (frames
// of one group share a tree, Sec. 3; group = 1: one tree per frame).
template <int D>
__device__ __forceinline__ void occ_frame_body(const uint8_t *__restrict__ frames, int64_t hw, int f0, int64_t chunk,
                                               uint32_t *__restrict__ occ, int64_t bx, int64_t by, int group = 1) {
  constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  extern __shared__ uint32_t seen[];  // [WPR]
  for (int i = threadIdx.x; i < WPR; i += blockDim.x) seen[i] = 0;
  __syncthreads();
  const uint8_t *fr = frames + (int64_t)(f0 + by) * hw * 3;
  const int64_t p0 = bx * chunk;
  const int64_t p1 = p0 + chunk < hw ? p0 + chunk : hw;
  cta_for_codes<D>(fr, p0, p1, [&](uint32_t q, int64_t) {
    const uint32_t m = 1u << (q & 31);
    if (!(seen[q >> 5] & m)) atomicOr(&seen[q >> 5], m);
  });
  __syncthreads();
  uint32_t *dst = occ + (by / group) * WPR;
  for (int i = threadIdx.x; i < WPR; i += blockDim.x)
    if (seen[i]) atomicOr(&dst[i], seen[i]);
}

// Any region kind and depth: one thread per pixel, global atomics into
// occ[((f - f0) / group) * R + r][...].
__device__ __forceinline__ void occ_global_body(const uint8_t *__restrict__ frames, int H, int W, int kind, int block,
                                                int d, int f0, int nf, int64_t R, int64_t wpr,
                                                uint32_t *__restrict__ occ, int64_t vb, int64_t vg, int group = 1) {
  const int64_t hw = (int64_t)H * W;
  const int64_t npix = hw * nf;
  const int bw = kind == OCQ_REGION_BLOCK ? (W + block - 1) / block : 1;
  const uint8_t *base = frames + (int64_t)f0 * hw * 3;
  for (int64_t i = vb * blockDim.x + threadIdx.x; i < npix; i += vg * blockDim.x) {
    const int64_t f = i / hw, p = i - f * hw;
    const int y = (int)(p / W), x = (int)(p - (int64_t)y * W);
    const uint8_t *px = base + i * 3;
    const uint32_t q = planar_code_rt(__ldg(px), __ldg(px + 1), __ldg(px + 2), d);
    uint32_t *word = occ + ((f / group) * R + region_of(y, x, W, kind, block, bw)) * wpr + (q >> 5);
    const uint32_t m = 1u << (q & 31);
    if (!(*(volatile uint32_t *)word & m)) atomicOr(word, m);
  }
}

// Folds nb frames of occupancy words into bit-sliced counters; on the last
// batch writes count >= T into the model.
__device__ __forceinline__ void planes_merge_body(const uint32_t *occ, int nb, int64_t nwords,
                                                  uint32_t *__restrict__ planes, int P, int first, int last,
                                                  uint32_t T, uint32_t *__restrict__ model, int64_t vb, int64_t vg) {
  for (int64_t w = vb * blockDim.x + threadIdx.x; w < nwords; w += vg * blockDim.x) {
    uint32_t pl[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) pl[k] = (!first && k < P) ? planes[k * nwords + w] : 0u;
    for (int f = 0; f < nb; ++f) planes_add_reg<16>(pl, P, occ[f * nwords + w]);
    if (last) {
      model[w] = planes_ge_reg<16>(pl, P, T);
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (k < P) planes[k * nwords + w] = pl[k];
    }
  }
}

// ---- block regions, depth <= 5 -----------------------------------------------
// One CTA per block region.  Per training frame the block's leaves are marked
// in a shared bitset; the first thread to set a bit in an empty word appends
// the word to a list, so only listed words are folded into the bit-sliced
// counters and cleared (a block has at most b*b leaves per frame, far fewer
// than 8^d/32 words at depth 4-5).
template <int D>
__device__ __forceinline__ void build_block_body(const uint8_t *__restrict__ frames, int N, int H, int W, int b, int bw,
                                                 int P, uint32_t T, uint32_t *__restrict__ model, int64_t R,
                                                 int64_t vb, int64_t vg) {
  constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  extern __shared__ uint32_t sm[];
  uint32_t *seen = sm;                   // [WPR]
  uint32_t *planes = sm + WPR;           // [P][WPR]
  uint32_t *list = planes + P * WPR;     // [WPR] words set in the current frame
  __shared__ uint32_t nlist;
  for (int64_t r = vb; r < R; r += vg) {
  __syncthreads();  // the previous block's rows are written out
  for (int i = threadIdx.x; i < WPR * (P + 1); i += blockDim.x) sm[i] = 0;
  if (threadIdx.x == 0) nlist = 0;
  const int y0 = (int)(r / bw) * b, x0 = (int)(r % bw) * b;
  const int h = min(b, H - y0), w = min(b, W - x0);
  const int npx = h * w;
  const int64_t hw = (int64_t)H * W;
  __syncthreads();
  // Each thread owns up to 4 pixels of the block (b <= 32 with 256 threads) and
  // loads their bytes for PF frames at once, so the per-frame marking and
  // folding below never waits on global memory.
  constexpr int PF = 8;
  const bool fast = npx <= 4 * (int)blockDim.x;
  const int64_t fstride = hw * 3;
  for (int f0 = 0; f0 < N; f0 += PF) {
    uint32_t yv[PF][4];
    if (fast) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = threadIdx.x + k * blockDim.x;
        if (i < npx) {
          const uint8_t *px = frames + ((int64_t)(y0 + i / w) * W + x0 + i % w) * 3;
#pragma unroll
          for (int j = 0; j < PF; ++j)
            if (f0 + j < N) {
              const uint8_t *s = px + (int64_t)(f0 + j) * fstride;
              yv[j][k] = (uint32_t)__ldg(s) | ((uint32_t)__ldg(s + 1) << 8) | ((uint32_t)__ldg(s + 2) << 16);
            }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      if (f0 + j >= N) break;
      const int f = f0 + j;
      // Marks leaf q; the lane that turns a word non-zero appends it to the
      // frame's list.  Appends are aggregated per warp (one shared atomic per
      // warp and frame instead of one per word).
      auto mark = [&](uint32_t q) {
        const uint32_t m = 1u << (q & 31);
        bool first = false;
        if (!(seen[q >> 5] & m)) first = atomicOr(&seen[q >> 5], m) == 0;
        const unsigned act = __activemask();
        const unsigned bal = __ballot_sync(act, first);
        if (bal) {
          const int lane = threadIdx.x & 31;
          const int leader = __ffs(bal) - 1;
          uint32_t base = 0;
          if (lane == leader) base = atomicAdd(&nlist, (uint32_t)__popc(bal));
          base = __shfl_sync(act, base, leader);
          if (first) list[base + __popc(bal & ((1u << lane) - 1u))] = q >> 5;
        }
      };
      if (fast) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (threadIdx.x + k * blockDim.x < npx) mark(planar_code<D>(yv[j][k]));
      } else {
        const uint8_t *fr = frames + (int64_t)f * fstride;
        for (int i = threadIdx.x; i < npx; i += blockDim.x) {
          const uint8_t *px = fr + ((int64_t)(y0 + i / w) * W + x0 + i % w) * 3;
          mark(planar_code_rt(__ldg(px), __ldg(px + 1), __ldg(px + 2), D));
        }
      }
      __syncthreads();
      const uint32_t n = nlist;
      for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
        const uint32_t wd = list[k];
        uint32_t x = seen[wd];
        for (int p = 0; p < P && x; ++p) {
          const uint32_t t = planes[p * WPR + wd] & x;
          planes[p * WPR + wd] ^= x;
          x = t;
        }
        seen[wd] = 0;
      }
      __syncthreads();
      if (threadIdx.x == 0) nlist = 0;
      __syncthreads();
    }
  }
  for (int wd = threadIdx.x; wd < WPR; wd += blockDim.x) {
    uint32_t gt = 0, eq = 0xFFFFFFFFu;
    for (int k = P - 1; k >= 0; --k) {
      const uint32_t c = planes[k * WPR + wd];
      if ((T >> k) & 1u) {
        eq &= c;
      } else {
        gt |= eq & c;
        eq &= ~c;
      }
    }
    model[r * WPR + wd] = gt | eq;
  }
  }
}

// ---- block regions, one warp per region ----------------------------------------
// A b x b block (b <= 16, so at most 8 pixels per lane) holds at most b*b
// distinct leaves per frame and usually a few dozen over all N frames, far
// fewer than the 8^d leaves of its row.  So each warp counts its region's
// leaves in a small table in shared memory instead of a dense counter row:
// entry = (leaf + 1) << 16 | last frame << 8 | frames counted (N <= 255).
// Every lane updates the entry of its own pixel's leaf: in frame f the entry
// is either still (leaf, earlier frame, c) or already (leaf, f, c + 1), and a
// lane that reads the first writes the second, so lanes holding the same leaf
// in the same frame write the same value and the leaf is counted once per
// frame whatever order they run in.  Only a new leaf claiming an empty slot of
// the hashed table needs an atomic (two leaves may hash to one slot).  One
// __syncwarp per frame makes frame f's updates visible before frame f + 1.
// With 8^d <= WarpTableCfg::S the table is indexed by the leaf itself; above
// it, by a multiplicative hash with linear probing.  A region with more than
// 3/4 S distinct leaves falls back to passes over S-leaf chunks of the code
// space, each indexed directly.  The model row is zeroed with vector stores and
// the kept leaves (count >= T) are ORed in.
template <int D>
struct WarpTableCfg {
  static constexpr int NC = 1 << (3 * D);
  static constexpr int S = NC < 1024 ? NC : 1024;  // entries per warp
  static constexpr bool DIRECT = NC <= S;
  static constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  static constexpr int LOGS = 3 * D < 10 ? 3 * D : 10;
};

// Counts leaf q in frame f; returns 1 if it took an empty slot of the hashed
// table.  INDEXED: the slot is q mod S (direct table, or a chunk pass).
template <int D, bool INDEXED>
__device__ __forceinline__ uint32_t warp_table_count(uint32_t *tab, uint32_t q, uint32_t f) {
  using C = WarpTableCfg<D>;
  const uint32_t stamp = ((q + 1) << 16) | (f << 8);
  if constexpr (INDEXED) {
    volatile uint32_t *slot = &tab[q & (C::S - 1)];
    const uint32_t e = *slot;
    if (e == 0u)
      *slot = stamp | 1u;
    else if (((e >> 8) & 255u) != f)
      *slot = stamp | ((e & 255u) + 1u);
    return 0u;
  } else {
    const uint32_t key = (q + 1) << 16;
    uint32_t h = (q * 2654435761u) >> (32 - C::LOGS);
    for (int probe = 0; probe < C::S; ++probe) {
      volatile uint32_t *slot = &tab[h];
      uint32_t e = *slot;
      if (e == 0u) {
        e = atomicCAS(&tab[h], 0u, stamp | 1u);
        if (e == 0u) return 1u;  // inserted
      }
      if ((e & 0xFFFF0000u) == key) {
        if (((e >> 8) & 255u) != f) *slot = stamp | ((e & 255u) + 1u);
        return 0u;
      }
      h = (h + 1) & (C::S - 1);
    }
    return 0u;  // unreachable: the table is never more than 3/4 + 1/4 full
  }
}

// Zeroes the region's model row (WPR words) with the warp's lanes.
template <int D>
__device__ __forceinline__ void warp_zero_row(uint32_t *row) {
  constexpr int WPR = WarpTableCfg<D>::WPR;
  const int lane = threadIdx.x & 31;
  if constexpr (WPR >= 4) {
    uint4 *r4 = reinterpret_cast<uint4 *>(row);
    for (int i = lane; i < WPR / 4; i += 32) r4[i] = make_uint4(0, 0, 0, 0);
  } else {
    if (lane < WPR) row[lane] = 0u;
  }
}

// Emits kept leaves of the table into the (zeroed) row and clears the table.
template <int D>
__device__ __forceinline__ void warp_emit(uint32_t *tab, uint32_t *row, uint32_t T) {
  using C = WarpTableCfg<D>;
  const int lane = threadIdx.x & 31;
  __syncwarp();
  for (int s = lane; s < C::S; s += 32) {
    const uint32_t e = tab[s];
    if (e) {
      tab[s] = 0u;
      if ((e & 255u) >= T) {
        const uint32_t q = (e >> 16) - 1u;
        atomicOr(&row[q >> 5], 1u << (q & 31));
      }
    }
  }
  __syncwarp();
}

// One pass over the region's N frames.  CHUNKED: only leaves in
// [chunk * S, chunk * S + S), indexed directly; otherwise every leaf.  Returns
// false if the hashed pass saw more than 3/4 S distinct leaves.
// SRC = uint16_t: `frames` holds planar leaf codes (a serving window's
// per-frame occupancy), fstride and off count codes instead of bytes.
template <int D, int PPL, int PF, bool CHUNKED, typename SRC = uint8_t>
__device__ __forceinline__ bool warp_region_pass(const SRC *__restrict__ frames, int N, int64_t fstride,
                                                 const uint32_t (&off)[PPL], int npx, uint32_t *tab, int chunk) {
  constexpr bool CODES = std::is_same<SRC, uint16_t>::value;
  using C = WarpTableCfg<D>;
  constexpr bool INDEXED = C::DIRECT || CHUNKED;
  const int lane = threadIdx.x & 31;
  uint32_t inserted = 0;
  for (int f0 = 0; f0 < N; f0 += PF) {
    uint32_t yv[PF][PPL];
    const SRC *fb = frames + (int64_t)f0 * fstride;
#pragma unroll
    for (int j = 0; j < PF; ++j)
#pragma unroll
      for (int k = 0; k < PPL; ++k)
        if (f0 + j < N && lane + 32 * k < npx) {
          const SRC *s = fb + (int64_t)j * fstride + off[k];
          if constexpr (CODES)
            yv[j][k] = __ldg(s);
          else
            yv[j][k] = (uint32_t)__ldg(s) | ((uint32_t)__ldg(s + 1) << 8) | ((uint32_t)__ldg(s + 2) << 16);
        }
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      if (f0 + j >= N) break;
#pragma unroll
      for (int k = 0; k < PPL; ++k) {
        if (lane + 32 * k < npx) {
          const uint32_t q = (CODES ? yv[j][k] : planar_code<D>(yv[j][k]));
          if (!CHUNKED || (int)(q >> C::LOGS) == chunk)
            inserted += warp_table_count<D, INDEXED>(tab, q, (uint32_t)(f0 + j));
        }
      }
      __syncwarp();
      if constexpr (!INDEXED)
        if (__reduce_add_sync(0xFFFFFFFFu, inserted) > (uint32_t)(3 * C::S / 4)) return false;
    }
  }
  return true;
}

// The same pass for a full 8 x 8 block whose rows start on 4-byte boundaries
// (W % 4 == 0, 4-byte aligned frames): per frame the block is 8 rows of 24
// bytes = 48 words, word m = row * 6 + u; lane l loads words l and 32 + l
// (l < 16), and each of the lane's two pixels (i = lane, lane + 32; row i / 8,
// column i % 8, bytes 24 * row + 3 * column .. + 2) is assembled from the two
// words holding it with shuffles and a funnel shift.  Two 4-byte loads per lane
// and frame instead of six byte loads.
template <int D, int PF, bool CHUNKED>
__device__ __forceinline__ bool warp_region_pass_b8(const uint8_t *__restrict__ frames, int N, int64_t fstride,
                                                    const uint8_t *blk, int W, uint32_t *tab, int chunk) {
  using C = WarpTableCfg<D>;
  constexpr bool INDEXED = C::DIRECT || CHUNKED;
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)W * 3;
  const uint32_t *wa = reinterpret_cast<const uint32_t *>(blk + (lane / 6) * row + 4 * (lane % 6));
  const int m2 = 32 + (lane & 15);
  const uint32_t *wb = reinterpret_cast<const uint32_t *>(blk + (m2 / 6) * row + 4 * (m2 % 6));
  int src[2][2], sh[2], hi[2][2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int i = lane + 32 * k;
    const int o = (i >> 3) * 24 + 3 * (i & 7);
    const int w0 = o >> 2;
    sh[k] = 8 * (o & 3);
    src[k][0] = w0 & 31, hi[k][0] = w0 >> 5;
    src[k][1] = (w0 + 1) & 31, hi[k][1] = (w0 + 1) >> 5;
  }
  uint32_t inserted = 0;
  const int64_t fwords = fstride / 4;
  for (int f0 = 0; f0 < N; f0 += PF) {
    uint32_t a[PF], bw[PF];
#pragma unroll
    for (int j = 0; j < PF; ++j)
      if (f0 + j < N) {
        a[j] = __ldg(wa + (int64_t)(f0 + j) * fwords);
        bw[j] = lane < 16 ? __ldg(wb + (int64_t)(f0 + j) * fwords) : 0u;
      }
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      if (f0 + j >= N) break;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const uint32_t l0 = __shfl_sync(0xFFFFFFFFu, a[j], src[k][0]), h0 = __shfl_sync(0xFFFFFFFFu, bw[j], src[k][0]);
        const uint32_t l1 = __shfl_sync(0xFFFFFFFFu, a[j], src[k][1]), h1 = __shfl_sync(0xFFFFFFFFu, bw[j], src[k][1]);
        const uint32_t lo = hi[k][0] ? h0 : l0, up = hi[k][1] ? h1 : l1;
        const uint32_t q = planar_code<D>(__funnelshift_r(lo, up, sh[k]));
        if (!CHUNKED || (int)(q >> C::LOGS) == chunk)
          inserted += warp_table_count<D, INDEXED>(tab, q, (uint32_t)(f0 + j));
      }
      __syncwarp();
      if constexpr (!INDEXED)
        if (__reduce_add_sync(0xFFFFFFFFu, inserted) > (uint32_t)(3 * C::S / 4)) return false;
    }
  }
  return true;
}

// Warp w of the caller handles regions r = r_first, r_first + r_step, ... < r_end.
// tab: this warp's S-entry table, zero on entry and on return.
template <int D, int PPL>
__device__ __forceinline__ void build_block_warp_body(const uint8_t *__restrict__ frames, int N, int H, int W, int b,
                                                      int bw, uint32_t T, uint32_t *__restrict__ model,
                                                      int64_t r_first, int64_t r_end, int64_t r_step,
                                                      uint32_t *tab) {
  using C = WarpTableCfg<D>;
  constexpr int PF = PPL >= 8 ? 2 : 16 / PPL;
  const int lane = threadIdx.x & 31;
  const int64_t fstride = (int64_t)H * W * 3;
  for (int64_t r = r_first; r < r_end; r += r_step) {
    const int y0 = (int)(r / bw) * b, x0 = (int)(r % bw) * b;
    const int h = min(b, H - y0), w = min(b, W - x0);
    const int npx = h * w;
    uint32_t off[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      const int i = lane + 32 * k;
      off[k] = i < npx ? (uint32_t)(((int64_t)(y0 + i / w) * W + x0 + i % w) * 3) : 0u;
    }
    uint32_t *row = model + r * C::WPR;
    warp_zero_row<D>(row);
    // Full 8 x 8 blocks with 4-byte aligned rows take the word-load pass at
    // depth <= 3 (at depth 4-5 its extra registers cost more occupancy than
    // the loads save: measured 0.226 / 0.252 ms vs 0.211 / 0.243 ms).
    bool fits;
    if constexpr (PPL == 2 && C::DIRECT) {
      const bool b8 = b == 8 && npx == 64 && (W & 3) == 0 && (reinterpret_cast<uintptr_t>(frames) & 3) == 0;
      const uint8_t *blk = frames + ((int64_t)y0 * W + x0) * 3;
      fits = b8 ? warp_region_pass_b8<D, PF, false>(frames, N, fstride, blk, W, tab, -1)
                : warp_region_pass<D, PPL, PF, false>(frames, N, fstride, off, npx, tab, -1);
    } else {
      fits = warp_region_pass<D, PPL, PF, false>(frames, N, fstride, off, npx, tab, -1);
    }
    if (fits) {
      warp_emit<D>(tab, row, T);
    } else {
      for (int s = lane; s < C::S; s += 32) tab[s] = 0u;
      for (int c = 0; c < C::NC / C::S; ++c) {
        __syncwarp();
        warp_region_pass<D, PPL, PF, true>(frames, N, fstride, off, npx, tab, c);
        warp_emit<D>(tab, row, T);
      }
    }
  }
}

// ---- block regions of 8 x 8 or 16 x 16 pixels, warp tiles ------------------------
// A warp covers a tile of 16 x 16 pixels: four 8 x 8 block regions or one
// 16 x 16 region.  Lane l owns the 8 consecutive pixels of tile row l / 2 in
// its left (l even) or right half, read per frame as three 8-byte loads and
// split into pixels with byte permutes, so all of a lane's pixels lie in one
// region.  The loads of the next frames are in flight while the current ones
// are counted (two register buffers of PF frames).  The table holds, per leaf
// of the region, the last frame that counted it and the number of frames that
// did (the per-frame tree of Alg. 1 holds a leaf once, however many pixels
// reach it; Alg. 2 counts trees):
//   * direct tables (depth <= 3, and depth 4 with one region per tile): a u16
//     entry (frame + 1) << 8 | count per leaf, at a bijective XOR-shuffle of the
//     leaf code (so leaves that differ only in their blue bits do not share a
//     bank) and with each region's table skewed by 8 banks.  A lane rewrites
//     its leaf's entry only while the frame field is older than the current
//     frame, so lanes holding the same leaf in the same frame store the same
//     value and the leaf is counted once per frame with no atomic;
//   * two-level tables (otherwise): a leaf of depth 4-5 is its depth-3 prefix
//     (the path's first three levels, 512 values) and a suffix (the remaining
//     levels, 8^(d-3) values).  Per region a directory maps each prefix the
//     region's pixels reach to a sub-table of u16 entries as above, one per
//     suffix, taken from a pool the warp's regions share on the prefix's first
//     touch (atomicCAS on the directory entry, then atomicAdd on the pool
//     count; a lane that finds the entry being claimed retries after the
//     frame's warp barrier).  A region's pixels reach few prefixes (a few dozen
//     at most on the synthetic scenes), so a lookup is two dependent shared
//     loads and no probing.  A region whose claim finds the pool exhausted
//     stops counting and is recounted by the chunked passes of the
//     one-warp-per-region build, so no result depends on the pool's size.
// A lane reads the entries of all its pixels of a frame before it writes any:
// the new value is a function of the old one and the frame, so a lane holding
// the same leaf twice writes the same value twice.  One __syncwarp per frame
// orders frame f's updates before frame f + 1's.
template <int D, int B>
struct BlockTileCfg {
  static constexpr int RPT = (16 / B) * (16 / B);  // regions per tile
  static constexpr int NPX = B * B;                // pixels per region
  static constexpr int NC = 1 << (3 * D);
  static constexpr bool DIRECT = D <= 3 || (D == 4 && B == 16);
  // direct tables: entries per region and between regions (8-bank skew)
  static constexpr int S = NC;
  static constexpr int SS = S + 16;
  // two-level tables: directory entries per region (depth-3 prefixes), entries
  // per sub-table (suffixes), sub-tables in the warp's pool
  static constexpr int NPRE = 512;
  static constexpr int SUB = D > 3 ? 1 << (3 * (D - 3)) : 1;
  static constexpr int SUBS = SUB + 2;  // entries between sub-tables (a one-bank skew)
  static constexpr int NP = D == 4 ? 128 : (B == 8 ? 96 : 128);  // (8 x 8 at depth 5 is not dispatched here)
  static constexpr int DIR_BYTES = RPT * NPRE * 2;
  static constexpr int POOL_BYTES = (NP * SUBS * 2 + 15) & ~15;
  static constexpr int OWNER_BYTES = NP * 2;
  static constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  static constexpr int TABLE_BYTES = DIRECT ? (RPT * SS * 2 + 15) & ~15
                                            : (DIR_BYTES + POOL_BYTES + OWNER_BYTES + 16 + 15) & ~15;
  static constexpr int WARP_SMEM = TABLE_BYTES + 16;  // + RPT per-region flags
  static constexpr int WPC = DIRECT ? 8 : 4;  // warps per CTA
  // CTAs resident per SM the kernel is compiled for (registers; two-level
  // tables at depth 5 fit 3 CTAs in shared memory)
  static constexpr int MINB = DIRECT ? 3 : (D == 4 ? 4 : 3);
  static constexpr int PF = DIRECT ? 4 : 2;  // frames per register buffer
  static_assert(DIRECT || TABLE_BYTES >= 4096, "the recount passes use a 4 KB table");
};

// Planar code of a masked pixel word (bytes r_d, g_d, b_d; byte 3 ignored)
// with one byte dot product at every depth <= 5.
template <int D>
__device__ __forceinline__ uint32_t planar_dp(uint32_t t) {
  if constexpr (D <= 3)
    return __dp4a(t, 1u | ((1u << D) << 8) | ((1u << (2 * D)) << 16), 0u);
  else
    return __dp4a(t, 1u | ((1u << D) << 8), (t >> (16 - 2 * D)) & (0xFFu << (2 * D)));
}

// Slot of leaf q in a direct table: a bijection of [0, 2^15) (each bit XORed
// with higher bits only).
__device__ __forceinline__ uint32_t tile_slot(uint32_t q) { return q ^ (q >> 5) ^ (q >> 10); }

// Packed pixel k (0..7) of 24 bytes held as 6 words.
template <int K>
__device__ __forceinline__ uint32_t oct_pixel(const uint32_t (&w)[6]) {
  constexpr int o = 3 * K, i = o / 4, s = o % 4;
  constexpr uint32_t sel = (uint32_t)(s | ((s + 1) << 4) | ((s + 2) << 8) | ((s + 2) << 12));
  if constexpr (i + 1 < 6)
    return __byte_perm(w[i], w[i + 1], sel);
  else
    return __byte_perm(w[i], 0u, sel);
}

// Two-level tables: the sub-table (1-based) of prefix p in directory `dir`,
// claiming one from the pool on the prefix's first touch; 0 when the entry is
// being claimed by another lane (retry after the frame's warp barrier) or the
// pool is exhausted (the region's flag is raised).
template <int D, int B>
__device__ __forceinline__ uint32_t tile_claim(uint16_t *dir, uint32_t p, int ri, uint32_t *pcount, uint16_t *owner,
                                               uint32_t *flag) {
  using C = BlockTileCfg<D, B>;
  const unsigned short old = atomicCAS(reinterpret_cast<unsigned short *>(dir + p), (unsigned short)0,
                                       (unsigned short)0xFFFF);
  if (old == 0) {
    const uint32_t j = atomicAdd(pcount, 1u);
    if (j < (uint32_t)C::NP) {
      owner[j] = (uint16_t)((ri << 9) | p);
      *reinterpret_cast<volatile uint16_t *>(dir + p) = (uint16_t)(j + 1);
      return j + 1;
    }
    atomicOr(flag, 1u);  // pool exhausted: recount the region
    return 0;
  }
  return old == 0xFFFF ? 0u : (uint32_t)old;
}

// Planar code of depth D from a depth-3 prefix and its suffix.
template <int D>
__device__ __forceinline__ uint32_t tile_compose(uint32_t p, uint32_t s) {
  constexpr int E = D - 3;
  constexpr uint32_t M = (1u << E) - 1u;
  const uint32_t r = ((p & 7u) << E) | (s & M), g = (((p >> 3) & 7u) << E) | ((s >> E) & M),
                 b = ((p >> 6) << E) | (s >> (2 * E));
  return r | (g << D) | (b << (2 * D));
}

// Warp w of the caller handles tiles t = t_first, t_first + t_step, ... < t_end
// (row-major over ceil(H/16) x ceil(W/16) tiles).  Needs b in {8, 16},
// W % 8 == 0, 8-byte aligned frames, N <= 255, H*W*3 < 2^32.
// wsm: this warp's WARP_SMEM bytes (16-byte aligned), zero on entry and on return.
template <int D, int B, int PF>
__device__ __forceinline__ void build_block_tile_body(const uint8_t *__restrict__ frames, int N, int H, int W, int bw,
                                                      uint32_t T, uint32_t *__restrict__ model, int64_t t_first,
                                                      int64_t t_end, int64_t t_step, uint8_t *wsm) {
  using C = BlockTileCfg<D, B>;
  const int lane = threadIdx.x & 31;
  const int trow = lane >> 1, half = lane & 1;
  const int tiles_x = (W + 15) >> 4;
  const int64_t fstride = (int64_t)H * W * 3;
  const int ri = B == 8 ? (((trow >> 3) << 1) | half) : 0;  // the lane's region within the tile
  uint32_t *flags = reinterpret_cast<uint32_t *>(wsm + C::TABLE_BYTES);  // per region: recount
  uint16_t *t16 = reinterpret_cast<uint16_t *>(wsm) + ri * C::SS;           // direct
  uint16_t *dir = reinterpret_cast<uint16_t *>(wsm) + ri * C::NPRE;         // two-level
  uint16_t *pool = reinterpret_cast<uint16_t *>(wsm + C::DIR_BYTES);
  uint16_t *owner = reinterpret_cast<uint16_t *>(wsm + C::DIR_BYTES + C::POOL_BYTES);
  uint32_t *pcount = reinterpret_cast<uint32_t *>(wsm + C::DIR_BYTES + C::POOL_BYTES + C::OWNER_BYTES);
  for (int64_t t = t_first; t < t_end; t += t_step) {
    const int ty = (int)(t / tiles_x), tx = (int)(t - (int64_t)ty * tiles_x);
    const int y = ty * 16 + trow, x = tx * 16 + half * 8;
    const bool active = y < H && x < W;
    const uint8_t *src = frames + ((int64_t)y * W + x) * 3;
    bool skip = !active;
    auto load = [&](uint32_t (&v)[PF][6], int f0) {
#pragma unroll
      for (int j = 0; j < PF; ++j)
        if (active && f0 + j < N) {
          const uint2 *s = reinterpret_cast<const uint2 *>(src + (int64_t)(f0 + j) * fstride);
          const uint2 a = __ldg(s), b = __ldg(s + 1), c = __ldg(s + 2);
          v[j][0] = a.x, v[j][1] = a.y, v[j][2] = b.x, v[j][3] = b.y, v[j][4] = c.x, v[j][5] = c.y;
        }
    };
    auto count = [&](const uint32_t (&v)[PF][6], int f0) {
#pragma unroll
      for (int j = 0; j < PF; ++j) {
        if (f0 + j >= N) break;
        const uint32_t fh = (uint32_t)(f0 + j + 1) << 8;
        uint32_t m[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) m[i] = (v[j][i] >> (8 - D)) & byte_mask(D);
        if constexpr (C::DIRECT) {
          if (!skip) {
            uint32_t q[8];
            static_for<0, 8>([&](auto kc) {
              constexpr int k = decltype(kc)::value;
              q[k] = planar_dp<D>(oct_pixel<k>(m));
            });
            volatile uint16_t *vt = t16;
            uint32_t e[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) e[k] = vt[tile_slot(q[k])];
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (e[k] < fh) vt[tile_slot(q[k])] = (uint16_t)(fh | ((e[k] + 1u) & 0xFFu));
          }
          __syncwarp();
        } else {
          // prefix: the top 3 of the D bits per channel; suffix: the rest
          constexpr int E = D - 3;
          uint32_t pre[8], suf[8], sub[8];
          uint32_t deferred = 0;
          if (!skip) {
            static_for<0, 8>([&](auto kc) {
              constexpr int k = decltype(kc)::value;
              const uint32_t px = oct_pixel<k>(m);
              pre[k] = __dp4a((px >> E) & byte_mask(3), 1u | (8u << 8) | (64u << 16), 0u);
              suf[k] = __dp4a(px & byte_mask(E), 1u | ((1u << E) << 8) | ((1u << (2 * E)) << 16), 0u);
            });
            volatile uint16_t *vd = dir;
#pragma unroll
            for (int k = 0; k < 8; ++k) sub[k] = vd[pre[k]];
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (sub[k] == 0u || sub[k] == 0xFFFFu) {
                sub[k] = tile_claim<D, B>(dir, pre[k], ri, pcount, owner, flags + ri);
                if (!sub[k]) deferred |= 1u << k;
              }
            volatile uint16_t *vp = pool;
            uint32_t e[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (!((deferred >> k) & 1u)) e[k] = vp[(sub[k] - 1u) * C::SUBS + suf[k]];
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (!((deferred >> k) & 1u) && e[k] < fh)
                vp[(sub[k] - 1u) * C::SUBS + suf[k]] = (uint16_t)(fh | ((e[k] + 1u) & 0xFFu));
          }
          __syncwarp();
          // pixels whose prefix another lane was claiming: its directory entry
          // is set now (or the pool ran out and the region is recounted)
          if (__any_sync(0xFFFFFFFFu, deferred != 0u)) {
            if (deferred && !*(volatile uint32_t *)(flags + ri)) {
              volatile uint16_t *vd = dir;
              volatile uint16_t *vp = pool;
#pragma unroll
              for (int k = 0; k < 8; ++k)
                if ((deferred >> k) & 1u) {
                  const uint32_t sb = vd[pre[k]];
                  if (sb == 0u || sb == 0xFFFFu) continue;  // unreachable unless the region overflowed
                  const uint32_t e = vp[(sb - 1u) * C::SUBS + suf[k]];
                  if (e < fh) vp[(sb - 1u) * C::SUBS + suf[k]] = (uint16_t)(fh | ((e + 1u) & 0xFFu));
                }
            }
            __syncwarp();
          }
          skip = skip || *(volatile uint32_t *)(flags + ri) != 0u;
        }
      }
    };
    {
      uint32_t va[PF][6], vb[PF][6];
      load(va, 0);
      for (int f0 = 0; f0 < N; f0 += 2 * PF) {
        load(vb, f0 + PF);
        count(va, f0);
        if (f0 + PF >= N) break;
        load(va, f0 + 2 * PF);
        count(vb, f0 + PF);
      }
    }
    __syncwarp();
    // Emit the tile's regions (a region is absent when its top-left pixel lies
    // outside the frame).
    auto ry0 = [&](int r) { return ty * 16 + (B == 8 ? (r >> 1) * 8 : 0); };
    auto rx0 = [&](int r) { return tx * 16 + (B == 8 ? (r & 1) * 8 : 0); };
    auto region_row = [&](int r) -> uint32_t * {
      const int y0 = ry0(r), x0 = rx0(r);
      if (y0 >= H || x0 >= W) return nullptr;
      return model + ((int64_t)(y0 / B) * bw + x0 / B) * C::WPR;
    };
    if constexpr (C::DIRECT) {
      // Word wd of region r's row: leaves 32 wd .. 32 wd + 31.
      constexpr int EPW = C::NC < 32 ? C::NC : 32;
      for (int g = lane; g < C::RPT * C::WPR; g += 32) {
        const int r = g / C::WPR, wd = g - r * C::WPR;
        const uint16_t *tr = reinterpret_cast<const uint16_t *>(wsm) + r * C::SS;
        uint32_t bits = 0;
#pragma unroll 8
        for (int i = 0; i < EPW; ++i) bits |= (uint32_t)((tr[tile_slot((uint32_t)(32 * wd + i))] & 0xFFu) >= T) << i;
        uint32_t *row = region_row(r);
        if (row) row[wd] = bits;
      }
      __syncwarp();
      uint4 *z = reinterpret_cast<uint4 *>(wsm);
      for (int i = lane; i < C::TABLE_BYTES / 16; i += 32) z[i] = make_uint4(0, 0, 0, 0);
      __syncwarp();
    } else {
      uint32_t ovf = 0;  // regions to recount
#pragma unroll
      for (int r = 0; r < C::RPT; ++r) {
        uint32_t *row = region_row(r);
        if (row && *(volatile uint32_t *)(flags + r)) ovf |= 1u << r;
        if (row) {
          uint4 *r4 = reinterpret_cast<uint4 *>(row);
          for (int i = lane; i < C::WPR / 4; i += 32) r4[i] = make_uint4(0, 0, 0, 0);
        }
      }
      __syncwarp();
      const uint32_t used = min(*(volatile uint32_t *)pcount, (uint32_t)C::NP);
      for (uint32_t i = lane; i < used * C::SUB; i += 32) {
        const uint32_t jt = i / C::SUB, sx = i - jt * C::SUB;
        const uint32_t e = pool[jt * C::SUBS + sx];
        if (e) {
          pool[jt * C::SUBS + sx] = 0;
          const uint32_t o = owner[jt];
          const int r = (int)(o >> 9);
          uint32_t *row = region_row(r);
          if (row && !((ovf >> r) & 1u) && (e & 0xFFu) >= T) {
            const uint32_t q = tile_compose<D>(o & 511u, sx);
            atomicOr(&row[q >> 5], 1u << (q & 31));
          }
        }
      }
      uint4 *z = reinterpret_cast<uint4 *>(wsm);  // the directories
      for (int i = lane; i < C::DIR_BYTES / 16; i += 32) z[i] = make_uint4(0, 0, 0, 0);
      if (lane == 0) *pcount = 0u;
      __syncwarp();
      // Recount regions whose pool claim failed: chunked direct passes over
      // 1024-leaf slices of the code space (table = the first 4 KB of wsm,
      // zero after the clearing above).
      uint32_t *tab = reinterpret_cast<uint32_t *>(wsm);
      while (ovf) {
        const int r = __ffs(ovf) - 1;
        ovf &= ovf - 1;
        uint32_t *row = region_row(r);
        const int y0 = ry0(r), x0 = rx0(r);
        const int h = min(B, H - y0), w = min(B, W - x0), npx = h * w;
        constexpr int PPL = C::NPX / 32;
        uint32_t off[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
          const int i = lane + 32 * k;
          off[k] = i < npx ? (uint32_t)(((int64_t)(y0 + i / w) * W + x0 + i % w) * 3) : 0u;
        }
        for (int c = 0; c < WarpTableCfg<D>::NC / WarpTableCfg<D>::S; ++c) {
          __syncwarp();
          warp_region_pass<D, PPL, 4, true>(frames, N, fstride, off, npx, tab, c);
          warp_emit<D>(tab, row, T);
        }
      }
      if (lane < C::RPT) flags[lane] = 0u;
      __syncwarp();
    }
  }
}

// ---- block regions, frames split over the warps of a CTA --------------------
// Sec. 3 regions with the N training frames dealt to the 8 warps of a CTA, so
// that a region's frames are counted in parallel (and a frame of few regions
// still fills the GPU).  The CTA's shared memory holds, per region of its
// group: u8 leaf counters (frame counts, N <= 255), the model row being built
// (a leaf's bit is set when its count reaches T) and, at depth 5, one bit per
// 16 counters marking the counters to clear; per warp and region: the leaf
// bitset of the frame it is counting (the per-frame "stored once" of Alg. 1,
// so that a frame adds at most one to a leaf's count, Alg. 2).
// Groups: 16 x 16 pixel tiles (one 16 x 16 or four 8 x 8 regions; a warp takes
// one frame of the tile, 8 pixels per lane as in the warp tiles) or, for 8 x 8
// regions at depth 5, single regions (a warp takes one frame of the region,
// 2 pixels per lane), which keeps the counters at 32 KB per CTA.
template <int D, int B>
struct BlockFsCfg {
  static constexpr bool TILE = !(B == 8 && D == 5);
  static constexpr int RPT = TILE ? (16 / B) * (16 / B) : 1;  // regions per group
  static constexpr int NC = 1 << (3 * D);
  static constexpr int CW = NC / 4;                 // counter words per region
  static constexpr int BW = NC >= 32 ? NC / 32 : 1;  // model row words (leaf bitset)
  static constexpr bool TOUCH = D >= 5;              // clear only the touched counters
  static constexpr int TW = TOUCH ? NC / 512 : 0;    // touch words per region
  static constexpr int WPC = 8;
  static constexpr bool FILTER = false;
  static constexpr int CNT_OFF = 0;
  static constexpr int MB_OFF = RPT * CW;
  static constexpr int TOUCH_OFF = MB_OFF + RPT * BW;
  static constexpr int FB_OFF = TOUCH_OFF + RPT * TW;
  static constexpr int WORDS = FB_OFF + WPC * RPT * BW;
  static constexpr int SMEM = ((WORDS * 4) + 15) & ~15;
  static constexpr int MINB = D >= 5 ? 3 : 4;
  static constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  static_assert(WPR == BW, "model rows are one bit per leaf");
};

// Counts one masked leaf code q of the warp's current frame: sets its bit in
// the frame bitset fb; the first pixel of the frame with this leaf adds one to
// its counter, marks the counter group touched and, when the count reaches T,
// sets the leaf's bit in the model row image mb.  A plain read of fb first
// keeps the lanes of a uniform patch from queueing on one atomic (a stale
// read only costs the atomic, whose result decides).
template <int D, int B>
__device__ __forceinline__ void fs_count_leaf(uint32_t q, uint32_t *fb, uint32_t *cnt, uint32_t *mb,
                                              uint32_t *touch, uint32_t T) {
  const uint32_t bit = 1u << (q & 31u);
  if (BlockFsCfg<D, B>::FILTER && (reinterpret_cast<volatile uint32_t *>(fb)[q >> 5] & bit)) return;
  const uint32_t old = atomicOr(fb + (q >> 5), bit);
  if (!(old & bit)) {
    const uint32_t sh = (q & 3u) << 3;
    const uint32_t c = (atomicAdd(cnt + (q >> 2), 1u << sh) >> sh) & 0xFFu;
    if constexpr (BlockFsCfg<D, B>::TOUCH)
      if (c == 0u) atomicOr(touch + (q >> 9), 1u << ((q >> 4) & 31u));
    if (c + 1u == T) atomicOr(mb + (q >> 5), bit);
  }
}

// CTA vb of vg handles groups vb, vb + vg, ... < ngroups (tiles row-major over
// ceil(H/16) x ceil(W/16), or 8 x 8 regions row-major).  Needs b in {8, 16},
// W % 8 == 0, 8-byte aligned frames, 1 <= T <= N <= 255, H*W*3 < 2^32, and
// blockDim.x == 256.  sm: BlockFsCfg::SMEM bytes, zero on entry and on return.
template <int D, int B>
__device__ __forceinline__ void build_block_fs_body(const uint8_t *__restrict__ frames, int N, int H, int W, int bw,
                                                    uint32_t T, uint32_t *__restrict__ model, int64_t ngroups,
                                                    int64_t vb, int64_t vg, uint32_t *sm) {
  using C = BlockFsCfg<D, B>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t fstride = (int64_t)H * W * 3;
  uint32_t *cnt = sm + C::CNT_OFF, *mb = sm + C::MB_OFF, *touch = sm + C::TOUCH_OFF;
  // lane geometry within a group
  int ly, lx, ri;
  if constexpr (C::TILE) {
    ly = lane >> 1, lx = (lane & 1) * 8;
    ri = B == 8 ? (((lane >> 4) << 1) | (lane & 1)) : 0;
  } else {
    ly = lane >> 2, lx = (lane & 3) * 2;
    ri = 0;
  }
  uint32_t *fb = sm + C::FB_OFF + (warp * C::RPT + ri) * C::BW;
  uint32_t *cr = cnt + ri * C::CW, *mr = mb + ri * C::BW, *tr = touch + ri * C::TW;
  const int gx = C::TILE ? (W + 15) >> 4 : bw;
  constexpr int GS = C::TILE ? 16 : 8;  // group side in pixels
  constexpr int NW = C::TILE ? 6 : 2;   // words a lane loads per frame
  // Where the lane's pixels of group g start (tile lanes read 24 bytes at an
  // 8-byte boundary; region lanes read the two words holding bytes 6j .. 6j + 5
  // of their row, j = lane & 3), and whether they lie in the frame.
  struct Geo {
    const uint8_t *src;
    uint32_t sel;
    bool active;
  };
  auto geo = [&](int64_t g) {
    Geo o{frames, 0u, false};
    if (g < ngroups) {
      const int gy = (int)(g / gx), gxi = (int)(g - (int64_t)gy * gx);
      const int y = gy * GS + ly, x = gxi * GS + lx;
      o.active = y < H && x < W;
      const int64_t pofs = ((int64_t)y * W + x) * 3;
      o.src = frames + (C::TILE ? pofs : (pofs & ~(int64_t)3));
      o.sel = C::TILE ? 0u : (uint32_t)(pofs & 3);
    }
    return o;
  };
  auto load = [&](uint32_t (&v)[NW], const Geo &o, int f) {
    if (o.active && f < N) {
      const uint8_t *s = o.src + (int64_t)f * fstride;
      if constexpr (C::TILE) {
        const uint2 a = __ldg(reinterpret_cast<const uint2 *>(s)), b2 = __ldg(reinterpret_cast<const uint2 *>(s) + 1),
                    c2 = __ldg(reinterpret_cast<const uint2 *>(s) + 2);
        v[0] = a.x, v[1] = a.y, v[2] = b2.x, v[3] = b2.y, v[4] = c2.x, v[5] = c2.y;
      } else {
        v[0] = __ldg(reinterpret_cast<const uint32_t *>(s));
        v[1] = __ldg(reinterpret_cast<const uint32_t *>(s) + 1);
      }
    }
  };
  auto count = [&](const uint32_t (&v)[NW], const Geo &o) {
    if (o.active) {
      uint32_t m[6];
#pragma unroll
      for (int i = 0; i < NW; ++i) m[i] = (v[i] >> (8 - D)) & byte_mask(D);
      if constexpr (C::TILE) {
        uint32_t q[8];
        static_for<0, 8>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          q[k] = planar_dp<D>(oct_pixel<k>(m));
        });
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k == 0 || q[k] != q[k - 1]) fs_count_leaf<D, B>(q[k], fb, cr, mr, tr, T);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; ++k) fb[q[k] >> 5] = 0u;
      } else {
        const uint32_t s0 = o.sel | ((o.sel + 1) << 4) | ((o.sel + 2) << 8), s1 = s0 + 0x333u;
        const uint32_t q0 = planar_dp<D>(__byte_perm(m[0], m[1], s0));
        const uint32_t q1 = planar_dp<D>(__byte_perm(m[0], m[1], s1));
        fs_count_leaf<D, B>(q0, fb, cr, mr, tr, T);
        if (q1 != q0) fs_count_leaf<D, B>(q1, fb, cr, mr, tr, T);
        __syncwarp();
        fb[q0 >> 5] = 0u;
        fb[q1 >> 5] = 0u;
      }
    } else {
      __syncwarp();
    }
    __syncwarp();
  };
  // Emits group g's model rows (a region is absent when its top-left pixel
  // lies outside the frame) and clears its counters.
  auto emit = [&](int64_t g) {
    const int gy = (int)(g / gx), gxi = (int)(g - (int64_t)gy * gx);
#pragma unroll
    for (int r = 0; r < C::RPT; ++r) {
      const int ry = gy * GS + (C::TILE && B == 8 ? (r >> 1) * 8 : 0);
      const int rx = gxi * GS + (C::TILE && B == 8 ? (r & 1) * 8 : 0);
      uint32_t *row = ry < H && rx < W ? model + ((int64_t)(ry / B) * bw + rx / B) * C::WPR : nullptr;
      uint32_t *m2 = mb + r * C::BW;
      if constexpr (C::BW >= 4) {
        for (int i = threadIdx.x; i < C::BW / 4; i += blockDim.x) {
          uint4 *s4 = reinterpret_cast<uint4 *>(m2) + i;
          if (row) reinterpret_cast<uint4 *>(row)[i] = *s4;
          *s4 = make_uint4(0, 0, 0, 0);
        }
      } else {
        for (int i = threadIdx.x; i < C::BW; i += blockDim.x) {
          if (row) row[i] = m2[i];
          m2[i] = 0u;
        }
      }
      uint32_t *c2 = cnt + r * C::CW;
      if constexpr (C::TOUCH) {
        // thread t clears the touched ones of counter groups 8t .. 8t + 7
        uint32_t *t2 = touch + r * C::TW;
        for (int t = threadIdx.x; t < C::CW / 32; t += blockDim.x) {
          uint32_t tb = (t2[t >> 2] >> ((t & 3) << 3)) & 0xFFu;
          while (tb) {
            const int i = __ffs(tb) - 1;
            tb &= tb - 1u;
            reinterpret_cast<uint4 *>(c2)[8 * t + i] = make_uint4(0, 0, 0, 0);
          }
        }
        __syncthreads();  // every thread has read the touch bits
        for (int t = threadIdx.x; t < C::TW; t += blockDim.x) t2[t] = 0u;
      } else {
        for (int i = threadIdx.x; i < C::CW / 4; i += blockDim.x)
          reinterpret_cast<uint4 *>(c2)[i] = make_uint4(0, 0, 0, 0);
      }
    }
  };
  // The warp's frames of a group are f = warp + 8 j; frame f + 8 is loaded
  // while f is counted, and the first frame of the next group while the
  // current group's rows are emitted.
  int64_t g = vb;
  Geo cur = geo(g);
  uint32_t v[NW];
  load(v, cur, warp);
  for (; g < ngroups; g += vg) {
    for (int f = warp; f < N; f += C::WPC) {
      uint32_t nx[NW];
      load(nx, cur, f + C::WPC);
      count(v, cur);
#pragma unroll
      for (int i = 0; i < NW; ++i) v[i] = nx[i];
    }
    const Geo next = geo(g + vg);
    load(v, next, warp);
    __syncthreads();
    emit(g);
    __syncthreads();
    cur = next;
  }
}

// ---- 8 x 8 block regions at depth 5: one region per warp, two-level tables --
// A warp counts one 8 x 8 region at a time, 2 pixels per lane (lane l: row
// l / 4, columns 2 (l % 4) and 2 (l % 4) + 1, read as the two words holding
// their 6 bytes).  The region's leaves are counted in the warp tiles'
// two-level tables (a depth-3 prefix directory, then a 64-entry sub-table per
// prefix claimed from a pool of NP; u16 entries (frame + 1, count), rewritten
// only while their frame field is older, so same-frame lanes store the same
// value): no probing, unlike the hashed one-warp-per-region table.  A region
// whose prefixes exhaust the pool is recounted by the chunked direct passes.
template <int D>
struct BlockR8CfgD {
  static_assert(D == 4 || D == 5, "two-level region tables at depth 4 or 5");
  static constexpr int E = D - 3;
  static constexpr int NPRE = 512;
  static constexpr int SUB = 1 << (3 * E), SUBS = SUB + 2;
  static constexpr int NP = D == 5 ? 32 : 128;
  static constexpr int DIR_BYTES = NPRE * 2;
  static constexpr int POOL_BYTES = (NP * SUBS * 2 + 15) & ~15;
  static constexpr int OWNER_BYTES = (NP * 2 + 15) & ~15;
  static constexpr int USED = DIR_BYTES + POOL_BYTES + OWNER_BYTES + 16;  // + pool count
  static constexpr int TABLE_BYTES = USED > 4096 ? USED : 4096;          // the recount passes use 4 KB
  static constexpr int WARP_SMEM = TABLE_BYTES + 16;                     // + overflow flag
  static constexpr int WPR = 1 << (3 * D - 5);
  static constexpr int PF = 4;
};
using BlockR8Cfg = BlockR8CfgD<5>;

// Warp w of the caller handles regions r = r_first, r_first + r_step, ... <
// r_end (row-major, bw = W / 8 per row).  Needs W % 8 == 0, 4-byte aligned
// frames, N <= 255, H*W*3 < 2^32.  wsm: this warp's WARP_SMEM bytes (16-byte
// aligned), zero on entry and on return.
// SRC = uint16_t: `frames` holds depth-5 planar leaf codes, u16 [N][H*W] (a
// serving window's per-frame occupancy); a lane's two pixels are one word.
template <int D = 5, typename SRC = uint8_t>
__device__ __forceinline__ void build_block_r8_body(const SRC *__restrict__ frames, int N, int H, int W, int bw,
                                                    uint32_t T, uint32_t *__restrict__ model, int64_t r_first,
                                                    int64_t r_end, int64_t r_step, uint8_t *wsm) {
  using C = BlockR8CfgD<D>;
  constexpr bool CODES = std::is_same<SRC, uint16_t>::value;
  constexpr int E = C::E;
  constexpr uint32_t SM = (1u << E) - 1u;
  const int lane = threadIdx.x & 31;
  const int ly = lane >> 2, lj = lane & 3;
  const int64_t fstride = (int64_t)H * W * (CODES ? 1 : 3);  // in SRC elements
  uint16_t *dir = reinterpret_cast<uint16_t *>(wsm);
  uint16_t *pool = reinterpret_cast<uint16_t *>(wsm + C::DIR_BYTES);
  uint16_t *owner = reinterpret_cast<uint16_t *>(wsm + C::DIR_BYTES + C::POOL_BYTES);
  uint32_t *pcount = reinterpret_cast<uint32_t *>(wsm + C::DIR_BYTES + C::POOL_BYTES + C::OWNER_BYTES);
  uint32_t *flag = reinterpret_cast<uint32_t *>(wsm + C::TABLE_BYTES);
  // byte selectors of the lane's two pixels within its two words
  const uint32_t sel = (uint32_t)((6 * lj) & 3);
  const uint32_t s0 = sel | ((sel + 1) << 4) | ((sel + 2) << 8), s1 = s0 + 0x333u;
  for (int64_t r = r_first; r < r_end; r += r_step) {
    const int by = (int)(r / bw), bx = (int)(r - (int64_t)by * bw);
    const int y = by * 8 + ly;
    const bool active = y < H;
    const int64_t pix = (int64_t)y * W + bx * 8 + 2 * lj;
    const int64_t pofs = CODES ? pix * 2 : pix * 3;  // bytes
    const uint32_t *src = reinterpret_cast<const uint32_t *>(reinterpret_cast<const uint8_t *>(frames) +
                                                             (pofs & ~(int64_t)3));
    const int64_t fwords = CODES ? fstride >> 1 : fstride >> 2;  // words per frame (2*H*W or H*W*3 bytes, W % 8 == 0)
    bool skip = !active;
    auto load = [&](uint32_t (&v)[C::PF][2], int f0) {
#pragma unroll
      for (int j = 0; j < C::PF; ++j)
        if (active && f0 + j < N) {
          const uint32_t *s = src + (int64_t)(f0 + j) * fwords;
          v[j][0] = __ldg(s);
          if constexpr (!CODES) v[j][1] = __ldg(s + 1);
        }
    };
    auto count = [&](const uint32_t (&v)[C::PF][2], int f0) {
#pragma unroll
      for (int j = 0; j < C::PF; ++j) {
        if (f0 + j >= N) break;
        const uint32_t fh = (uint32_t)(f0 + j + 1) << 8;
        uint32_t pre[2], suf[2], sub[2];
        uint32_t deferred = 0;
        if (!skip) {
          if constexpr (CODES) {  // q = r | g << 5 | b << 10: prefix = top 3 bits, suffix = low 2 of each
            const uint32_t q[2] = {v[j][0] & 0xFFFFu, v[j][0] >> 16};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              pre[k] = ((q[k] >> E) & 7u) | ((q[k] >> (D + E - 3)) & 0x38u) | ((q[k] >> (2 * D + E - 6)) & 0x1C0u);
              suf[k] = (q[k] & SM) | ((q[k] >> (D - E)) & (SM << E)) | ((q[k] >> (2 * D - 2 * E)) & (SM << (2 * E)));
            }
          } else {
            const uint32_t m0 = (v[j][0] >> (8 - D)) & byte_mask(D), m1 = (v[j][1] >> (8 - D)) & byte_mask(D);
            const uint32_t px[2] = {__byte_perm(m0, m1, s0), __byte_perm(m0, m1, s1)};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              pre[k] = __dp4a((px[k] >> E) & byte_mask(3), 1u | (8u << 8) | (64u << 16), 0u);
              suf[k] = __dp4a(px[k] & byte_mask(E), 1u | ((1u << E) << 8) | ((1u << (2 * E)) << 16), 0u);
            }
          }
          volatile uint16_t *vd = dir;
#pragma unroll
          for (int k = 0; k < 2; ++k) sub[k] = vd[pre[k]];
#pragma unroll
          for (int k = 0; k < 2; ++k)
            if (sub[k] == 0u || sub[k] == 0xFFFFu) {
              // claim the prefix's sub-table (0: another lane is claiming it,
              // or the pool ran out and the region is recounted)
              sub[k] = 0u;
              const unsigned short old = atomicCAS(reinterpret_cast<unsigned short *>(dir + pre[k]),
                                                   (unsigned short)0, (unsigned short)0xFFFF);
              if (old == 0) {
                const uint32_t jt = atomicAdd(pcount, 1u);
                if (jt < (uint32_t)C::NP) {
                  owner[jt] = (uint16_t)pre[k];
                  *reinterpret_cast<volatile uint16_t *>(dir + pre[k]) = (uint16_t)(jt + 1);
                  sub[k] = jt + 1;
                } else {
                  atomicOr(flag, 1u);
                }
              } else if (old != 0xFFFF) {
                sub[k] = old;
              }
              if (!sub[k]) deferred |= 1u << k;
            }
          volatile uint16_t *vp = pool;
          uint32_t e[2];
#pragma unroll
          for (int k = 0; k < 2; ++k)
            if (!((deferred >> k) & 1u)) e[k] = vp[(sub[k] - 1u) * C::SUBS + suf[k]];
#pragma unroll
          for (int k = 0; k < 2; ++k)
            if (!((deferred >> k) & 1u) && e[k] < fh)
              vp[(sub[k] - 1u) * C::SUBS + suf[k]] = (uint16_t)(fh | ((e[k] + 1u) & 0xFFu));
        }
        __syncwarp();
        if (__any_sync(0xFFFFFFFFu, deferred != 0u)) {  // their prefixes are set now (or the pool ran out)
          if (deferred && !*(volatile uint32_t *)flag) {
            volatile uint16_t *vd = dir;
            volatile uint16_t *vp = pool;
#pragma unroll
            for (int k = 0; k < 2; ++k)
              if ((deferred >> k) & 1u) {
                const uint32_t sb = vd[pre[k]];
                if (sb == 0u || sb == 0xFFFFu) continue;  // unreachable unless the region overflowed
                const uint32_t ee = vp[(sb - 1u) * C::SUBS + suf[k]];
                if (ee < fh) vp[(sb - 1u) * C::SUBS + suf[k]] = (uint16_t)(fh | ((ee + 1u) & 0xFFu));
              }
          }
          __syncwarp();
        }
        skip = skip || *(volatile uint32_t *)flag != 0u;
      }
    };
    {
      uint32_t va[C::PF][2], vb[C::PF][2];
      load(va, 0);
      for (int f0 = 0; f0 < N; f0 += 2 * C::PF) {
        load(vb, f0 + C::PF);
        count(va, f0);
        if (f0 + C::PF >= N) break;
        load(va, f0 + 2 * C::PF);
        count(vb, f0 + C::PF);
      }
    }
    __syncwarp();
    // Emit: the row zeroed, then the kept leaves' bits; the tables cleared.
    uint32_t *row = model + r * C::WPR;
    const bool ovf = *(volatile uint32_t *)flag != 0u;
    {
      uint4 *r4 = reinterpret_cast<uint4 *>(row);
      for (int i = lane; i < C::WPR / 4; i += 32) r4[i] = make_uint4(0, 0, 0, 0);
    }
    __syncwarp();
    const uint32_t used = min(*(volatile uint32_t *)pcount, (uint32_t)C::NP);
    for (uint32_t i = lane; i < used * C::SUB; i += 32) {
      const uint32_t jt = i / C::SUB, sx = i - jt * C::SUB;
      const uint32_t e = pool[jt * C::SUBS + sx];
      if (e) {
        pool[jt * C::SUBS + sx] = 0;
        if (!ovf && (e & 0xFFu) >= T) {
          const uint32_t q = tile_compose<D>(owner[jt], sx);
          atomicOr(&row[q >> 5], 1u << (q & 31));
        }
      }
    }
    {
      uint4 *z = reinterpret_cast<uint4 *>(wsm);  // the directory
      for (int i = lane; i < C::DIR_BYTES / 16; i += 32) z[i] = make_uint4(0, 0, 0, 0);
    }
    if (lane == 0) *pcount = 0u;
    __syncwarp();
    if (ovf) {  // chunked direct passes over 1024-leaf slices (table = the first 4 KB of wsm)
      uint32_t *tab = reinterpret_cast<uint32_t *>(wsm);
      {  // at depth 4 the sub-tables' owners lie in those 4 KB too
        uint4 *z = reinterpret_cast<uint4 *>(wsm);
        for (int i = lane; i < 4096 / 16; i += 32) z[i] = make_uint4(0, 0, 0, 0);
      }
      __syncwarp();
      const int x0 = bx * 8, h = min(8, H - by * 8), npx = h * 8;
      uint32_t off[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int i = lane + 32 * k;
        off[k] = i < npx ? (uint32_t)(((int64_t)(by * 8 + i / 8) * W + x0 + i % 8) * (CODES ? 1 : 3)) : 0u;
      }
      for (int c = 0; c < WarpTableCfg<D>::NC / WarpTableCfg<D>::S; ++c) {
        __syncwarp();
        warp_region_pass<D, 2, 4, true, SRC>(frames, N, fstride, off, npx, tab, c);
        warp_emit<D>(tab, row, T);
      }
      if (lane == 0) *flag = 0u;
      __syncwarp();
    }
  }
}

// ---- pixel regions, depth <= 3 -------------------------------------------------
// Thread t of a 128-thread CTA owns pixel location p and a private column of
// counter words cnt[k * 128 + t] (4 u8 or 2 u16 counters per word).
template <int D, bool WIDE>
__device__ __forceinline__ void build_pixel_counters_body(const uint8_t *__restrict__ frames, int N, int64_t hw,
                                                          int64_t p_begin, uint32_t T, uint32_t *__restrict__ model,
                                                          int64_t vb) {
  constexpr int NC = 1 << (3 * D);
  constexpr int CPW = WIDE ? 2 : 4;
  constexpr int BITS = 32 / CPW;
  constexpr int NW = (NC + CPW - 1) / CPW;
  constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  extern __shared__ uint32_t cnt[];
  const int t = threadIdx.x;
  const int64_t p = p_begin + vb * 128 + t;
  if (t >= 128 || p >= hw) return;  // columns are private: no CTA-wide synchronisation below
#pragma unroll 8
  for (int k = 0; k < NW; ++k) cnt[k * 128 + t] = 0;
  const uint8_t *px = frames + p * 3;
  const int64_t fstride = hw * 3;
  int f = 0;
  for (; f + 4 <= N; f += 4) {
    uint32_t q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint8_t *s = px + (int64_t)(f + u) * fstride;
      q[u] = planar_code_rt(__ldg(s), __ldg(s + 1), __ldg(s + 2), D);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) cnt[(q[u] / CPW) * 128 + t] += 1u << ((q[u] % CPW) * BITS);
  }
  for (; f < N; ++f) {
    const uint8_t *s = px + (int64_t)f * fstride;
    const uint32_t q = planar_code_rt(__ldg(s), __ldg(s + 1), __ldg(s + 2), D);
    cnt[(q / CPW) * 128 + t] += 1u << ((q % CPW) * BITS);
  }
  uint32_t out[WPR];
#pragma unroll
  for (int w = 0; w < WPR; ++w) out[w] = 0;
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    const uint32_t v = cnt[k * 128 + t];
    uint32_t bits;
    if constexpr (WIDE) {
      const uint32_t ge = __vcmpgeu2(v, T * 0x00010001u);
      bits = ((ge >> 15) & 1u) | ((ge >> 30) & 2u);
    } else {
      const uint32_t ge = __vcmpgeu4(v, T * 0x01010101u);
      bits = ((ge >> 7) & 1u) | ((ge >> 14) & 2u) | ((ge >> 21) & 4u) | ((ge >> 28) & 8u);
    }
    const int c0 = k * CPW;  // first leaf of this counter word
    if (c0 < NC) out[c0 >> 5] |= bits << (c0 & 31);
  }
  if (NC < 32) out[0] &= (NC < 32 ? ((1u << NC) - 1u) : 0xFFFFFFFFu);
  uint32_t *dst = model + p * WPR;
#pragma unroll
  for (int w = 0; w < WPR; ++w) dst[w] = out[w];
}

// ---- pixel regions, depth >= 4 --------------------------------------------------
// Counts leaves chunk by chunk (512 leaves, u16 counters in a private column
// of 256 words) for the chunks the pixel's training colours touch.  `touched`
// is a per-pixel chunk bitmap in global scratch (depth >= 6) or a register.
template <int D>
__device__ __forceinline__ void build_pixel_chunked_body(const uint8_t *__restrict__ frames, int N, int64_t hw,
                                                         uint32_t T, uint32_t *__restrict__ model,
                                                         uint32_t *__restrict__ touched_g, int64_t vb) {
  constexpr int NCH = 1 << (3 * D - 9);
  constexpr int WPR = 1 << (3 * D - 5);
  constexpr int TW = NCH / 32 > 0 ? NCH / 32 : 1;  // touched words per pixel (global form)
  extern __shared__ uint32_t cnt[];                 // [256][64]
  const int t = threadIdx.x;
  const int64_t p = vb * 64 + t;
  if (t >= 64 || p >= hw) return;
  const uint8_t *px = frames + p * 3;
  const int64_t fstride = hw * 3;
  uint64_t touched = 0;
  uint32_t *tg = touched_g ? touched_g + p * TW : nullptr;
  for (int f = 0; f < N; ++f) {
    const uint8_t *s = px + (int64_t)f * fstride;
    const uint32_t q = planar_code_rt(__ldg(s), __ldg(s + 1), __ldg(s + 2), D);
    const uint32_t c = q >> 9;
    if constexpr (NCH <= 64)
      touched |= 1ull << c;
    else
      tg[c >> 5] |= 1u << (c & 31);
  }
  uint32_t *row = model + p * WPR;
  int tw = 0;
  uint32_t cur = 0;
  while (true) {
    int c;
    if constexpr (NCH <= 64) {
      if (!touched) break;
      c = __ffsll((long long)touched) - 1;
      touched &= touched - 1;
    } else {
      while (!cur && tw < TW) cur = tg[tw++];
      if (!cur) break;
      c = (tw - 1) * 32 + __ffs(cur) - 1;
      cur &= cur - 1;
    }
    for (int k = 0; k < 256; ++k) cnt[k * 64 + t] = 0;
    for (int f = 0; f < N; ++f) {
      const uint8_t *s = px + (int64_t)f * fstride;
      const uint32_t q = planar_code_rt(__ldg(s), __ldg(s + 1), __ldg(s + 2), D);
      if ((int)(q >> 9) == c) cnt[((q & 511u) >> 1) * 64 + t] += 1u << ((q & 1u) * 16);
    }
    for (int w = 0; w < 16; ++w) {
      uint32_t out = 0;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const uint32_t ge = __vcmpgeu2(cnt[(w * 16 + k) * 64 + t], T * 0x00010001u);
        out |= (((ge >> 15) & 1u) | ((ge >> 30) & 2u)) << (2 * k);
      }
      row[c * 16 + w] = out;
    }
  }
}

// ---- pixel regions, any depth: frequent-leaf candidates ---------------------------
// A pixel location sees one leaf per frame, so its N leaves can hold at most
// k = floor(N / T) leaves that occur in T or more frames.  Pass 1 keeps a
// Misra-Gries summary of KM >= k counters over the pixel's leaves (every leaf
// seen more than N / (KM + 1) < T times keeps a non-zero counter, so every leaf
// to be kept is among the KM candidates) and stores the leaves in shared
// memory; pass 2 counts each candidate exactly.  KM = 0 (large k): pass 2
// instead counts every distinct leaf at its first occurrence.  With one tree
// per group of frames the same bound holds for the stream of leaves taken once
// per group, which is what the summary then sees.  The warp then
// writes its 32 pixels' rows, which are contiguous: zeros with vector stores,
// then the kept words.  Lane = pixel; the frames are read once and the model
// written once, whatever the depth.  With candidates (KM > 0) at depth <= 5,
// `kept` (if not null) also receives each location's kept leaves as 8 u16
// codes padded with kKeptNone: the kept-leaf index of the classify; model =
// null (a list model) then writes no rows at all.
template <int D>
using leaf_t = typename std::conditional<(D <= 5), uint16_t, uint32_t>::type;

template <int D, int KM, bool GRP = false, bool CODES = false>
__device__ __forceinline__ void build_pixel_mg_body(const uint8_t *__restrict__ frames, int N, int64_t hw, uint32_t T,
                                                    uint32_t *__restrict__ model, int64_t tile, leaf_t<D> *codes,
                                                    int group = 1, uint16_t *kept = nullptr) {
  // GRP: one tree per group of `group` consecutive frames (Sec. 3): a leaf
  // enters the summary once per group that holds it, and the exact pass counts
  // the groups holding each candidate (T counts groups).
  // CODES: `frames` holds planar leaf codes, u16 [N][hw] (depth <= 5), the
  // per-frame occupancy a serving window keeps, instead of RGB bytes.
  constexpr int64_t WPR = D == 1 ? 1 : (int64_t)1 << (3 * D - 5);
  constexpr int PF = 8;
  const int lane = threadIdx.x & 31;
  const int64_t p0 = tile * 32, p = p0 + lane;
  const bool valid = p < hw;
  const uint8_t *px = frames + (valid ? p : 0) * 3;
  const int64_t fstride = hw * 3;
  // a counter at zero holds the key kNoKey, which no leaf code equals, so a
  // key match alone tells a live candidate
  constexpr uint32_t kNoKey = 0xFFFFFFFFu;
  uint32_t key[KM > 0 ? KM : 1], cnt[KM > 0 ? KM : 1];
#pragma unroll
  for (int i = 0; i < (KM > 0 ? KM : 1); ++i) key[i] = kNoKey, cnt[i] = 0u;
  for (int f0 = 0; f0 < N; f0 += PF) {
    uint32_t yv[PF];
#pragma unroll
    for (int j = 0; j < PF; ++j)
      if (valid && f0 + j < N) {
        if constexpr (CODES) {
          yv[j] = __ldg(reinterpret_cast<const uint16_t *>(frames) + (int64_t)(f0 + j) * hw + p);
        } else {
          const uint8_t *s = px + (int64_t)(f0 + j) * fstride;
          yv[j] = (uint32_t)__ldg(s) | ((uint32_t)__ldg(s + 1) << 8) | ((uint32_t)__ldg(s + 2) << 16);
        }
      }
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      if (!valid || f0 + j >= N) break;
      const int f = f0 + j;
      const uint32_t q = CODES ? yv[j] : planar_code<D>(yv[j]);
      codes[f * 32 + lane] = (leaf_t<D>)q;
      if constexpr (KM > 0) {
        bool seen = false;
        if constexpr (GRP)
          for (int e = f - f % group; e < f && !seen; ++e) seen = codes[e * 32 + lane] == q;
        if (!seen) {
          bool hit = false;
#pragma unroll
          for (int i = 0; i < KM; ++i)
            if (key[i] == q) ++cnt[i], hit = true;
          if (!hit) {
            bool placed = false;
#pragma unroll
            for (int i = 0; i < KM; ++i)
              if (!placed && !cnt[i]) key[i] = q, cnt[i] = 1u, placed = true;
            if (!placed) {  // every counter is >= 1 here
#pragma unroll
              for (int i = 0; i < KM; ++i)
                if (--cnt[i] == 0u) key[i] = kNoKey;
            }
          }
        }
      }
    }
  }
  uint32_t exact[KM > 0 ? KM : 1];
  if constexpr (KM > 0) {
    int last[KM];
#pragma unroll
    for (int i = 0; i < KM; ++i) exact[i] = 0u, last[i] = -1;
    if (valid)
      for (int f = 0; f < N; ++f) {
        const uint32_t q = codes[f * 32 + lane];
        if constexpr (GRP) {  // count each group once
          const int g = f / group;
#pragma unroll
          for (int i = 0; i < KM; ++i)
            if (key[i] == q && last[i] != g) ++exact[i], last[i] = g;
        } else {  // one leaf per frame: a frame matches a key at most once
#pragma unroll
          for (int i = 0; i < KM; ++i)
            if (key[i] == q) ++exact[i];
        }
      }
  }
  const int64_t np = hw - p0 < 32 ? hw - p0 : 32;
  uint32_t *base = model ? model + p0 * WPR : nullptr;  // null: a list model, no rows
  if (base) {
    if constexpr (WPR >= 4) {
      uint4 *b4 = reinterpret_cast<uint4 *>(base);
      for (int64_t i = lane; i < np * WPR / 4; i += 32) b4[i] = make_uint4(0, 0, 0, 0);
    } else {
      for (int64_t i = lane; i < np * WPR; i += 32) base[i] = 0u;
    }
  }
  __syncwarp();
  if (!valid) return;
  uint32_t *row = base ? base + lane * WPR : nullptr;
  if constexpr (KM > 0) {
    uint32_t list[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
    int n = 0;
#pragma unroll
    for (int i = 0; i < KM; ++i) {
      if (exact[i] < T) continue;
      if (row) {
        uint32_t v = 0u;
#pragma unroll
        for (int j = 0; j < KM; ++j)
          if (exact[j] >= T && (key[j] >> 5) == (key[i] >> 5)) v |= 1u << (key[j] & 31);
        row[key[i] >> 5] = v;
      }
      if constexpr (D <= 5) {  // at most KM <= 8 kept leaves: the whole list
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (n >> 1 == e) list[e] = (n & 1) ? (list[e] & 0xFFFFu) | (key[i] << 16) : 0xFFFF0000u | key[i];
        ++n;
      }
    }
    if constexpr (D <= 5)
      if (kept) reinterpret_cast<uint4 *>(kept)[p] = make_uint4(list[0], list[1], list[2], list[3]);
  } else {
    for (int f = 0; f < N; ++f) {
      const uint32_t q = codes[f * 32 + lane];
      bool first = true;
      for (int g = 0; g < f && first; ++g) first = codes[g * 32 + lane] != q;
      if (!first) continue;
      uint32_t c = 0u;
      int last = -1;
      for (int g = f; g < N; ++g)
        if (codes[g * 32 + lane] == q) {
          const int grp = GRP ? g / group : g;
          if (grp != last) ++c, last = grp;
        }
      if (c >= T) atomicOr(&row[q >> 5], 1u << (q & 31));
    }
  }
}


// Warp-specialised form of build_pixel_red_kernel: NT counting threads plus
// one copy warp.  The copy warp refills stage s as soon as every counting
// warp has signalled (mbarrier "empty[s]") that it is done with it; counting
// warps wait only on "full[s]".  No CTA-wide barrier in the steady state.
// TENSOR: a stage is one 2-D tensor copy (FPS frame rows x NT*3 bytes)
// instead of FPS row copies.  KEPT: the counters are bumped with an atomic
// add that returns the old count, and the leaf's bit is set in the thread's
// "kept" row (registers) the moment its count reaches T; the end of a tile
// then only writes the kept row out and zeroes the touched counters (no
// threshold pass).
template <int D, int NT, int FPS, int S, bool KEPT>
struct WsBuildCfg {
  static constexpr int NC = 1 << (3 * D);
  static constexpr int CW = (NC + 3) / 4;  // u8 counter words per pixel
  static constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  static constexpr int ROW = NT * 3;
  static constexpr int STAGE = ROW * FPS;
  static constexpr size_t STATE = (size_t)CW * NT * 4;
  static constexpr size_t SMEM = STATE + (size_t)S * STAGE + (size_t)S * 16;
  static_assert(ROW % 128 == 0 && STATE % 128 == 0, "stages stay 128-byte aligned");
};

template <int D, int NT, int FPS, int S, bool TENSOR, bool KEPT>
__device__ __forceinline__ void build_pixel_ws_body(const uint8_t *__restrict__ frames, int N, int64_t hw,
                                                    int64_t ntiles, uint32_t T, uint32_t *__restrict__ model,
                                                    const CUtensorMap *tmap, int64_t vb, int64_t vg,
                                                    unsigned int *timeout_flag) {
  using C = WsBuildCfg<D, NT, FPS, S, KEPT>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);  // [CW][NT]
  uint8_t *stages = smem + C::STATE;
  uint64_t *full = reinterpret_cast<uint64_t *>(stages + (size_t)S * C::STAGE);
  uint64_t *empty = full + S;
  const int t = threadIdx.x;
  constexpr int NCW = NT / 32;  // counting warps
  if (t == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_addr(&full[s]), 1);
      mbar_init(smem_addr(&empty[s]), NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (t < NT) {
#pragma unroll 8
    for (int c = 0; c < C::CW; ++c) cnt[c * NT + t] = 0;
  }
  __syncthreads();
  const int G = (N + FPS - 1) / FPS;  // stages per tile
  const int64_t my_tiles = vb < ntiles ? (ntiles - 1 - vb) / vg + 1 : 0;

  if (t >= NT) {  // ---- copy warp ----
    if (t != NT) return;
    int s = 0;
    uint32_t round = 0;
    bool ok = true;
    for (int64_t i = 0; i < my_tiles && ok; ++i) {
      const int64_t tile = vb + i * vg;
      const uint8_t *base = frames + tile * NT * 3;
      for (int g = 0; g < G; ++g) {
        if (round > 0) {  // wait until the counting warps released this stage's previous fill
          if (!mbar_wait_bounded(smem_addr(&empty[s]), (round - 1) & 1, kWaitLimitNs)) {
            atomicExch(timeout_flag, 1u);
            ok = false;
            break;
          }
        }
        const int f0 = g * FPS;
        const uint32_t bar = smem_addr(&full[s]);
        if constexpr (TENSOR) {
          // rows past frame N-1 are filled with zeros and still count as bytes
          mbar_expect_tx(bar, (uint32_t)C::STAGE);
          tensor2d_g2s(smem_addr(stages + (size_t)s * C::STAGE), tmap, (int)(tile * (C::ROW / 4)), f0, bar);
        } else {
          const int nf = N - f0 < FPS ? N - f0 : FPS;
          mbar_expect_tx(bar, (uint32_t)(nf * C::ROW));
          for (int j = 0; j < nf; ++j)
            bulk_g2s(smem_addr(stages + (size_t)s * C::STAGE + (size_t)j * C::ROW),
                     base + (int64_t)(f0 + j) * hw * 3, C::ROW, bar);
        }
        if (++s == S) s = 0, ++round;
      }
    }
    // let the last fills land before this CTA can retire
    for (int k = 0; k < S; ++k) {
      const uint32_t fills = round + (k < s ? 1u : 0u);
      if (fills > 0) mbar_wait_bounded(smem_addr(&full[k]), (fills - 1) & 1, kWaitLimitNs);
    }
    return;
  }

  // ---- counting threads ----
  const int lane = t & 31;
  int s = 0;
  uint32_t round = 0;
  for (int64_t i = 0; i < my_tiles; ++i) {
    uint32_t words = 0;     // KEPT: model words (32 leaves each) this pixel touched
    uint64_t touched = 0;   // else: groups of 8 leaves (two counter words) this pixel touched
    uint32_t kept[C::WPR];
#pragma unroll
    for (int w = 0; w < C::WPR; ++w) kept[w] = 0;
    for (int g = 0; g < G; ++g) {
      if (!mbar_wait_bounded(smem_addr(&full[s]), round & 1, kWaitLimitNs)) {
        atomicExch(timeout_flag, 1u);
        return;
      }
      const uint8_t *stage = stages + (size_t)s * C::STAGE + 3 * t;
      const int nf = N - g * FPS < FPS ? N - g * FPS : FPS;
#pragma unroll
      for (int j = 0; j < FPS; ++j) {
        if (j < nf) {
          const uint8_t *px = stage + j * C::ROW;
          const uint32_t y = (uint32_t)px[0] | ((uint32_t)px[1] << 8) | ((uint32_t)px[2] << 16);
          const uint32_t q = planar_code<D>(y);
          const uint32_t sh = (q & 3u) * 8;
          if constexpr (KEPT) {
            const uint32_t old = atomicAdd(&cnt[(q >> 2) * NT + t], 1u << sh);
            if (((old >> sh) & 0xFFu) + 1u == T) {  // once per kept leaf and tile
#pragma unroll
              for (int w = 0; w < C::WPR; ++w)
                if ((int)(q >> 5) == w) kept[w] |= 1u << (q & 31);
            }
            words |= 1u << (q >> 5);
          } else {
            red_add_shared(&cnt[(q >> 2) * NT + t], 1u << sh);
            touched |= 1ull << (q >> 3);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
      if (++s == S) s = 0, ++round;
    }
    uint32_t *dst = model + ((vb + i * vg) * NT + t) * C::WPR;
    if constexpr (KEPT) {
      if constexpr (C::WPR % 4 == 0) {
#pragma unroll
        for (int w = 0; w < C::WPR; w += 4)
          *reinterpret_cast<uint4 *>(dst + w) = make_uint4(kept[w], kept[w + 1], kept[w + 2], kept[w + 3]);
      } else {
#pragma unroll
        for (int w = 0; w < C::WPR; ++w) dst[w] = kept[w];
      }
      for (; words; words &= words - 1) {  // zero the counters this tile used
        const int w = __ffs(words) - 1;
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (w * 8 + c < C::CW) cnt[(w * 8 + c) * NT + t] = 0;
      }
    } else {
      if constexpr (C::WPR % 4 == 0) {
#pragma unroll
        for (int w = 0; w < C::WPR; w += 4) *reinterpret_cast<uint4 *>(dst + w) = make_uint4(0, 0, 0, 0);
      } else {
#pragma unroll
        for (int w = 0; w < C::WPR; ++w) dst[w] = 0;
      }
      // threshold only the counter words of the 8-leaf groups that occurred,
      // in increasing order, so each model word is assembled then stored once
      int cur = -1;
      uint32_t o = 0;
      for (; touched; touched &= touched - 1) {
        const int g = __ffsll((long long)touched) - 1;
        if ((g >> 2) != cur) {
          if (cur >= 0) dst[cur] = o;
          cur = g >> 2, o = 0;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (2 * g + c < C::CW) {
            uint32_t *cp = &cnt[(2 * g + c) * NT + t];
            const uint32_t ge = __vcmpgeu4(*cp, T * 0x01010101u);
            o |= (((ge >> 7) & 1u) | ((ge >> 14) & 2u) | ((ge >> 21) & 4u) | ((ge >> 28) & 8u)) << ((g & 3) * 8 + 4 * c);
            *cp = 0;
          }
        }
      }
      if (cur >= 0) dst[cur] = o;
    }
  }
}

}  // namespace ocq
