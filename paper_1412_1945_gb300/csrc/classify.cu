// S4: Check Color (Alg. 3) for every pixel of incoming frames (Sec. 4).
// A pixel is background when the bit of its leaf is set in its region's row.
//
// Kernels:
//   classify_generic_kernel      any region/depth: per-pixel global lookups.
//   classify_frame_kernel<D>     whole-frame regions, depth <= 6: the one row
//                                lives in shared memory (replicated per lane
//                                for depth <= 4 so lookups never conflict),
//                                frames stream through 16-byte loads.
//   classify_pixel_tiled_kernel  pixel regions, depth <= 3: temporal blocking.
//                                A CTA keeps the rows of a tile of pixel
//                                locations in shared memory (lane-interleaved:
//                                each lane's rows sit in its own bank) and
//                                streams that tile of many frames through a
//                                ring of stages filled by bulk asynchronous
//                                copies (cp.async.bulk + mbarrier), so each
//                                row is read from HBM about once per launch.
#include <cstdint>

#include "async_copy.cuh"
#include "pixels.cuh"

namespace ocq {

// Set when a bounded wait gives up; read and cleared by device_status().
__device__ unsigned int g_classify_timeout;

// ---- generic ---------------------------------------------------------------------
__global__ void classify_generic_kernel(const uint8_t *__restrict__ frames, int F, int H, int W, int kind, int block,
                                        int d, int64_t wpr, const uint32_t *__restrict__ model,
                                        uint8_t *__restrict__ mask, int64_t pb, int64_t pe) {
  const int64_t hw = (int64_t)H * W;
  const int64_t n = pe - pb;
  const int64_t total = n * F;
  const int bw = kind == OCQ_REGION_BLOCK ? (W + block - 1) / block : 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = i / n;
    const int64_t p = pb + (i - f * n);
    const int64_t g = f * hw + p;
    const uint8_t *px = frames + g * 3;
    const uint32_t q = planar_code_rt(__ldg(px), __ldg(px + 1), __ldg(px + 2), d);
    const int y = (int)(p / W), x = (int)(p - (int64_t)y * W);
    const uint32_t word = __ldg(model + region_of(y, x, W, kind, block, bw) * wpr + (q >> 5));
    mask[g] = (uint8_t)(((word >> (q & 31)) & 1u) ^ 1u);
  }
}

// Four pixels' background bits (bit 0 of each of f0..f3) -> four mask bytes.
__device__ __forceinline__ uint32_t pack_mask4(uint32_t f0, uint32_t f1, uint32_t f2, uint32_t f3) {
  const uint32_t lo = __byte_perm(f0, f1, 0x0040);
  const uint32_t hi = __byte_perm(f2, f3, 0x0040);
  const uint32_t v = __byte_perm(lo, hi, 0x5410);
  return ~v & 0x01010101u;
}

// ---- whole-frame regions ------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256) classify_frame_kernel(const uint8_t *__restrict__ frames, int64_t npix,
                                                             const uint32_t *__restrict__ model,
                                                             uint8_t *__restrict__ mask) {
  constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  constexpr int REP = D <= 4 ? 32 : 1;
  extern __shared__ uint32_t row[];  // [WPR][REP]
  for (int i = threadIdx.x; i < WPR * REP; i += blockDim.x) row[i] = __ldg(model + i / REP);
  __syncthreads();
  const int rep = REP == 32 ? (threadIdx.x & 31) : 0;
  const bool vec = ((reinterpret_cast<uintptr_t>(frames) | reinterpret_cast<uintptr_t>(mask)) & 15) == 0;
  int64_t tail = 0;
  if (vec) {
    const int64_t ng = npix >> 4;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
      uint32_t w[12];
      load_group_masked<D, true>(frames + g * 48, w);
      uint32_t fbit[16];
      static_for<0, 16>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const uint32_t q = planar_from_masked<D>(group_pixel<k>(w));
        const uint32_t v = row[(q >> 5) * REP + rep];
        fbit[k] = __funnelshift_r(v, v, q);
      });
      uint4 o;
      o.x = pack_mask4(fbit[0], fbit[1], fbit[2], fbit[3]);
      o.y = pack_mask4(fbit[4], fbit[5], fbit[6], fbit[7]);
      o.z = pack_mask4(fbit[8], fbit[9], fbit[10], fbit[11]);
      o.w = pack_mask4(fbit[12], fbit[13], fbit[14], fbit[15]);
      st_stream16(mask + g * 16, o);
    }
    tail = ng << 4;
  }
  for (int64_t p = tail + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t *px = frames + p * 3;
    const uint32_t q = planar_code_rt(px[0], px[1], px[2], D);
    mask[p] = (uint8_t)(((row[(q >> 5) * REP + rep] >> (q & 31)) & 1u) ^ 1u);
  }
}

// ---- pixel regions: temporal blocking with bulk async copies --------------------------

template <int D, int NW, int PPT, int S, int FPS>
struct TiledCfg {
  static constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  static constexpr int THREADS = NW * 32;
  static constexpr int TILE = THREADS * PPT;       // pixel locations per tile
  static constexpr int FRAME_BYTES = TILE * 3;     // one frame's tile
  static constexpr int STAGE = FRAME_BYTES * FPS;  // one stage holds FPS frames
  static constexpr int MODEL_WORDS = TILE * WPR;
  static constexpr size_t SMEM = (size_t)MODEL_WORDS * 4 + (size_t)S * STAGE + (size_t)S * 8;
  static_assert(FRAME_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
  static_assert(PPT == 8 || PPT == 16, "8 or 16 pixels per thread");
};

// Classifies one frame of the tile from shared memory: thread (warp, lane)
// handles pixels (warp*32 + lane)*PPT + j of the tile.
template <int D, int NW, int PPT, int S, int FPS>
__device__ __forceinline__ void classify_tile_frame(const uint8_t *__restrict__ src, const uint32_t *__restrict__ mrow,
                                                    uint8_t *__restrict__ dst) {
  using C = TiledCfg<D, NW, PPT, S, FPS>;
  const int tid = threadIdx.x;
  uint32_t fbit[PPT];
  uint32_t w[12];
  if constexpr (PPT == 16) {
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src + tid * 48);
    const uint4 a = s4[0], b = s4[1], c = s4[2];
    w[0] = a.x, w[1] = a.y, w[2] = a.z, w[3] = a.w, w[4] = b.x, w[5] = b.y;
    w[6] = b.z, w[7] = b.w, w[8] = c.x, w[9] = c.y, w[10] = c.z, w[11] = c.w;
#pragma unroll
    for (int e = 0; e < 12; ++e) w[e] = (w[e] >> (8 - D)) & byte_mask(D);
  } else {
    const uint2 *s2 = reinterpret_cast<const uint2 *>(src + tid * 24);
    const uint2 a = s2[0], b = s2[1], c = s2[2];
    w[0] = a.x, w[1] = a.y, w[2] = b.x, w[3] = b.y, w[4] = c.x, w[5] = c.y;
    w[6] = w[7] = w[8] = w[9] = w[10] = w[11] = 0;
#pragma unroll
    for (int e = 0; e < 6; ++e) w[e] = (w[e] >> (8 - D)) & byte_mask(D);
  }
  // mrow points at word 0 of pixel j=0 for this lane; pixel j's word q>>5 is at
  // mrow[(j*WPR + (q>>5))*32]
  static_for<0, PPT>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    const uint32_t q = planar_from_masked<D>(group_pixel<j>(w));
    const uint32_t v = mrow[(j * C::WPR + (q >> 5)) * 32];
    fbit[j] = __funnelshift_r(v, v, q);
  });
  if constexpr (PPT == 16) {
    uint4 o;
    o.x = pack_mask4(fbit[0], fbit[1], fbit[2], fbit[3]);
    o.y = pack_mask4(fbit[4], fbit[5], fbit[6], fbit[7]);
    o.z = pack_mask4(fbit[8], fbit[9], fbit[10], fbit[11]);
    o.w = pack_mask4(fbit[12], fbit[13], fbit[14], fbit[15]);
    st_stream16(dst + tid * 16, o);
  } else {
    const uint32_t x = pack_mask4(fbit[0], fbit[1], fbit[2], fbit[3]);
    const uint32_t y = pack_mask4(fbit[4], fbit[5], fbit[6], fbit[7]);
    asm volatile("st.global.cs.v2.u32 [%0], {%1,%2};" ::"l"(dst + tid * 8), "r"(x), "r"(y) : "memory");
  }
}

// Work item u = tile * F + f; CTA b handles u in [b*U/G, (b+1)*U/G), i.e. a run
// of frames of one tile, then of the next, reloading the tile's rows at each
// tile change.  Frames move in groups of FPS per stage.  Requires: frames and
// mask 16-byte aligned, H*W % 16 == 0.
template <int D, int NW, int PPT, int S, int FPS>
__global__ void __launch_bounds__(NW * 32, 1)
    classify_pixel_tiled_kernel(const uint8_t *__restrict__ frames, int F, int64_t hw, int64_t ntiles,
                                const uint32_t *__restrict__ model, uint8_t *__restrict__ mask) {
  using C = TiledCfg<D, NW, PPT, S, FPS>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *msm = reinterpret_cast<uint32_t *>(smem);
  uint8_t *stages = smem + (size_t)C::MODEL_WORDS * 4;
  uint64_t *bars = reinterpret_cast<uint64_t *>(stages + (size_t)S * C::STAGE);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(smem_addr(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int64_t U = ntiles * (int64_t)F;
  const int64_t u_begin = U * blockIdx.x / gridDim.x;
  const int64_t u_end = U * (blockIdx.x + 1) / gridDim.x;
  const uint32_t *mrow = msm + warp * PPT * C::WPR * 32 + lane;
  uint64_t kc = 0;  // stages consumed so far (stage = kc % S, phase = (kc / S) & 1)

  for (int64_t u = u_begin; u < u_end;) {
    const int64_t tile = u / F;
    const int fa = (int)(u - tile * F);
    const int nfr = (int)((u_end - u) < (int64_t)(F - fa) ? (u_end - u) : (int64_t)(F - fa));
    const int ngroups = (nfr + FPS - 1) / FPS;
    const int64_t p_tile = tile * C::TILE;

    // Rows of this tile -> shared memory, word w of pixel (warp, lane, j) at
    // ((warp*PPT + j)*WPR + w)*32 + lane.
    {
      const uint32_t *src = model + (p_tile + (int64_t)tid * PPT) * C::WPR;
      if constexpr (C::WPR % 4 == 0) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
#pragma unroll 4
        for (int i = 0; i < PPT * C::WPR / 4; ++i) {
          const uint4 v = __ldg(s4 + i);
          const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int idx = i * 4 + e, j = idx / C::WPR, w = idx % C::WPR;
            msm[((warp * PPT + j) * C::WPR + w) * 32 + lane] = vv[e];
          }
        }
      } else {
#pragma unroll
        for (int idx = 0; idx < PPT * C::WPR; ++idx) {
          const int j = idx / C::WPR, w = idx % C::WPR;
          msm[((warp * PPT + j) * C::WPR + w) * 32 + lane] = __ldg(src + idx);
        }
      }
    }
    __syncthreads();

    auto issue = [&](int g) {  // group g of this run -> stage (kc + g) % S
      const int s = (int)((kc + g) % S);
      const int f0 = fa + g * FPS;
      const int nf = (nfr - g * FPS) < FPS ? (nfr - g * FPS) : FPS;
      const uint32_t bar = smem_addr(&bars[s]);
      mbar_expect_tx(bar, (uint32_t)(nf * C::FRAME_BYTES));
      for (int i = 0; i < nf; ++i)
        bulk_g2s(smem_addr(stages + (size_t)s * C::STAGE + (size_t)i * C::FRAME_BYTES),
                 frames + ((int64_t)(f0 + i) * hw + p_tile) * 3, C::FRAME_BYTES, bar);
    };
    if (tid == 0) {
      const int pre = ngroups < S ? ngroups : S;
      for (int g = 0; g < pre; ++g) issue(g);
    }

    for (int g = 0; g < ngroups; ++g) {
      const uint64_t k = kc + g;
      const int s = (int)(k % S);
      const bool ok = mbar_wait_bounded(smem_addr(&bars[s]), (uint32_t)((k / S) & 1), kWaitLimitNs);
      const uint8_t *stage = stages + (size_t)s * C::STAGE;
      const int f0 = fa + g * FPS;
      const int nf = (nfr - g * FPS) < FPS ? (nfr - g * FPS) : FPS;
#pragma unroll
      for (int i = 0; i < FPS; ++i) {
        if (i < nf)
          classify_tile_frame<D, NW, PPT, S, FPS>(stage + (size_t)i * C::FRAME_BYTES, mrow,
                                                  mask + (int64_t)(f0 + i) * hw + p_tile);
      }
      // Stage s is consumed by every thread; refill it with group g + S.
      if (__syncthreads_or(!ok)) {
        // A copy did not arrive in time: record it, let every copy this CTA
        // still has in flight land (bounded), and leave.
        if (tid == 0) {
          atomicExch(&g_classify_timeout, 1u);
          const int inflight = (ngroups - g) < S ? (ngroups - g) : S;
          for (int j = 0; j < inflight; ++j) {
            const uint64_t kk = k + j;
            mbar_wait_bounded(smem_addr(&bars[kk % S]), (uint32_t)((kk / S) & 1), kWaitLimitNs);
          }
        }
        __syncthreads();
        return;
      }
      if (tid == 0 && g + S < ngroups) issue(g + S);
    }
    kc += ngroups;
    u += nfr;
    __syncthreads();  // all reads of this tile's rows are done before the next reload
  }
}

// Warp-specialised form: NW classifying warps plus one copy warp.  The copy
// warp streams every group of the CTA's work range, refilling a stage as soon
// as all classifying warps have released it (mbarrier "empty"); classifying
// warps wait only on "full".  At a tile change the classifying warps (named
// barrier 1, the copy warp is not part of it) reload the tile's rows.  A
// timed-out wait raises a shared abort flag; the warps then run to the end
// without waiting, so no barrier is left short of arrivals.
template <int D, int NW, int PPT, int S, int FPS>
__global__ void __launch_bounds__(NW * 32 + 32, 1)
    classify_pixel_ws_kernel(const uint8_t *__restrict__ frames, int F, int64_t hw, int64_t ntiles,
                             const uint32_t *__restrict__ model, uint8_t *__restrict__ mask) {
  using C = TiledCfg<D, NW, PPT, S, FPS>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *msm = reinterpret_cast<uint32_t *>(smem);
  uint8_t *stages = smem + (size_t)C::MODEL_WORDS * 4;
  uint64_t *full = reinterpret_cast<uint64_t *>(stages + (size_t)S * C::STAGE);
  uint64_t *empty = full + S;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_addr(&full[s]), 1);
      mbar_init(smem_addr(&empty[s]), NW);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t U = ntiles * (int64_t)F;
  const int64_t u_begin = U * blockIdx.x / gridDim.x;
  const int64_t u_end = U * (blockIdx.x + 1) / gridDim.x;

  if (tid >= NW * 32) {  // ---- copy warp ----
    if (tid != NW * 32) return;
    int s = 0;
    uint32_t round = 0;
    for (int64_t u = u_begin; u < u_end && !abort_flag;) {
      const int64_t tile = u / F;
      const int fa = (int)(u - tile * F);
      const int nfr = (int)((u_end - u) < (int64_t)(F - fa) ? (u_end - u) : (int64_t)(F - fa));
      const uint8_t *base = frames + tile * C::TILE * 3;
      for (int g = 0; g * FPS < nfr; ++g) {
        if (round > 0 && !mbar_wait_bounded(smem_addr(&empty[s]), (round - 1) & 1, kWaitLimitNs)) {
          atomicExch(&g_classify_timeout, 1u);
          abort_flag = 1;
          break;
        }
        const int f0 = fa + g * FPS;
        const int nf = (nfr - g * FPS) < FPS ? (nfr - g * FPS) : FPS;
        const uint32_t bar = smem_addr(&full[s]);
        mbar_expect_tx(bar, (uint32_t)(nf * C::FRAME_BYTES));
        for (int i = 0; i < nf; ++i)
          bulk_g2s(smem_addr(stages + (size_t)s * C::STAGE + (size_t)i * C::FRAME_BYTES),
                   base + (int64_t)(f0 + i) * hw * 3, C::FRAME_BYTES, bar);
        if (++s == S) s = 0, ++round;
      }
      u += nfr;
    }
    for (int k = 0; k < S; ++k) {  // let the last fills land before the CTA can retire
      const uint32_t fills = round + (k < s ? 1u : 0u);
      if (fills > 0) mbar_wait_bounded(smem_addr(&full[k]), (fills - 1) & 1, kWaitLimitNs);
    }
    return;
  }

  // ---- classifying warps ----
  const int lane = tid & 31, warp = tid >> 5;
  const uint32_t *mrow = msm + warp * PPT * C::WPR * 32 + lane;
  int s = 0;
  uint32_t round = 0;
  for (int64_t u = u_begin; u < u_end;) {
    const int64_t tile = u / F;
    const int fa = (int)(u - tile * F);
    const int nfr = (int)((u_end - u) < (int64_t)(F - fa) ? (u_end - u) : (int64_t)(F - fa));
    const int64_t p_tile = tile * C::TILE;
    named_sync(1, NW * 32);  // every warp is done with the previous tile's rows
    {
      const uint32_t *src = model + (p_tile + (int64_t)tid * PPT) * C::WPR;
      if constexpr (C::WPR % 4 == 0) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
#pragma unroll 4
        for (int i = 0; i < PPT * C::WPR / 4; ++i) {
          const uint4 v = __ldg(s4 + i);
          const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int idx = i * 4 + e, j = idx / C::WPR, w = idx % C::WPR;
            msm[((warp * PPT + j) * C::WPR + w) * 32 + lane] = vv[e];
          }
        }
      } else {
#pragma unroll
        for (int idx = 0; idx < PPT * C::WPR; ++idx) {
          const int j = idx / C::WPR, w = idx % C::WPR;
          msm[((warp * PPT + j) * C::WPR + w) * 32 + lane] = __ldg(src + idx);
        }
      }
    }
    named_sync(1, NW * 32);
    for (int g = 0; g * FPS < nfr; ++g) {
      const int f0 = fa + g * FPS;
      const int nf = (nfr - g * FPS) < FPS ? (nfr - g * FPS) : FPS;
      if (!abort_flag) {
        if (mbar_wait_bounded(smem_addr(&full[s]), round & 1, kWaitLimitNs)) {
          const uint8_t *stage = stages + (size_t)s * C::STAGE;
#pragma unroll
          for (int i = 0; i < FPS; ++i)
            if (i < nf)
              classify_tile_frame<D, NW, PPT, S, FPS>(stage + (size_t)i * C::FRAME_BYTES, mrow,
                                                      mask + (int64_t)(f0 + i) * hw + p_tile);
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
        } else {
          atomicExch(&g_classify_timeout, 1u);
          abort_flag = 1;
        }
      }
      if (++s == S) s = 0, ++round;
    }
    u += nfr;
  }
}

// ---- host dispatch -----------------------------------------------------------------------

static unsigned grid_cap(int64_t work, int threads, int per_sm) {
  int64_t b = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

static ocq_status launch_generic(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask, int64_t pb,
                                 int64_t pe, cudaStream_t st) {
  if (pe <= pb) return OCQ_OK;
  classify_generic_kernel<<<grid_cap((pe - pb) * F, 256, 16), 256, 0, st>>>(
      frames, F, m->H, m->W, m->kind, m->block, m->depth, m->wpr, m->bits, mask, pb, pe);
  count_launch();
  return cuda_status(cudaGetLastError(), "classify_generic_kernel");
}

template <int D>
static ocq_status launch_frame(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask, cudaStream_t st) {
  constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  constexpr int REP = D <= 4 ? 32 : 1;
  const size_t smem = (size_t)WPR * REP * 4;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(classify_frame_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t npix = (int64_t)F * m->H * m->W;
  const int per_sm = smem > 64 * 1024 ? 1 : 4;
  classify_frame_kernel<D><<<grid_cap((npix + 15) / 16, 256, per_sm), 256, smem, st>>>(frames, npix, m->bits, mask);
  count_launch();
  return cuda_status(cudaGetLastError(), "classify_frame_kernel");
}

template <int D, int NW, int PPT, int S, int FPS>
static ocq_status launch_tiled(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask, cudaStream_t st) {
  using C = TiledCfg<D, NW, PPT, S, FPS>;
  const int64_t hw = (int64_t)m->H * m->W;
  const int64_t ntiles = hw / C::TILE;
  ocq_status rc = OCQ_OK;
  if (ntiles > 0) {
    auto kern = classify_pixel_tiled_kernel<D, NW, PPT, S, FPS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return cuda_status(e, "classify_pixel_tiled_kernel smem");
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::THREADS, C::SMEM);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sm_count() * per_sm;
    const int64_t U = ntiles * F;
    if (grid > U) grid = U;
    kern<<<(unsigned)grid, C::THREADS, C::SMEM, st>>>(frames, F, hw, ntiles, m->bits, mask);
    count_launch();
    rc = cuda_status(cudaGetLastError(), "classify_pixel_tiled_kernel");
  }
  if (rc == OCQ_OK) rc = launch_generic(m, frames, F, mask, ntiles * C::TILE, hw, st);
  return rc;
}

template <int D, int NW, int PPT, int S, int FPS>
static ocq_status launch_tiled_ws(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask, cudaStream_t st) {
  using C = TiledCfg<D, NW, PPT, S, FPS>;
  const int64_t hw = (int64_t)m->H * m->W;
  const size_t smem = C::SMEM + (size_t)S * 8;
  const int64_t ntiles = smem <= 227 * 1024 ? hw / C::TILE : 0;
  ocq_status rc = OCQ_OK;
  if (ntiles > 0) {
    auto kern = classify_pixel_ws_kernel<D, NW, PPT, S, FPS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e, "classify_pixel_ws_kernel smem");
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::THREADS + 32, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sm_count() * per_sm;
    const int64_t U = ntiles * F;
    if (grid > U) grid = U;
    kern<<<(unsigned)grid, C::THREADS + 32, smem, st>>>(frames, F, hw, ntiles, m->bits, mask);
    count_launch();
    rc = cuda_status(cudaGetLastError(), "classify_pixel_ws_kernel");
  }
  if (rc == OCQ_OK) rc = launch_generic(m, frames, F, mask, ntiles * C::TILE, hw, st);
  return rc;
}

// ---- tunable variants of the per-pixel tiled kernel ---------------------------------
using ClassifyFn = ocq_status (*)(const ocq_model *, const uint8_t *, int, uint8_t *, cudaStream_t);
struct ClassifyVariant {
  int nw, ppt, stages, fps, ws;
  ClassifyFn fn[3];  // depth 1, 2, 3
};
#define OCQ_CV(NW, PPT, S, FPS)                                                          \
  {                                                                                      \
    NW, PPT, S, FPS, 0, {                                                                \
      launch_tiled<1, NW, PPT, S, FPS>, launch_tiled<2, NW, PPT, S, FPS>, launch_tiled<3, NW, PPT, S, FPS> \
    }                                                                                    \
  }
#define OCQ_WV(NW, PPT, S, FPS)                                                          \
  {                                                                                      \
    NW, PPT, S, FPS, 1, {                                                                \
      launch_tiled_ws<1, NW, PPT, S, FPS>, launch_tiled_ws<2, NW, PPT, S, FPS>,           \
          launch_tiled_ws<3, NW, PPT, S, FPS>                                            \
    }                                                                                    \
  }
// ws (5th field): 1 = a dedicated copy warp with full/empty mbarriers
static const ClassifyVariant kClassifyVariants[] = {
    OCQ_CV(8, 8, 3, 4), OCQ_CV(4, 8, 4, 4), OCQ_CV(4, 8, 12, 1), OCQ_CV(8, 8, 4, 2),
    OCQ_WV(8, 8, 3, 4), OCQ_WV(4, 8, 4, 4), OCQ_WV(8, 8, 6, 2), OCQ_WV(4, 8, 8, 2), OCQ_WV(4, 8, 3, 5)};
#undef OCQ_CV
#undef OCQ_WV
static int g_classify_variant = 5;

int classify_variant_count() { return (int)(sizeof kClassifyVariants / sizeof kClassifyVariants[0]); }
int classify_variant_selected() { return g_classify_variant; }
bool classify_variant_select(int v) {
  if (v < 0 || v >= classify_variant_count()) return false;
  g_classify_variant = v;
  return true;
}
void classify_variant_describe(int v, int *nw, int *ppt, int *stages, int *fps, int *ws) {
  *nw = kClassifyVariants[v].nw, *ppt = kClassifyVariants[v].ppt;
  *stages = kClassifyVariants[v].stages, *fps = kClassifyVariants[v].fps;
  *ws = kClassifyVariants[v].ws;
}

ocq_status launch_classify(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask, cudaStream_t st) {
  const int64_t hw = (int64_t)m->H * m->W;
  const int d = m->depth;
  if (m->kind == OCQ_REGION_FRAME && d <= 6) {
    switch (d) {
      case 1: return launch_frame<1>(m, frames, F, mask, st);
      case 2: return launch_frame<2>(m, frames, F, mask, st);
      case 3: return launch_frame<3>(m, frames, F, mask, st);
      case 4: return launch_frame<4>(m, frames, F, mask, st);
      case 5: return launch_frame<5>(m, frames, F, mask, st);
      default: return launch_frame<6>(m, frames, F, mask, st);
    }
  }
  const bool aligned = ((reinterpret_cast<uintptr_t>(frames) | reinterpret_cast<uintptr_t>(mask)) & 15) == 0;
  if (m->kind == OCQ_REGION_PIXEL && d <= 3 && aligned && hw % 16 == 0)
    return kClassifyVariants[g_classify_variant].fn[d - 1](m, frames, F, mask, st);
  return launch_generic(m, frames, F, mask, 0, hw, st);
}

bool classify_take_timeout() {
  unsigned int flag = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&flag, g_classify_timeout, sizeof flag) != cudaSuccess) return false;
  if (flag) cudaMemcpyToSymbol(g_classify_timeout, &zero, sizeof zero);
  return flag != 0;
}

}  // namespace ocq
