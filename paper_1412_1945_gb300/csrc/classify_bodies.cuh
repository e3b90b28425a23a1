// Device bodies of the classify kernels (S4, Alg. 3), parameterised by a
// virtual CTA index vb of vg so that the same code runs as a plain grid
// (vb = blockIdx.x, vg = gridDim.x) and as an item of the batched persistent
// kernel.  Model words are read with ordinary (coherent, not read-only-path)
// loads: in the batched kernel a model is written earlier in the same launch,
// and its readers start only after an acquire (counter wait + fence).
#pragma once

#include "async_copy.cuh"
#include "pixels.cuh"

namespace ocq {

// ---- generic ---------------------------------------------------------------------
__device__ __forceinline__ void classify_generic_body(const uint8_t *__restrict__ frames, int F, int H, int W, int kind, int block,
                                        int d, int64_t wpr, const uint32_t *model,
                                        uint8_t *__restrict__ mask, int64_t pb, int64_t pe,
                                                     int64_t vb, int64_t vg) {
  const int64_t hw = (int64_t)H * W;
  const int64_t n = pe - pb;
  const int64_t total = n * F;
  const int bw = kind == OCQ_REGION_BLOCK ? (W + block - 1) / block : 1;
  for (int64_t i = vb * blockDim.x + threadIdx.x; i < total; i += vg * blockDim.x) {
    const int64_t f = i / n;
    const int64_t p = pb + (i - f * n);
    const int64_t g = f * hw + p;
    const uint8_t *px = frames + g * 3;
    const uint32_t q = planar_code_rt(__ldg(px), __ldg(px + 1), __ldg(px + 2), d);
    const int y = (int)(p / W), x = (int)(p - (int64_t)y * W);
    const uint32_t word = *(model + region_of(y, x, W, kind, block, bw) * wpr + (q >> 5));
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
__device__ __forceinline__ void classify_frame_body(const uint8_t *__restrict__ frames, int64_t npix,
                                                    const uint32_t *model, uint8_t *__restrict__ mask,
                                                    int64_t vb, int64_t vg) {
  constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  constexpr int REP = D <= 4 ? 32 : 1;
  extern __shared__ uint32_t row[];  // [WPR][REP]
  for (int i = threadIdx.x; i < WPR * REP; i += blockDim.x) row[i] = model[i / REP];
  __syncthreads();
  const int rep = REP == 32 ? (threadIdx.x & 31) : 0;
  const bool vec = ((reinterpret_cast<uintptr_t>(frames) | reinterpret_cast<uintptr_t>(mask)) & 15) == 0;
  int64_t tail = 0;
  if (vec) {
    const int64_t ng = npix >> 4;
    for (int64_t g = vb * blockDim.x + threadIdx.x; g < ng; g += vg * blockDim.x) {
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
  for (int64_t p = tail + vb * blockDim.x + threadIdx.x; p < npix; p += vg * blockDim.x) {
    const uint8_t *px = frames + p * 3;
    const uint32_t q = planar_code_rt(px[0], px[1], px[2], D);
    mask[p] = (uint8_t)(((row[(q >> 5) * REP + rep] >> (q & 31)) & 1u) ^ 1u);
  }
}

// ---- pixel regions, any depth: temporal blocking through L1 ----------------------
// A warp owns 128 consecutive pixel locations (4 per lane) and walks all F
// frames for them, so the few model sectors each location's colours hit stay
// in the SM's L1 between frames instead of being fetched once per frame: the
// rows are 8^d/8 bytes (512 B at d = 4, 4 KB at d = 5), too large to stage
// whole in shared memory.  Frames are read with streaming 4-byte loads and the
// mask written with streaming 4-byte stores, so neither displaces the model
// lines.  Needs H*W % 4 == 0 and 4-byte aligned frames and mask.
__device__ __forceinline__ uint32_t ld_stream4(const void *p) {
  uint32_t v;
  asm volatile("ld.global.cs.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_stream4(void *p, uint32_t v) {
  asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Packed pixel k (0..3) of 4 pixels held as 3 words.
template <int K>
__device__ __forceinline__ uint32_t quad_pixel(const uint32_t (&w)[3]) {
  constexpr int o = 3 * K, i = o / 4, s = o % 4;
  constexpr uint32_t sel = (uint32_t)(s | ((s + 1) << 4) | ((s + 2) << 8) | ((s + 2) << 12));
  if constexpr (i + 1 < 3)
    return __byte_perm(w[i], w[i + 1], sel);
  else
    return __byte_perm(w[i], 0u, sel);
}

template <int D, int PF>
__device__ __forceinline__ void classify_pixel_tb_body(const uint8_t *__restrict__ frames, int F, int64_t hw,
                                                       const uint32_t *model, uint8_t *__restrict__ mask,
                                                       int64_t tile) {
  constexpr int64_t WPR = D == 1 ? 1 : (int64_t)1 << (3 * D - 5);
  const int lane = threadIdx.x & 31;
  const int64_t pq = tile * 128 + 4 * lane;
  if (pq >= hw) return;
  const uint8_t *rows = reinterpret_cast<const uint8_t *>(model + pq * WPR);
  const uint8_t *src = frames + pq * 3;
  uint8_t *dst = mask + pq;
  for (int f0 = 0; f0 < F; f0 += PF) {
    uint32_t w[PF][3];
#pragma unroll
    for (int j = 0; j < PF; ++j)
      if (f0 + j < F) {
        const uint8_t *s = src + (int64_t)(f0 + j) * hw * 3;
        w[j][0] = ld_stream4(s), w[j][1] = ld_stream4(s + 4), w[j][2] = ld_stream4(s + 8);
      }
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      if (f0 + j >= F) break;
      uint32_t m[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) m[i] = (w[j][i] >> (8 - D)) & byte_mask(D);
      uint32_t bg[4];
      static_for<0, 4>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const uint32_t q = planar_from_masked<D>(quad_pixel<k>(m));
        bg[k] = (uint32_t)rows[k * WPR * 4 + (q >> 3)] >> (q & 7);
      });
      st_stream4(dst + (int64_t)(f0 + j) * hw, pack_mask4(bg[0], bg[1], bg[2], bg[3]));
    }
  }
}

// Block regions (b % 4 == 0, W % 4 == 0), any depth: as the per-pixel form,
// a warp walks all F frames of 128 consecutive pixels of one pixel row (4 per
// lane, all 4 in one block), their lookups hitting L1.  Tile t covers pixel row
// k = t % b of block row br and 128-pixel segment sg, t / b = br * nseg + sg,
// so the b warps of consecutive tiles cover whole blocks: a CTA of 8 warps
// reads each block row's model sectors once per SM when b <= 8.
//
// Frames [fb, fe) only (fe < 0: all F), so a launch can split the frames of a
// small frame over more warps.  The loads of the next PF frames are in flight
// while the current PF are looked up (two register buffers).
// ftab/mtab (device tables, or null): frame f and its mask at ftab[f] and
// mtab[f] instead of frames + f*H*W*3 and mask + f*H*W (frames gathered from
// several buffers, as a serving tick's).  ctab (or null): frame f's u16 leaf
// codes are written at ctab[f] too (a serving window's slot), 8-byte aligned.
template <int D, int PF>
__device__ __forceinline__ void classify_block_tb_body(const uint8_t *__restrict__ frames, int F, int H, int W,
                                                       int b, int bw, int nseg, const uint32_t *model,
                                                       uint8_t *__restrict__ mask, int64_t t, int fb = 0,
                                                       int fe = -1, const uint8_t *const *ftab = nullptr,
                                                       uint8_t *const *mtab = nullptr,
                                                       uint16_t *const *ctab = nullptr) {
  constexpr int64_t WPR = D == 1 ? 1 : (int64_t)1 << (3 * D - 5);
  if (fe < 0 || fe > F) fe = F;
  const int lane = threadIdx.x & 31;
  const int k = (int)(t % b);
  const int64_t q = t / b;
  const int br = (int)(q / nseg), sg = (int)(q % nseg);
  const int y = br * b + k;
  const int x = sg * 128 + 4 * lane;
  if (y >= H || x >= W) return;
  const int64_t hw = (int64_t)H * W;
  const int64_t pq = (int64_t)y * W + x;
  const uint8_t *row = reinterpret_cast<const uint8_t *>(model + ((int64_t)br * bw + x / b) * WPR);
  const uint8_t *src = frames + pq * 3;
  uint8_t *dst = mask + pq;
  auto fsrc = [&](int f) { return ftab ? ftab[f] + pq * 3 : src + (int64_t)f * hw * 3; };
  auto fdst = [&](int f) { return mtab ? mtab[f] + pq : dst + (int64_t)f * hw; };
  auto load = [&](uint32_t (&w)[PF][3], int f0) {
#pragma unroll
    for (int j = 0; j < PF; ++j)
      if (f0 + j < fe) {
        const uint8_t *s = fsrc(f0 + j);
        w[j][0] = ld_stream4(s), w[j][1] = ld_stream4(s + 4), w[j][2] = ld_stream4(s + 8);
      }
  };
  auto work = [&](const uint32_t (&w)[PF][3], int f0) {
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      if (f0 + j >= fe) break;
      uint32_t m[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) m[i] = (w[j][i] >> (8 - D)) & byte_mask(D);
      uint32_t bg[4], cq[4];
      static_for<0, 4>([&](auto kc) {
        constexpr int kk = decltype(kc)::value;
        const uint32_t c = planar_from_masked<D>(quad_pixel<kk>(m));
        cq[kk] = c;
        bg[kk] = (uint32_t)row[c >> 3] >> (c & 7);
      });
      st_stream4(fdst(f0 + j), pack_mask4(bg[0], bg[1], bg[2], bg[3]));
      if (ctab)
        *reinterpret_cast<uint2 *>(ctab[f0 + j] + pq) = make_uint2(cq[0] | (cq[1] << 16), cq[2] | (cq[3] << 16));
    }
  };
  uint32_t wa[PF][3], wb[PF][3];
  load(wa, fb);
  for (int f0 = fb; f0 < fe; f0 += 2 * PF) {
    load(wb, f0 + PF);
    work(wa, f0);
    if (f0 + PF >= fe) break;
    load(wa, f0 + 2 * PF);
    work(wb, f0 + PF);
  }
}

// Kept-leaf lists: a location's entry of the index is 8 u16 planar codes
// (16 B), of which only the first KL (2, 4 or 8: the build's candidate count)
// can be kept leaves; the rest are kKeptNone.  They are unpacked into one
// register per code, in the form a pixel's leaf takes before its planar code
// is formed: r_d | g_d << 8 | b_d << 16 | b_d << 24 (what group_pixel and
// quad_pixel return from masked words).  A lookup is then KL integer compares
// of that word; an unused entry becomes 0xFFFFFFFF, which no pixel gives.
template <int D, int KL>
__device__ __forceinline__ void list_unpack(const uint4 v, uint32_t (&l)[KL]) {
  constexpr uint32_t M = (1u << D) - 1u;
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int e = 0; e < KL; ++e) {
    const uint32_t c = (w[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
    l[e] = c == kKeptNone ? 0xFFFFFFFFu : (c & M) | (((c >> D) & M) << 8) | (((c >> (2 * D)) & M) * 0x01010000u);
  }
}

template <int KL>
__device__ __forceinline__ bool list_holds(const uint32_t (&l)[KL], uint32_t t) {
  bool hit = false;
#pragma unroll
  for (int e = 0; e < KL; ++e) hit |= l[e] == t;
  return hit;
}

// Pixel regions, depth 4-5, model with a kept-leaf index (from the candidate
// build): as classify_pixel_tb_body, but a lookup compares the pixel's leaf
// with its location's kept leaves held in registers instead of gathering a
// byte of a 512 B / 4 KB row.
// ftab/mtab/ctab as in classify_block_tb_body.
template <int D, int PF, int KL>
__device__ __forceinline__ void classify_pixel_list_body(const uint8_t *__restrict__ frames, int F, int64_t hw,
                                                         const uint16_t *kept, uint8_t *__restrict__ mask,
                                                         int64_t tile, const uint8_t *const *ftab = nullptr,
                                                         uint8_t *const *mtab = nullptr,
                                                         uint16_t *const *ctab = nullptr) {
  const int lane = threadIdx.x & 31;
  const int64_t pq = tile * 128 + 4 * lane;
  if (pq >= hw) return;
  uint32_t lst[4][KL];
#pragma unroll
  for (int k = 0; k < 4; ++k) list_unpack<D, KL>(__ldg(reinterpret_cast<const uint4 *>(kept) + pq + k), lst[k]);
  const uint8_t *src = frames + pq * 3;
  uint8_t *dst = mask + pq;
  for (int f0 = 0; f0 < F; f0 += PF) {
    uint32_t w[PF][3];
#pragma unroll
    for (int j = 0; j < PF; ++j)
      if (f0 + j < F) {
        const uint8_t *sp = ftab ? ftab[f0 + j] + pq * 3 : src + (int64_t)(f0 + j) * hw * 3;
        w[j][0] = ld_stream4(sp), w[j][1] = ld_stream4(sp + 4), w[j][2] = ld_stream4(sp + 8);
      }
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      if (f0 + j >= F) break;
      uint32_t m[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) m[i] = (w[j][i] >> (8 - D)) & byte_mask(D);
      uint32_t bg[4];
      static_for<0, 4>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        bg[k] = list_holds<KL>(lst[k], quad_pixel<k>(m)) ? 1u : 0u;
      });
      st_stream4(mtab ? mtab[f0 + j] + pq : dst + (int64_t)(f0 + j) * hw, pack_mask4(bg[0], bg[1], bg[2], bg[3]));
      if (ctab) {
        uint32_t cq[4];
        static_for<0, 4>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          cq[k] = planar_from_masked<D>(quad_pixel<k>(m));
        });
        *reinterpret_cast<uint2 *>(ctab[f0 + j] + pq) = make_uint2(cq[0] | (cq[1] << 16), cq[2] | (cq[3] << 16));
      }
    }
  }
}

// Pixel regions, depth <= 3: as classify_pixel_tb_body, with the warp's 128
// rows (WPR <= 16 words each) staged in shared memory first, interleaved so
// that word w of the lane's k-th pixel sits at [(w * 4 + k) * 32 + lane]: every
// lookup of a warp instruction hits 32 different banks.  rows: this warp's
// 128 * WPR words.
template <int D, int PF>
__device__ __forceinline__ void classify_pixel_tbs_body(const uint8_t *__restrict__ frames, int F, int64_t hw,
                                                        const uint32_t *model, uint8_t *__restrict__ mask,
                                                        int64_t tile, uint32_t *rows) {
  constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  static_assert(D <= 3, "rows of at most 16 words");
  const int lane = threadIdx.x & 31;
  const int64_t p0 = tile * 128;
  const int64_t np = hw - p0 < 128 ? hw - p0 : 128;
  __syncwarp();
  for (int e = lane; e < np * WPR; e += 32) {  // coalesced: element e = pixel e / WPR, word e % WPR
    const int pl = e / WPR, w = e % WPR;
    rows[(w * 4 + (pl & 3)) * 32 + (pl >> 2)] = model[p0 * WPR + e];
  }
  __syncwarp();
  const int64_t pq = p0 + 4 * lane;
  if (pq >= hw) return;
  const uint8_t *src = frames + pq * 3;
  uint8_t *dst = mask + pq;
  for (int f0 = 0; f0 < F; f0 += PF) {
    uint32_t w[PF][3];
#pragma unroll
    for (int j = 0; j < PF; ++j)
      if (f0 + j < F) {
        const uint8_t *sp = src + (int64_t)(f0 + j) * hw * 3;
        w[j][0] = ld_stream4(sp), w[j][1] = ld_stream4(sp + 4), w[j][2] = ld_stream4(sp + 8);
      }
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      if (f0 + j >= F) break;
      uint32_t m[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) m[i] = (w[j][i] >> (8 - D)) & byte_mask(D);
      uint32_t bg[4];
      static_for<0, 4>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const uint32_t q = planar_from_masked<D>(quad_pixel<k>(m));
        const uint32_t v = rows[((q >> 5) * 4 + k) * 32 + lane];
        bg[k] = __funnelshift_r(v, v, q);
      });
      st_stream4(dst + (int64_t)(f0 + j) * hw, pack_mask4(bg[0], bg[1], bg[2], bg[3]));
    }
  }
}

// One pixel location per lane (a warp owns 32): a smaller model working set
// per warp than the 4-per-lane form, so more warps fit their lines in L1.
__device__ __forceinline__ uint32_t ld_stream1(const uint8_t *p) {
  uint32_t v;
  asm volatile("ld.global.cs.u8 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_stream1(uint8_t *p, uint32_t v) {
  asm volatile("st.global.cs.u8 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int D, int PF>
__device__ __forceinline__ void classify_pixel_tb1_body(const uint8_t *__restrict__ frames, int F, int64_t hw,
                                                        const uint32_t *model, uint8_t *__restrict__ mask,
                                                        int64_t tile) {
  constexpr int64_t WPR = D == 1 ? 1 : (int64_t)1 << (3 * D - 5);
  const int64_t p = tile * 32 + (threadIdx.x & 31);
  if (p >= hw) return;
  const uint8_t *row = reinterpret_cast<const uint8_t *>(model + p * WPR);
  const uint8_t *src = frames + p * 3;
  uint8_t *dst = mask + p;
  for (int f0 = 0; f0 < F; f0 += PF) {
    uint32_t y[PF];
#pragma unroll
    for (int j = 0; j < PF; ++j)
      if (f0 + j < F) {
        const uint8_t *s = src + (int64_t)(f0 + j) * hw * 3;
        y[j] = ld_stream1(s) | (ld_stream1(s + 1) << 8) | (ld_stream1(s + 2) << 16);
      }
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      if (f0 + j >= F) break;
      const uint32_t q = planar_code<D>(y[j]);
      st_stream1(dst + (int64_t)(f0 + j) * hw, ((~(uint32_t)row[q >> 3]) >> (q & 7)) & 1u);
    }
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

// Loads this thread's PPT pixels of one frame's tile from shared memory
// (thread tid holds pixels tid*PPT ..) and keeps the top D bits of each byte.
template <int D, int PPT>
__device__ __forceinline__ void tile_frame_words(const uint8_t *__restrict__ src, uint32_t (&w)[12]) {
  const int tid = threadIdx.x;
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
}

// Writes this thread's PPT mask bytes (bit 0 of fbit[j] = leaf kept).
template <int PPT>
__device__ __forceinline__ void store_tile_mask(uint8_t *__restrict__ dst, const uint32_t (&fbit)[PPT]) {
  const int tid = threadIdx.x;
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

// Classifies one frame of the tile from shared memory: thread (warp, lane)
// handles pixels (warp*32 + lane)*PPT + j of the tile.  cdst (or null): the
// tile's u16 leaf codes of this frame are written there too (16-byte aligned).
template <int D, int NW, int PPT, int S, int FPS>
__device__ __forceinline__ void classify_tile_frame(const uint8_t *__restrict__ src, const uint32_t *__restrict__ mrow,
                                                    uint8_t *__restrict__ dst, uint16_t *__restrict__ cdst = nullptr) {
  using C = TiledCfg<D, NW, PPT, S, FPS>;
  uint32_t fbit[PPT], q[PPT];
  uint32_t w[12];
  tile_frame_words<D, PPT>(src, w);
  // mrow points at word 0 of pixel j=0 for this lane; pixel j's word q>>5 is at
  // mrow[(j*WPR + (q>>5))*32]
  static_for<0, PPT>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    q[j] = planar_from_masked<D>(group_pixel<j>(w));
    const uint32_t v = mrow[(j * C::WPR + (q[j] >> 5)) * 32];
    fbit[j] = __funnelshift_r(v, v, q[j]);
  });
  store_tile_mask<PPT>(dst, fbit);
  if (cdst) {
    uint4 *c4 = reinterpret_cast<uint4 *>(cdst + threadIdx.x * PPT);
#pragma unroll
    for (int h = 0; h < PPT / 8; ++h)
      c4[h] = make_uint4(q[8 * h] | (q[8 * h + 1] << 16), q[8 * h + 2] | (q[8 * h + 3] << 16),
                         q[8 * h + 4] | (q[8 * h + 5] << 16), q[8 * h + 6] | (q[8 * h + 7] << 16));
  }
}

// As classify_tile_frame for depth 4-5 models with a kept-leaf index: pixel
// j's (at most KL) kept leaves sit in lst[j].
template <int D, int PPT, int KL>
__device__ __forceinline__ void classify_tile_frame_list(const uint8_t *__restrict__ src, const uint32_t (&lst)[PPT][KL],
                                                         uint8_t *__restrict__ dst) {
  uint32_t fbit[PPT];
  uint32_t w[12];
  tile_frame_words<D, PPT>(src, w);
  static_for<0, PPT>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    fbit[j] = list_holds<KL>(lst[j], group_pixel<j>(w)) ? 1u : 0u;
  });
  store_tile_mask<PPT>(dst, fbit);
}

// Warp-specialised form: NW classifying warps plus one copy warp.  The copy
// warp streams every group of the CTA's work range, refilling a stage as soon
// as all classifying warps have released it (mbarrier "empty"); classifying
// warps wait only on "full".  At a tile change the classifying warps (named
// barrier 1, the copy warp is not part of it) reload the tile's rows.  A
// timed-out wait raises a shared abort flag; the warps then run to the end
// without waiting, so no barrier is left short of arrivals.
//
// KL > 0 (depth 4-5, models with a kept-leaf index of KL codes per location):
// no rows in shared memory; each classifying thread holds the kept-leaf lists
// of its PPT locations in registers (read from `kept` at a tile change) and
// compares.
// ftab/mtab/ctab as in classify_block_tb_body (ctab only without KL).
template <int D, int NW, int PPT, int S, int FPS, int KL = 0>
__device__ __forceinline__ void classify_pixel_ws_body(const uint8_t *__restrict__ frames, int F, int64_t hw,
                                                       int64_t ntiles, const uint32_t *model,
                                                       uint8_t *__restrict__ mask, int64_t vb, int64_t vg,
                                                       unsigned int *timeout_flag, const uint16_t *kept = nullptr,
                                                       const uint8_t *const *ftab = nullptr,
                                                       uint8_t *const *mtab = nullptr,
                                                       uint16_t *const *ctab = nullptr) {
  using C = TiledCfg<D, NW, PPT, S, FPS>;
  constexpr bool LIST = KL > 0;
  constexpr size_t MODEL_BYTES = LIST ? 0 : (size_t)C::MODEL_WORDS * 4;
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *msm = reinterpret_cast<uint32_t *>(smem);
  uint8_t *stages = smem + MODEL_BYTES;
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
  const int64_t u_begin = U * vb / vg;
  const int64_t u_end = U * (vb + 1) / vg;

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
          atomicExch(timeout_flag, 1u);
          abort_flag = 1;
          break;
        }
        const int f0 = fa + g * FPS;
        const int nf = (nfr - g * FPS) < FPS ? (nfr - g * FPS) : FPS;
        const uint32_t bar = smem_addr(&full[s]);
        mbar_expect_tx(bar, (uint32_t)(nf * C::FRAME_BYTES));
        for (int i = 0; i < nf; ++i)
          bulk_g2s(smem_addr(stages + (size_t)s * C::STAGE + (size_t)i * C::FRAME_BYTES),
                   ftab ? ftab[f0 + i] + tile * C::TILE * 3 : base + (int64_t)(f0 + i) * hw * 3, C::FRAME_BYTES,
                   bar);
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
  uint32_t lst[LIST ? PPT : 1][LIST ? KL : 1];
  int s = 0;
  uint32_t round = 0;
  for (int64_t u = u_begin; u < u_end;) {
    const int64_t tile = u / F;
    const int fa = (int)(u - tile * F);
    const int nfr = (int)((u_end - u) < (int64_t)(F - fa) ? (u_end - u) : (int64_t)(F - fa));
    const int64_t p_tile = tile * C::TILE;
    if constexpr (LIST) {
      const uint4 *k4 = reinterpret_cast<const uint4 *>(kept) + p_tile + (int64_t)tid * PPT;
#pragma unroll
      for (int j = 0; j < PPT; ++j) list_unpack<D, KL>(__ldg(k4 + j), lst[j]);
    } else {
      named_sync(1, NW * 32);  // every warp is done with the previous tile's rows
      {
        const uint32_t *src = model + (p_tile + (int64_t)tid * PPT) * C::WPR;
        if constexpr (C::WPR % 4 == 0) {
          const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
#pragma unroll 4
          for (int i = 0; i < PPT * C::WPR / 4; ++i) {
            const uint4 v = s4[i];
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
            msm[((warp * PPT + j) * C::WPR + w) * 32 + lane] = src[idx];
          }
        }
      }
      named_sync(1, NW * 32);
    }
    for (int g = 0; g * FPS < nfr; ++g) {
      const int f0 = fa + g * FPS;
      const int nf = (nfr - g * FPS) < FPS ? (nfr - g * FPS) : FPS;
      if (!abort_flag) {
        if (mbar_wait_bounded(smem_addr(&full[s]), round & 1, kWaitLimitNs)) {
          const uint8_t *stage = stages + (size_t)s * C::STAGE;
#pragma unroll
          for (int i = 0; i < FPS; ++i)
            if (i < nf) {
              uint8_t *md = mtab ? mtab[f0 + i] + p_tile : mask + (int64_t)(f0 + i) * hw + p_tile;
              if constexpr (LIST)
                classify_tile_frame_list<D, PPT, KL>(stage + (size_t)i * C::FRAME_BYTES, lst, md);
              else
                classify_tile_frame<D, NW, PPT, S, FPS>(stage + (size_t)i * C::FRAME_BYTES, mrow, md,
                                                        ctab ? ctab[f0 + i] + p_tile : nullptr);
            }
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
        } else {
          atomicExch(timeout_flag, 1u);
          abort_flag = 1;
        }
      }
      if (++s == S) s = 0, ++round;
    }
    u += nfr;
  }
}

// ---- block regions: strips of whole blocks, warp-specialised ----------------------
// A tile is bh rows (one row of blocks, bh = b except at the bottom edge) by
// wt pixels (a whole number of blocks, wt*bh <= 1024).  The tile's block rows
// stay in shared memory while its frames stream through the stage ring: the
// copy warp issues one bulk copy per pixel row of the tile per frame.  A
// classifying thread handles 8 consecutive pixels of one row, all inside one
// block (b % 8 == 0).  Requires W % 16 == 0, b % 8 == 0, aligned buffers.
__host__ __device__ __forceinline__ size_t classify_block_ws_rows_bytes(int b, int wt, int wpr) {
  return (((size_t)((wt + b - 1) / b) * wpr * 4) + 127) & ~(size_t)127;
}

template <int D, int S, int FPS>
__device__ __forceinline__ void classify_block_ws_body(const uint8_t *__restrict__ frames, int F, int H, int W, int b,
                                                       int wt, int ntx, int64_t ntiles,
                                                       const uint32_t *model,
                                                       uint8_t *__restrict__ mask, int64_t vb, int64_t vg,
                                                       unsigned int *timeout_flag) {
  constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  constexpr int TILE_BYTES = 1024 * 3;  // largest tile of one frame
  constexpr int STAGE = TILE_BYTES * FPS;
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *rows = reinterpret_cast<uint32_t *>(smem);
  uint8_t *stages = smem + classify_block_ws_rows_bytes(b, wt, WPR);
  uint64_t *full = reinterpret_cast<uint64_t *>(stages + (size_t)S * STAGE);
  uint64_t *empty = full + S;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x;
  const int bw = (W + b - 1) / b;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_addr(&full[s]), 1);
      mbar_init(smem_addr(&empty[s]), 4);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t U = ntiles * (int64_t)F;
  const int64_t u_begin = U * vb / vg;
  const int64_t u_end = U * (vb + 1) / vg;

  if (tid >= 128) {  // ---- copy warp ----
    if (tid != 128) return;
    int s = 0;
    uint32_t round = 0;
    for (int64_t u = u_begin; u < u_end && !abort_flag;) {
      const int64_t tile = u / F;
      const int fa = (int)(u - tile * F);
      const int nfr = (int)((u_end - u) < (int64_t)(F - fa) ? (u_end - u) : (int64_t)(F - fa));
      const int ty = (int)(tile / ntx), tx = (int)(tile % ntx);
      const int y0 = ty * b, x0 = tx * wt;
      const int bh = min(b, H - y0), wtt = min(wt, W - x0);
      const uint32_t rowb = (uint32_t)wtt * 3;
      for (int g = 0; g * FPS < nfr; ++g) {
        if (round > 0 && !mbar_wait_bounded(smem_addr(&empty[s]), (round - 1) & 1, kWaitLimitNs)) {
          atomicExch(timeout_flag, 1u);
          abort_flag = 1;
          break;
        }
        const int f0 = fa + g * FPS;
        const int nf = (nfr - g * FPS) < FPS ? (nfr - g * FPS) : FPS;
        const uint32_t bar = smem_addr(&full[s]);
        mbar_expect_tx(bar, (uint32_t)nf * bh * rowb);
        for (int i = 0; i < nf; ++i)
          for (int r = 0; r < bh; ++r)
            bulk_g2s(smem_addr(stages + (size_t)s * STAGE + (size_t)i * TILE_BYTES + (size_t)r * rowb),
                     frames + (((int64_t)(f0 + i) * H + y0 + r) * W + x0) * 3, rowb, bar);
        if (++s == S) s = 0, ++round;
      }
      u += nfr;
    }
    for (int k = 0; k < S; ++k) {
      const uint32_t fills = round + (k < s ? 1u : 0u);
      if (fills > 0) mbar_wait_bounded(smem_addr(&full[k]), (fills - 1) & 1, kWaitLimitNs);
    }
    return;
  }

  // ---- classifying warps: thread tid handles pixel group tid (8 pixels) ----
  const int lane = tid & 31;
  int s = 0;
  uint32_t round = 0;
  for (int64_t u = u_begin; u < u_end;) {
    const int64_t tile = u / F;
    const int fa = (int)(u - tile * F);
    const int nfr = (int)((u_end - u) < (int64_t)(F - fa) ? (u_end - u) : (int64_t)(F - fa));
    const int ty = (int)(tile / ntx), tx = (int)(tile % ntx);
    const int y0 = ty * b, x0 = tx * wt;
    const int bh = min(b, H - y0), wtt = min(wt, W - x0);
    const int gpr = wtt / 8;  // pixel groups per row
    const int nblk = (wtt + b - 1) / b;
    named_sync(1, 128);
    for (int i = tid; i < nblk * WPR; i += 128) {
      const int j = i / WPR, w = i % WPR;
      rows[i] = *(model + ((int64_t)ty * bw + (x0 / b) + j) * WPR + w);
    }
    named_sync(1, 128);
    const bool act = tid < bh * gpr;
    const int r = act ? tid / gpr : 0, gx = act ? tid % gpr : 0;
    const uint32_t *row = rows + ((gx * 8) / b) * WPR;
    const size_t soff = (size_t)r * wtt * 3 + (size_t)gx * 24;
    for (int g = 0; g * FPS < nfr; ++g) {
      const int f0 = fa + g * FPS;
      const int nf = (nfr - g * FPS) < FPS ? (nfr - g * FPS) : FPS;
      if (!abort_flag) {
        if (mbar_wait_bounded(smem_addr(&full[s]), round & 1, kWaitLimitNs)) {
          if (act) {
#pragma unroll
            for (int i = 0; i < FPS; ++i) {
              if (i < nf) {
                const uint2 *s2 = reinterpret_cast<const uint2 *>(stages + (size_t)s * STAGE + (size_t)i * TILE_BYTES + soff);
                const uint2 a = s2[0], bb = s2[1], c = s2[2];
                uint32_t w12[12] = {a.x, a.y, bb.x, bb.y, c.x, c.y, 0, 0, 0, 0, 0, 0};
#pragma unroll
                for (int e = 0; e < 6; ++e) w12[e] = (w12[e] >> (8 - D)) & byte_mask(D);
                uint32_t fbit[8];
                static_for<0, 8>([&](auto jc) {
                  constexpr int j = decltype(jc)::value;
                  const uint32_t q = planar_from_masked<D>(group_pixel<j>(w12));
                  const uint32_t v = row[q >> 5];
                  fbit[j] = __funnelshift_r(v, v, q);
                });
                const uint32_t x = pack_mask4(fbit[0], fbit[1], fbit[2], fbit[3]);
                const uint32_t y = pack_mask4(fbit[4], fbit[5], fbit[6], fbit[7]);
                uint8_t *dst = mask + ((int64_t)(f0 + i) * H + y0 + r) * W + x0 + gx * 8;
                asm volatile("st.global.cs.v2.u32 [%0], {%1,%2};" ::"l"(dst), "r"(x), "r"(y) : "memory");
              }
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
        } else {
          atomicExch(timeout_flag, 1u);
          abort_flag = 1;
        }
      }
      if (++s == S) s = 0, ++round;
    }
    u += nfr;
  }
}

// Tile width for block regions: the widest whole number of blocks, multiple of
// 16 pixels, with b*wt <= 1024 and the tile's rows in <= 64 KB; 0 if none.
inline int block_tile_width(int b, int d, int W) {
  if (b % 8 || b > 64 || W % 16) return 0;
  const int64_t rowb = wpr32(d) * 4;
  int best = 0;
  for (int wt = 16; b * wt <= 1024; wt += 16)
    if (wt % b == 0 && (int64_t)(wt / b) * rowb <= 64 * 1024) best = wt;
  if (best == 0) return 0;
  return best > W ? ((W + 15) / 16) * 16 : best;
}

}  // namespace ocq
