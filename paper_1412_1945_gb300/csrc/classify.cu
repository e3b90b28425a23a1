// S4: Check Color (Alg. 3) for every pixel of incoming frames (Sec. 4).
// A pixel is background when the bit of its leaf is set in its region's row.
//
// Kernels:
//   classify_generic_kernel      any region/depth: per-pixel global lookups.
//   classify_frame_kernel<D>     whole-frame regions, depth <= 6: the one row
//                                lives in shared memory (replicated per lane
//                                for depth <= 4 so lookups never conflict),
//                                frames stream through 16-byte loads.
//   classify_block_tb_kernel<D>  b x b blocks (b % 4 == 0), depth >= 4: as the
//                                per-pixel form, 8-warp CTAs over whole blocks.
//   classify_pixel_list_kernel   pixel regions, depth 4-5, models with a kept-leaf
//                                index: leaves compared in registers, no row gathers.
//   classify_pixel_wsl_kernel    the same lists in the warp-specialised bulk-copy
//                                form of classify_pixel_ws_kernel.
//   classify_pixel_tb_kernel     pixel regions, depth >= 4: a warp walks all
//                                frames of 32 or 128 pixel locations; their
//                                model sectors stay in L1 between frames.
//   classify_pixel_tiled_kernel  pixel regions, depth <= 3: temporal blocking.
//                                A CTA keeps the rows of a tile of pixel
//                                locations in shared memory (lane-interleaved:
//                                each lane's rows sit in its own bank) and
//                                streams that tile of many frames through a
//                                ring of stages filled by bulk asynchronous
//                                copies (cp.async.bulk + mbarrier), so each
//                                row is read from HBM about once per launch.
#include <algorithm>
#include <cstdint>

#include "classify_bodies.cuh"

namespace ocq {

// Set when a bounded wait gives up; read and cleared by device_status().
__device__ unsigned int g_classify_timeout;

// ---- plain kernels: one grid, virtual CTA = real CTA ----------------------------------

__global__ void classify_generic_kernel(const uint8_t *__restrict__ frames, int F, int H, int W, int kind, int block,
                                        int d, int64_t wpr, const uint32_t *__restrict__ model,
                                        uint8_t *__restrict__ mask, int64_t pb, int64_t pe) {
  classify_generic_body(frames, F, H, W, kind, block, d, wpr, model, mask, pb, pe, blockIdx.x, gridDim.x);
}

template <int D>
__global__ void __launch_bounds__(256) classify_frame_kernel(const uint8_t *__restrict__ frames, int64_t npix,
                                                             const uint32_t *__restrict__ model,
                                                             uint8_t *__restrict__ mask) {
  classify_frame_body<D>(frames, npix, model, mask, blockIdx.x, gridDim.x);
}

template <int D, int NW, int PPT, int S, int FPS>
__global__ void __launch_bounds__(NW * 32 + 32, 1)
    classify_pixel_ws_kernel(const uint8_t *__restrict__ frames, int F, int64_t hw, int64_t ntiles,
                             const uint32_t *__restrict__ model, uint8_t *__restrict__ mask) {
  classify_pixel_ws_body<D, NW, PPT, S, FPS>(frames, F, hw, ntiles, model, mask, blockIdx.x, gridDim.x,
                                             &g_classify_timeout);
}

// Pixel regions at any depth (used for depth >= 4): warps stride over
// 128-pixel tiles and walk all frames of each.
template <int D, int PXL, int PF>
__global__ void __launch_bounds__(128) classify_pixel_tb_kernel(const uint8_t *__restrict__ frames, int F,
                                                                int64_t hw, const uint32_t *__restrict__ model,
                                                                uint8_t *__restrict__ mask) {
  const int64_t tiles = (hw + 32 * PXL - 1) / (32 * PXL);
  const int64_t nw = (int64_t)gridDim.x * 4;
  for (int64_t t = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5); t < tiles; t += nw) {
    if constexpr (PXL == 4)
      classify_pixel_tb_body<D, PF>(frames, F, hw, model, mask, t);
    else
      classify_pixel_tb1_body<D, PF>(frames, F, hw, model, mask, t);
  }
}

// Item u = chunk * tiles + tile: frames [chunk * fchunk, chunk * fchunk +
// fchunk) of tile `tile` (one chunk of all F frames unless the frame is too
// small to give every warp of the grid a tile).
template <int D>
__global__ void __launch_bounds__(256) classify_block_tb_kernel(const uint8_t *__restrict__ frames, int F, int H,
                                                                int W, int b, int bw, int nseg, int64_t tiles,
                                                                int fchunk, int64_t items,
                                                                const uint32_t *__restrict__ model,
                                                                uint8_t *__restrict__ mask) {
  const int64_t nw = (int64_t)gridDim.x * 8;
  for (int64_t u = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); u < items; u += nw) {
    const int64_t c = u / tiles;
    const int f0 = (int)(c * fchunk);
    classify_block_tb_body<D, 4>(frames, F, H, W, b, bw, nseg, model, mask, u - c * tiles, f0, f0 + fchunk);
  }
}

// Pixel regions, depth 4-5, models with a kept-leaf index.
template <int D, int KL>
__global__ void __launch_bounds__(128) classify_pixel_list_kernel(const uint8_t *__restrict__ frames, int F,
                                                                  int64_t hw, const uint16_t *__restrict__ kept,
                                                                  uint8_t *__restrict__ mask) {
  const int64_t tiles = (hw + 127) / 128;
  const int64_t nw = (int64_t)gridDim.x * 4;
  for (int64_t t = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5); t < tiles; t += nw)
    classify_pixel_list_body<D, 8, KL>(frames, F, hw, kept, mask, t);
}

template <int D, int S, int FPS>
__global__ void __launch_bounds__(160, 1)
    classify_block_ws_kernel(const uint8_t *__restrict__ frames, int F, int H, int W, int b, int wt, int ntx,
                             int64_t ntiles, const uint32_t *__restrict__ model, uint8_t *__restrict__ mask) {
  classify_block_ws_body<D, S, FPS>(frames, F, H, W, b, wt, ntx, ntiles, model, mask, blockIdx.x, gridDim.x,
                                    &g_classify_timeout);
}

// ---- pixel regions: temporal blocking with bulk async copies (barrier form) ------------

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

// Pixel regions, depth 4-5, models with a kept-leaf index: the warp-specialised
// form with each location's kept leaves held in registers.
template <int D, int NW, int PPT, int S, int FPS, int KL>
__global__ void __launch_bounds__(NW * 32 + 32, 1)
    classify_pixel_wsl_kernel(const uint8_t *__restrict__ frames, int F, int64_t hw, int64_t ntiles,
                              const uint32_t *__restrict__ model, const uint16_t *__restrict__ kept,
                              uint8_t *__restrict__ mask) {
  classify_pixel_ws_body<D, NW, PPT, S, FPS, KL>(frames, F, hw, ntiles, model, mask, blockIdx.x, gridDim.x,
                                                 &g_classify_timeout, kept);
}

// Pixel regions, depth 4-5, kept-leaf index, any alignment: one pixel-frame per
// thread step over locations [pb, pe); the planar code is compared with the
// location's 8 list entries.
__global__ void __launch_bounds__(256) classify_list_generic_kernel(const uint8_t *__restrict__ frames, int F,
                                                                    int64_t hw, int d,
                                                                    const uint16_t *__restrict__ kept,
                                                                    uint8_t *__restrict__ mask, int64_t pb,
                                                                    int64_t pe) {
  const int64_t np = pe - pb, n = np * F;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = i / np, p = pb + i % np;
    const uint8_t *px = frames + (f * hw + p) * 3;
    const uint32_t q = planar_code_rt(px[0], px[1], px[2], d);
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(kept) + p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    bool hit = false;
#pragma unroll
    for (int e = 0; e < 8; ++e) hit |= ((w[e >> 1] >> (16 * (e & 1))) & 0xFFFFu) == q;
    mask[f * hw + p] = hit ? 0 : 1;
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

// Deep per-pixel classify variants: pixel locations per lane (4 or 1), frames
// prefetched, CTAs of 4 warps resident per SM.  Fewer resident pixel locations
// leave more L1 per location for its model lines.
struct DeepVariant {
  int pxl, pf, cps;
  ocq_status (*fn[5])(const ocq_model *, const uint8_t *, int, uint8_t *, int, cudaStream_t);
};

template <int D, int PXL, int PF>
static ocq_status launch_pixel_tb(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask, int cps,
                                  cudaStream_t st) {
  const int64_t hw = (int64_t)m->H * m->W;
  const int64_t ctas = (hw + 128 * PXL - 1) / (128 * PXL);
  const int64_t cap = (int64_t)sm_count() * cps;
  auto kern = classify_pixel_tb_kernel<D, PXL, PF>;
  static bool carved = false;
  if (!carved) {  // no shared memory: leave the whole unified array to L1
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    carved = true;
  }
  kern<<<(unsigned)(ctas < cap ? ctas : cap), 128, 0, st>>>(frames, F, hw, m->bits, mask);
  count_launch();
  return cuda_status(cudaGetLastError(), "classify_pixel_tb_kernel");
}

#define OCQ_DV(PXL, PF, CPS)                                                                              \
  DeepVariant {                                                                                          \
    PXL, PF, CPS, {                                                                                      \
      launch_pixel_tb<4, PXL, PF>, launch_pixel_tb<5, PXL, PF>, launch_pixel_tb<6, PXL, PF>,             \
          launch_pixel_tb<7, PXL, PF>, launch_pixel_tb<8, PXL, PF>                                       \
    }                                                                                                    \
  }
static const DeepVariant kDeepVariants[] = {OCQ_DV(4, 8, 2),   OCQ_DV(4, 8, 3),  OCQ_DV(4, 8, 4),
                                            OCQ_DV(1, 16, 4),  OCQ_DV(1, 16, 8), OCQ_DV(1, 16, 12),
                                            OCQ_DV(1, 16, 16), OCQ_DV(1, 8, 16)};
#undef OCQ_DV
static int g_deep_variant = 1;

int deep_variant_count() { return (int)(sizeof kDeepVariants / sizeof kDeepVariants[0]); }
int deep_variant_selected() { return g_deep_variant; }
bool deep_variant_select(int v) {
  if (v < 0 || v >= deep_variant_count()) return false;
  g_deep_variant = v;
  return true;
}
void deep_variant_describe(int v, int *pxl, int *pf, int *cps) {
  *pxl = kDeepVariants[v].pxl, *pf = kDeepVariants[v].pf, *cps = kDeepVariants[v].cps;
}

// Block classify form (see classify_block_tb_body): 0 = rows staged in shared
// memory (classify_block_ws_kernel), 1 = L1 (tb) for depth >= 4, 2 = L1 for
// depth >= 3 as well.
static int g_block_deep_form = 2;
static int g_block_tb_cps = 4;  // CTAs of 8 warps per SM

int block_form_count() { return 3; }
int block_form_selected() { return g_block_deep_form; }
bool block_form_select(int v) {
  if (v < 0 || v > 2) return false;
  g_block_deep_form = v;
  return true;
}

static ocq_status launch_list_generic(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask, int64_t pb,
                                      int64_t pe, cudaStream_t st) {
  if (pe <= pb) return OCQ_OK;
  classify_list_generic_kernel<<<grid_cap((pe - pb) * F, 256, 16), 256, 0, st>>>(
      frames, F, (int64_t)m->H * m->W, m->depth, m->kept, mask, pb, pe);
  count_launch();
  return cuda_status(cudaGetLastError(), "classify_list_generic_kernel");
}

template <int D, int NW, int PPT, int S, int FPS, int KL>
static ocq_status launch_list_ws_kl(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask,
                                    cudaStream_t st) {
  using C = TiledCfg<D, NW, PPT, S, FPS>;
  const int64_t hw = (int64_t)m->H * m->W;
  const size_t smem = (size_t)S * C::STAGE + (size_t)S * 16;
  const int64_t ntiles = hw / C::TILE;
  ocq_status rc = OCQ_OK;
  if (ntiles > 0) {
    auto kern = classify_pixel_wsl_kernel<D, NW, PPT, S, FPS, KL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e, "classify_pixel_wsl_kernel smem");
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::THREADS + 32, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sm_count() * per_sm;
    const int64_t U = ntiles * F;
    if (grid > U) grid = U;
    kern<<<(unsigned)grid, C::THREADS + 32, smem, st>>>(frames, F, hw, ntiles, m->bits, m->kept, mask);
    count_launch();
    rc = cuda_status(cudaGetLastError(), "classify_pixel_wsl_kernel");
  }
  if (rc == OCQ_OK) rc = launch_list_generic(m, frames, F, mask, ntiles * C::TILE, hw, st);
  return rc;
}

template <int D, int NW, int PPT, int S, int FPS>
static ocq_status launch_list_ws(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask, cudaStream_t st) {
  if (m->kept_len <= 2) return launch_list_ws_kl<D, NW, PPT, S, FPS, 2>(m, frames, F, mask, st);
  if (m->kept_len <= 4) return launch_list_ws_kl<D, NW, PPT, S, FPS, 4>(m, frames, F, mask, st);
  return launch_list_ws_kl<D, NW, PPT, S, FPS, 8>(m, frames, F, mask, st);
}

// Deep per-pixel classify forms for models with a kept-leaf index: 0 = from
// the rows (classify_pixel_tb_kernel), 1 = lists, one warp per 128 locations
// walking all frames (classify_pixel_list_kernel), 2-3 = lists, warp-
// specialised with bulk copies (classify_pixel_wsl_kernel; NW, PPT, S, FPS).
struct ListForm {
  int nw, ppt, stages, fps;
  ClassifyFn fn[2];  // depth 4, 5
};
#define OCQ_LF(NW, PPT, S, FPS) \
  { NW, PPT, S, FPS, {launch_list_ws<4, NW, PPT, S, FPS>, launch_list_ws<5, NW, PPT, S, FPS>} }
static const ListForm kListForms[] = {{0, 0, 0, 0, {nullptr, nullptr}}, {0, 0, 0, 0, {nullptr, nullptr}},
                                      OCQ_LF(4, 16, 3, 2), OCQ_LF(8, 8, 4, 2)};
#undef OCQ_LF
static int g_use_kept = 2;
int list_form_count() { return (int)(sizeof kListForms / sizeof kListForms[0]); }
int list_form_selected() { return g_use_kept; }
bool list_form_select(int v) {
  if (v < 0 || v >= list_form_count()) return false;
  g_use_kept = v;
  return true;
}
void list_form_describe(int v, int *nw, int *ppt, int *stages, int *fps) {
  *nw = kListForms[v].nw, *ppt = kListForms[v].ppt, *stages = kListForms[v].stages, *fps = kListForms[v].fps;
}

template <int D>
static ocq_status launch_pixel_list(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask,
                                   cudaStream_t st) {
  const int64_t hw = (int64_t)m->H * m->W;
  const int64_t ctas = (hw + 511) / 512;
  const int64_t cap = (int64_t)sm_count() * 8;
  const unsigned grid = (unsigned)(ctas < cap ? ctas : cap);
  if (m->kept_len <= 2)
    classify_pixel_list_kernel<D, 2><<<grid, 128, 0, st>>>(frames, F, hw, m->kept, mask);
  else if (m->kept_len <= 4)
    classify_pixel_list_kernel<D, 4><<<grid, 128, 0, st>>>(frames, F, hw, m->kept, mask);
  else
    classify_pixel_list_kernel<D, 8><<<grid, 128, 0, st>>>(frames, F, hw, m->kept, mask);
  count_launch();
  return cuda_status(cudaGetLastError(), "classify_pixel_list_kernel");
}

template <int D>
static ocq_status launch_block_tb(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask, cudaStream_t st) {
  const int bw = (m->W + m->block - 1) / m->block;
  const int bh = (m->H + m->block - 1) / m->block;
  const int nseg = (m->W + 127) / 128;
  const int64_t tiles = (int64_t)bh * nseg * m->block;
  const int64_t cap = (int64_t)sm_count() * g_block_tb_cps;
  // Split the frames when the tiles alone cannot give each warp of the grid
  // two items (a frame of a few hundred thousand pixels), in chunks of at
  // least 16 frames.
  int chunks = 1;
  if (tiles < 2 * cap * 8) chunks = (int)std::min<int64_t>((2 * cap * 8 + tiles - 1) / tiles, (F + 15) / 16);
  if (chunks < 1) chunks = 1;
  const int fchunk = (F + chunks - 1) / chunks;
  chunks = (F + fchunk - 1) / fchunk;
  const int64_t items = tiles * chunks;
  const int64_t ctas = (items + 7) / 8;
  static bool carved = false;
  if (!carved) {
    cudaFuncSetAttribute(classify_block_tb_kernel<D>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    carved = true;
  }
  classify_block_tb_kernel<D><<<(unsigned)(ctas < cap ? ctas : cap), 256, 0, st>>>(
      frames, F, m->H, m->W, m->block, bw, nseg, tiles, fchunk, items, m->bits, mask);
  count_launch();
  return cuda_status(cudaGetLastError(), "classify_block_tb_kernel");
}

template <int D>
static ocq_status launch_block_ws(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask, int wt,
                                  cudaStream_t st) {
  constexpr int S = 4, FPS = 4;
  constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  const int b = m->block;
  const int ntx = (m->W + wt - 1) / wt, nty = (m->H + b - 1) / b;
  const int64_t ntiles = (int64_t)ntx * nty;
  const size_t rows = classify_block_ws_rows_bytes(b, wt, WPR);
  const size_t smem = rows + (size_t)S * FPS * 1024 * 3 + (size_t)S * 16;
  auto kern = classify_block_ws_kernel<D, S, FPS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e, "classify_block_ws_kernel smem");
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 160, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)sm_count() * per_sm;
  if (grid > ntiles * F) grid = ntiles * F;
  kern<<<(unsigned)grid, 160, smem, st>>>(frames, F, m->H, m->W, b, wt, ntx, ntiles, m->bits, mask);
  count_launch();
  return cuda_status(cudaGetLastError(), "classify_block_ws_kernel");
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
  const bool aligned4 = ((reinterpret_cast<uintptr_t>(frames) | reinterpret_cast<uintptr_t>(mask)) & 3) == 0;
  const bool indexed = m->kind == OCQ_REGION_PIXEL && (d == 4 || d == 5) && m->kept && m->kept_len > 0;
  // a list model (no rows) always takes an index form; form 0 then acts as 1
  const int form = indexed && !m->bits && g_use_kept == 0 ? 1 : g_use_kept;
  if (indexed && form >= 2 && aligned && hw % 16 == 0)
    return kListForms[form].fn[d - 4](m, frames, F, mask, st);
  if (indexed && form && aligned4 && hw % 4 == 0)
    return d == 4 ? launch_pixel_list<4>(m, frames, F, mask, st) : launch_pixel_list<5>(m, frames, F, mask, st);
  if (indexed && !m->bits) return launch_list_generic(m, frames, F, mask, 0, hw, st);
  if (m->kind == OCQ_REGION_PIXEL && d >= 4 && aligned4 && hw % 4 == 0) {
    const DeepVariant &v = kDeepVariants[g_deep_variant];
    return v.fn[d - 4](m, frames, F, mask, v.cps, st);
  }
  const bool ws_ok = m->kind == OCQ_REGION_BLOCK && d <= 5 && aligned && block_tile_width(m->block, d, m->W) > 0;
  if (m->kind == OCQ_REGION_BLOCK && d >= 3 && m->block % 4 == 0 && m->W % 4 == 0 && aligned4 &&
      (!ws_ok || (d >= 4 && g_block_deep_form >= 1) || g_block_deep_form == 2)) {
    switch (d) {
      case 3: return launch_block_tb<3>(m, frames, F, mask, st);
      case 4: return launch_block_tb<4>(m, frames, F, mask, st);
      case 5: return launch_block_tb<5>(m, frames, F, mask, st);
      case 6: return launch_block_tb<6>(m, frames, F, mask, st);
      case 7: return launch_block_tb<7>(m, frames, F, mask, st);
      default: return launch_block_tb<8>(m, frames, F, mask, st);
    }
  }
  if (m->kind == OCQ_REGION_BLOCK && d <= 5 && aligned) {
    const int wt = block_tile_width(m->block, d, m->W);
    if (wt > 0) {
      switch (d) {
        case 1: return launch_block_ws<1>(m, frames, F, mask, wt, st);
        case 2: return launch_block_ws<2>(m, frames, F, mask, wt, st);
        case 3: return launch_block_ws<3>(m, frames, F, mask, wt, st);
        case 4: return launch_block_ws<4>(m, frames, F, mask, wt, st);
        default: return launch_block_ws<5>(m, frames, F, mask, wt, st);
      }
    }
  }
  return launch_generic(m, frames, F, mask, 0, hw, st);
}

bool classify_take_timeout() {
  unsigned int flag = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&flag, g_classify_timeout, sizeof flag) != cudaSuccess) return false;
  if (flag) cudaMemcpyToSymbol(g_classify_timeout, &zero, sizeof zero);
  return flag != 0;
}

}  // namespace ocq
