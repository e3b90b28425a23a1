// S2 (per-frame leaf sets, Alg. 1 per frame and region) and S3 (merge by
// frequency, Alg. 2) on the GPU.
//
// Merge Trees keeps a leaf exactly when at least T of the N per-frame trees
// contain it (every tree holding a leaf holds all its ancestors, so the
// level-by-level test never rejects an ancestor of a kept leaf).  The kernels
// therefore count, per region and leaf, the frames whose tree holds the leaf,
// and compare with T:
//   * whole-frame regions (and large-depth blocks): per-frame leaf bitsets in
//     global scratch, folded into bit-sliced counters (32 leaves per word);
//   * block regions, depth <= 5: one CTA per block, per-frame bitset and
//     bit-sliced counters in shared memory;
//   * pixel regions, depth <= 3: one thread per pixel location with private
//     byte (or u16) counters for all 8^d leaves in shared memory;
//   * pixel regions, depth >= 4: per-thread counters for 512-leaf chunks, only
//     for chunks the pixel's N colours touch.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "build_bodies.cuh"

namespace ocq {

// Set when a bounded wait gives up; read and cleared by build_take_timeout().
__device__ unsigned int g_build_timeout;

static int bit_length(uint32_t v) {
  int n = 0;
  while (v) ++n, v >>= 1;
  return n;
}

// ---- plain kernels: one grid, virtual CTA = real CTA ----------------------------------

template <int D>
__global__ void __launch_bounds__(256) occ_frame_kernel(const uint8_t *__restrict__ frames, int64_t hw, int f0,
                                                        int64_t chunk, uint32_t *__restrict__ occ, int group) {
  occ_frame_body<D>(frames, hw, f0, chunk, occ, blockIdx.x, blockIdx.y, group);
}

__global__ void occ_global_kernel(const uint8_t *__restrict__ frames, int H, int W, int kind, int block, int d,
                                  int f0, int nf, int64_t R, int64_t wpr, uint32_t *__restrict__ occ, int group) {
  occ_global_body(frames, H, W, kind, block, d, f0, nf, R, wpr, occ, blockIdx.x, gridDim.x, group);
}

__global__ void planes_merge_kernel(const uint32_t *__restrict__ occ, int nb, int64_t nwords,
                                    uint32_t *__restrict__ planes, int P, int first, int last, uint32_t T,
                                    uint32_t *__restrict__ model) {
  planes_merge_body(occ, nb, nwords, planes, P, first, last, T, model, blockIdx.x, gridDim.x);
}

template <int D>
__global__ void __launch_bounds__(256) build_block_kernel(const uint8_t *__restrict__ frames, int N, int H, int W,
                                                          int b, int bw, int P, uint32_t T,
                                                          uint32_t *__restrict__ model, int64_t R) {
  build_block_body<D>(frames, N, H, W, b, bw, P, T, model, R, blockIdx.x, gridDim.x);
}

template <int D, int PPL>
__global__ void __launch_bounds__(256) build_block_warp_kernel(const uint8_t *__restrict__ frames, int N, int H, int W,
                                                               int b, int bw, uint32_t T,
                                                               uint32_t *__restrict__ model, int64_t R) {
  extern __shared__ uint32_t tabs[];
  constexpr int S = WarpTableCfg<D>::S;
  uint32_t *tab = tabs + (threadIdx.x >> 5) * S;
  for (int i = threadIdx.x & 31; i < S; i += 32) tab[i] = 0u;
  __syncwarp();
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  build_block_warp_body<D, PPL>(frames, N, H, W, b, bw, T, model, (int64_t)blockIdx.x * (blockDim.x >> 5) +
                                (threadIdx.x >> 5), R, nw, tab);
}

template <int D, int B, int PF>
__global__ void __launch_bounds__(BlockTileCfg<D, B>::WPC * 32, BlockTileCfg<D, B>::MINB) build_block_tile_kernel(const uint8_t *__restrict__ frames, int N, int H, int W,
                                                               int bw, uint32_t T, uint32_t *__restrict__ model,
                                                               int64_t ntiles) {
  extern __shared__ __align__(16) uint8_t tile_smem[];
  constexpr int WB = BlockTileCfg<D, B>::WARP_SMEM;
  uint8_t *wsm = tile_smem + (threadIdx.x >> 5) * WB;
  for (int i = threadIdx.x & 31; i < WB / 4; i += 32) reinterpret_cast<uint32_t *>(wsm)[i] = 0u;
  __syncwarp();
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  build_block_tile_body<D, B, PF>(frames, N, H, W, bw, T, model,
                                  (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), ntiles, nw, wsm);
}

template <int D>
__global__ void __launch_bounds__(256, 4) build_block_r8_kernel(const uint8_t *__restrict__ frames, int N, int H, int W,
                                                             int bw, uint32_t T, uint32_t *__restrict__ model,
                                                             int64_t R) {
  extern __shared__ __align__(16) uint8_t r8_smem[];
  constexpr int WB = BlockR8CfgD<D>::WARP_SMEM;
  uint8_t *wsm = r8_smem + (threadIdx.x >> 5) * WB;
  for (int i = threadIdx.x & 31; i < WB / 4; i += 32) reinterpret_cast<uint32_t *>(wsm)[i] = 0u;
  __syncwarp();
  build_block_r8_body<D>(frames, N, H, W, bw, T, model, (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5), R,
                         (int64_t)gridDim.x * 8, wsm);
}

template <int D, int B>
__global__ void __launch_bounds__(256, BlockFsCfg<D, B>::MINB) build_block_fs_kernel(const uint8_t *__restrict__ frames, int N, int H, int W,
                                                               int bw, uint32_t T, uint32_t *__restrict__ model,
                                                               int64_t ngroups) {
  extern __shared__ __align__(16) uint32_t fs_smem[];
  for (int i = threadIdx.x; i < BlockFsCfg<D, B>::SMEM / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(fs_smem)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  build_block_fs_body<D, B>(frames, N, H, W, bw, T, model, ngroups, blockIdx.x, gridDim.x, fs_smem);
}

template <int D, int KM, bool GRP>
__global__ void __launch_bounds__(128) build_pixel_mg_kernel(const uint8_t *__restrict__ frames, int N, int64_t hw,
                                                             uint32_t T, uint32_t *__restrict__ model, int group,
                                                             uint16_t *__restrict__ kept) {
  extern __shared__ __align__(16) uint8_t mg_smem[];
  leaf_t<D> *codes = reinterpret_cast<leaf_t<D> *>(mg_smem) + (size_t)(threadIdx.x >> 5) * N * 32;
  build_pixel_mg_body<D, KM, GRP>(frames, N, hw, T, model, (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5), codes,
                                  group, kept);
}

template <int D, bool WIDE>
__global__ void __launch_bounds__(128) build_pixel_counters_kernel(const uint8_t *__restrict__ frames, int N,
                                                                   int64_t hw, int64_t p_begin, uint32_t T,
                                                                   uint32_t *__restrict__ model) {
  build_pixel_counters_body<D, WIDE>(frames, N, hw, p_begin, T, model, blockIdx.x);
}

template <int D>
__global__ void __launch_bounds__(64) build_pixel_chunked_kernel(const uint8_t *__restrict__ frames, int N,
                                                                 int64_t hw, uint32_t T, uint32_t *__restrict__ model,
                                                                 uint32_t *__restrict__ touched_g) {
  build_pixel_chunked_body<D>(frames, N, hw, T, model, touched_g, blockIdx.x);
}

template <int D, int NT, int FPS, int S, bool TENSOR, bool KEPT>
__global__ void __launch_bounds__(NT + 32) build_pixel_ws_kernel(const uint8_t *__restrict__ frames, int N, int64_t hw,
                                                                 int64_t ntiles, uint32_t T,
                                                                 uint32_t *__restrict__ model,
                                                                 const __grid_constant__ CUtensorMap tmap) {
  build_pixel_ws_body<D, NT, FPS, S, TENSOR, KEPT>(frames, N, hw, ntiles, T, model, &tmap, blockIdx.x, gridDim.x,
                                                   &g_build_timeout);
}

// Same counting with the frames staged by bulk asynchronous copies.  A
// persistent CTA of NT threads owns NT-pixel tiles; thread 0 streams each
// tile's rows of FPS frames per stage into a ring of S stages (mbarrier
// completion, bounded waits) while every thread counts its pixel from shared
// memory.  Counters are CB-bit (4 or 8) and saturate at T, which keeps the
// test count >= T exact.  A per-pixel "touched" bitset records which leaves
// occurred, so the end of a tile visits only those leaves, and leaves their
// counters at zero for the next tile.  Requires frames 16-byte aligned and
// H*W % 16 == 0; covers full tiles only.
// TENSOR: each stage is one 2-D tensor copy (TMA) of a box of FPS frame rows x
// ROW bytes, instead of FPS row copies.
template <int D, int CB, int NT, int FPS, int S>
struct StagedBuildCfg {
  static constexpr int NC = 1 << (3 * D);
  static constexpr int CPW = 32 / CB;                  // counters per word
  static constexpr int CW = (NC + CPW - 1) / CPW;      // counter words per pixel
  static constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  static constexpr int ROW = NT * 3;                   // bytes of one frame's tile
  static constexpr int STAGE = ROW * FPS;
  static constexpr size_t STATE = ((size_t)CW + WPR) * NT * 4;
  static constexpr size_t SMEM = STATE + 128 + (size_t)S * STAGE + (size_t)S * 8;
  static_assert(ROW % 128 == 0 && STAGE % 128 == 0, "stages stay 128-byte aligned");
};

template <int D, int CB, int NT, int FPS, int S, bool TENSOR>
__global__ void __launch_bounds__(NT) build_pixel_staged_kernel(const uint8_t *__restrict__ frames, int N, int64_t hw,
                                                                int64_t ntiles, uint32_t T,
                                                                uint32_t *__restrict__ model,
                                                                const __grid_constant__ CUtensorMap tmap) {
  using C = StagedBuildCfg<D, CB, NT, FPS, S>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);  // [CW][NT]
  uint32_t *touched = cnt + C::CW * NT;                // [WPR][NT]
  uint8_t *stages = smem + ((C::STATE + (128 - (smem_addr(smem) + C::STATE) % 128) % 128));
  uint64_t *bars = reinterpret_cast<uint64_t *>(stages + (size_t)S * C::STAGE);
  const int t = threadIdx.x;
  constexpr uint32_t CMASK = (1u << CB) - 1u;
  if (t == 0) {
    for (int s = 0; s < S; ++s) mbar_init(smem_addr(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
#pragma unroll 8
  for (int c = 0; c < C::CW; ++c) cnt[c * NT + t] = 0;
  __syncthreads();
  const int G = (N + FPS - 1) / FPS;  // stages per tile
  const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = my_tiles * G;

  auto issue = [&](int64_t k) {
    const int64_t i = k / G;
    const int g = (int)(k - i * G);
    const int64_t tile = blockIdx.x + i * gridDim.x;
    const int f0 = g * FPS;
    const int nf = N - f0 < FPS ? N - f0 : FPS;
    const int s = (int)(k % S);
    const uint32_t bar = smem_addr(&bars[s]);
    if constexpr (TENSOR) {
      // rows past frame N-1 are filled with zeros and still count as bytes
      mbar_expect_tx(bar, (uint32_t)C::STAGE);
      tensor2d_g2s(smem_addr(stages + (size_t)s * C::STAGE), &tmap, (int)(tile * (C::ROW / 4)), f0, bar);
    } else {
      mbar_expect_tx(bar, (uint32_t)(nf * C::ROW));
      for (int j = 0; j < nf; ++j)
        bulk_g2s(smem_addr(stages + (size_t)s * C::STAGE + (size_t)j * C::ROW),
                 frames + ((int64_t)(f0 + j) * hw + tile * NT) * 3, C::ROW, bar);
    }
  };
  if (t == 0)
    for (int64_t k = 0; k < total && k < S; ++k) issue(k);

  for (int64_t k = 0; k < total; ++k) {
    const int64_t i = k / G;
    const int g = (int)(k - i * G);
    if (g == 0) {
#pragma unroll
      for (int w = 0; w < C::WPR; ++w) touched[w * NT + t] = 0;
    }
    const int s = (int)(k % S);
    const bool ok = mbar_wait_bounded(smem_addr(&bars[s]), (uint32_t)((k / S) & 1), kWaitLimitNs);
    const uint8_t *stage = stages + (size_t)s * C::STAGE + 3 * t;
    const int nf = N - g * FPS < FPS ? N - g * FPS : FPS;
#pragma unroll
    for (int j = 0; j < FPS; ++j) {
      if (j < nf) {
        const uint8_t *px = stage + j * C::ROW;
        const uint32_t y = (uint32_t)px[0] | ((uint32_t)px[1] << 8) | ((uint32_t)px[2] << 16);
        const uint32_t q = planar_code<D>(y);
        uint32_t *cw = &cnt[(q / C::CPW) * NT + t];
        const uint32_t sh = (q % C::CPW) * CB;
        const uint32_t v = *cw;
        const uint32_t c = (v >> sh) & CMASK;
        if (c < T) *cw = v + (1u << sh);
        if (c == 0) touched[(q >> 5) * NT + t] |= 1u << (q & 31);
      }
    }
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        atomicExch(&g_build_timeout, 1u);
        for (int64_t kk = k; kk < total && kk < k + S; ++kk)
          mbar_wait_bounded(smem_addr(&bars[kk % S]), (uint32_t)((kk / S) & 1), kWaitLimitNs);
      }
      __syncthreads();
      return;
    }
    if (t == 0 && k + S < total) issue(k + S);
    if (g == G - 1) {
      const int64_t p = (blockIdx.x + i * gridDim.x) * NT + t;
      // the touched word w is replaced by model word w of this pixel
#pragma unroll 1
      for (int w = 0; w < C::WPR; ++w) {
        const uint32_t tb = touched[w * NT + t];
        uint32_t o = 0;
        for (uint32_t x = tb; x; x &= x - 1) {
          const uint32_t b = __ffs(x) - 1;
          const uint32_t q = (uint32_t)w * 32u + b;
          const uint32_t c = (cnt[(q / C::CPW) * NT + t] >> ((q % C::CPW) * CB)) & CMASK;
          o |= (uint32_t)(c >= T) << b;
        }
        for (uint32_t x = tb; x; x &= x - 1) {  // leave the counters at zero
          const uint32_t q = (uint32_t)w * 32u + (__ffs(x) - 1);
          cnt[(q / C::CPW) * NT + t] = 0;
        }
        touched[w * NT + t] = o;
      }
      uint32_t *dst = model + p * C::WPR;
      if constexpr (C::WPR % 4 == 0) {
#pragma unroll
        for (int w = 0; w < C::WPR; w += 4)
          *reinterpret_cast<uint4 *>(dst + w) = make_uint4(touched[w * NT + t], touched[(w + 1) * NT + t],
                                                           touched[(w + 2) * NT + t], touched[(w + 3) * NT + t]);
      } else {
#pragma unroll
        for (int w = 0; w < C::WPR; ++w) dst[w] = touched[w * NT + t];
      }
    }
  }
}

// Byte counters bumped with shared-memory reductions (red.shared.add, no
// return value), so successive frames of one pixel do not form a
// read-modify-write chain.  Counts stay <= N <= 255.  Each thread keeps a
// 16-bit mask of the model words (32 leaves each) its pixel touched; at the
// end of a tile only those words' counters are read, thresholded and zeroed.
// Same staging, alignment and coverage rules as build_pixel_staged_kernel.
template <int D, int NT, int FPS, int S>
struct RedBuildCfg {
  static constexpr int NC = 1 << (3 * D);
  static constexpr int CW = (NC + 3) / 4;  // u8 counter words per pixel
  static constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  static constexpr int ROW = NT * 3;
  static constexpr int STAGE = ROW * FPS;
  static constexpr size_t STATE = (size_t)CW * NT * 4;
  static constexpr size_t SMEM = STATE + 128 + (size_t)S * STAGE + (size_t)S * 8;
  static_assert(ROW % 128 == 0, "stages stay 128-byte aligned");
};

template <int D, int NT, int FPS, int S>
__global__ void __launch_bounds__(NT) build_pixel_red_kernel(const uint8_t *__restrict__ frames, int N, int64_t hw,
                                                             int64_t ntiles, uint32_t T,
                                                             uint32_t *__restrict__ model) {
  using C = RedBuildCfg<D, NT, FPS, S>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);  // [CW][NT]
  uint8_t *stages = smem + ((C::STATE + (128 - (smem_addr(smem) + C::STATE) % 128) % 128));
  uint64_t *bars = reinterpret_cast<uint64_t *>(stages + (size_t)S * C::STAGE);
  const int t = threadIdx.x;
  if (t == 0) {
    for (int s = 0; s < S; ++s) mbar_init(smem_addr(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
#pragma unroll 8
  for (int c = 0; c < C::CW; ++c) cnt[c * NT + t] = 0;
  __syncthreads();
  const int G = (N + FPS - 1) / FPS;
  const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = my_tiles * G;
  auto issue = [&](int64_t k) {
    const int64_t i = k / G;
    const int g = (int)(k - i * G);
    const int64_t tile = blockIdx.x + i * gridDim.x;
    const int f0 = g * FPS;
    const int nf = N - f0 < FPS ? N - f0 : FPS;
    const int s = (int)(k % S);
    const uint32_t bar = smem_addr(&bars[s]);
    mbar_expect_tx(bar, (uint32_t)(nf * C::ROW));
    for (int j = 0; j < nf; ++j)
      bulk_g2s(smem_addr(stages + (size_t)s * C::STAGE + (size_t)j * C::ROW),
               frames + ((int64_t)(f0 + j) * hw + tile * NT) * 3, C::ROW, bar);
  };
  if (t == 0)
    for (int64_t k = 0; k < total && k < S; ++k) issue(k);

  uint32_t words = 0;  // model words (32 leaves each) this pixel touched in the current tile
  for (int64_t k = 0; k < total; ++k) {
    const int64_t i = k / G;
    const int g = (int)(k - i * G);
    const int s = (int)(k % S);
    const bool ok = mbar_wait_bounded(smem_addr(&bars[s]), (uint32_t)((k / S) & 1), kWaitLimitNs);
    const uint8_t *stage = stages + (size_t)s * C::STAGE + 3 * t;
    const int nf = N - g * FPS < FPS ? N - g * FPS : FPS;
#pragma unroll
    for (int j = 0; j < FPS; ++j) {
      if (j < nf) {
        const uint8_t *px = stage + j * C::ROW;
        const uint32_t y = (uint32_t)px[0] | ((uint32_t)px[1] << 8) | ((uint32_t)px[2] << 16);
        const uint32_t q = planar_code<D>(y);
        red_add_shared(&cnt[(q >> 2) * NT + t], 1u << ((q & 3u) * 8));
        words |= 1u << (q >> 5);
      }
    }
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        atomicExch(&g_build_timeout, 1u);
        for (int64_t kk = k; kk < total && kk < k + S; ++kk)
          mbar_wait_bounded(smem_addr(&bars[kk % S]), (uint32_t)((kk / S) & 1), kWaitLimitNs);
      }
      __syncthreads();
      return;
    }
    if (t == 0 && k + S < total) issue(k + S);
    if (g == G - 1) {
      uint32_t *dst = model + ((blockIdx.x + i * gridDim.x) * NT + t) * C::WPR;
      if constexpr (C::WPR % 4 == 0) {
#pragma unroll
        for (int w = 0; w < C::WPR; w += 4) *reinterpret_cast<uint4 *>(dst + w) = make_uint4(0, 0, 0, 0);
      } else {
#pragma unroll
        for (int w = 0; w < C::WPR; ++w) dst[w] = 0;
      }
      for (; words; words &= words - 1) {
        const int w = __ffs(words) - 1;
        uint32_t o = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          if (w * 8 + c < C::CW) {
            uint32_t *cp = &cnt[(w * 8 + c) * NT + t];
            const uint32_t v = *cp;
            if (v) {
              const uint32_t ge = __vcmpgeu4(v, T * 0x01010101u);
              o |= (((ge >> 7) & 1u) | ((ge >> 14) & 2u) | ((ge >> 21) & 4u) | ((ge >> 28) & 8u)) << (4 * c);
              *cp = 0;
            }
          }
        }
        dst[w] = o;
      }
    }
  }
}

// Direct-load form: one CTA of NT threads per NT-pixel tile, no staging ring.
// Each thread prefetches its pixel's bytes of PF frames into registers, then
// counts them in its private column of CB-bit counters (saturating at T) and
// sets the leaf's bit in a private "kept" row the moment its count reaches T.
// All shared memory is counter state, so a SM keeps many pixels in flight.
template <int D, int CB, int NT, int PF>
struct DirectBuildCfg {
  static constexpr int NC = 1 << (3 * D);
  static constexpr int CPW = 32 / CB;
  static constexpr int CW = (NC + CPW - 1) / CPW;
  static constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  static constexpr size_t SMEM = ((size_t)CW + WPR) * NT * 4;
};

template <int D, int CB, int NT, int PF>
__global__ void __launch_bounds__(NT) build_pixel_direct_kernel(const uint8_t *__restrict__ frames, int N, int64_t hw,
                                                                int64_t p_begin, uint32_t T,
                                                                uint32_t *__restrict__ model) {
  using C = DirectBuildCfg<D, CB, NT, PF>;
  extern __shared__ uint32_t sm[];
  uint32_t *cnt = sm;                    // [CW][NT]
  uint32_t *kept = sm + C::CW * NT;      // [WPR][NT]
  constexpr uint32_t CMASK = (1u << CB) - 1u;
  const int t = threadIdx.x;
  const int64_t p = p_begin + (int64_t)blockIdx.x * NT + t;
  if (p >= hw) return;  // columns are private: no CTA-wide synchronisation
#pragma unroll 8
  for (int c = 0; c < C::CW; ++c) cnt[c * NT + t] = 0;
#pragma unroll
  for (int w = 0; w < C::WPR; ++w) kept[w * NT + t] = 0;
  const uint8_t *px = frames + p * 3;
  const int64_t fstride = hw * 3;
  for (int f0 = 0; f0 < N; f0 += PF) {
    uint32_t y[PF];
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      if (f0 + j < N) {
        const uint8_t *s = px + (int64_t)(f0 + j) * fstride;
        y[j] = (uint32_t)__ldg(s) | ((uint32_t)__ldg(s + 1) << 8) | ((uint32_t)__ldg(s + 2) << 16);
      }
    }
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      if (f0 + j < N) {
        const uint32_t q = planar_code<D>(y[j]);
        uint32_t *cw = &cnt[(q / C::CPW) * NT + t];
        const uint32_t sh = (q % C::CPW) * CB;
        const uint32_t v = *cw;
        const uint32_t c = (v >> sh) & CMASK;
        if (c < T) {
          *cw = v + (1u << sh);
          if (c + 1 == T) kept[(q >> 5) * NT + t] |= 1u << (q & 31);
        }
      }
    }
  }
  uint32_t *dst = model + p * C::WPR;
  if constexpr (C::WPR % 4 == 0) {
#pragma unroll
    for (int w = 0; w < C::WPR; w += 4)
      *reinterpret_cast<uint4 *>(dst + w) =
          make_uint4(kept[w * NT + t], kept[(w + 1) * NT + t], kept[(w + 2) * NT + t], kept[(w + 3) * NT + t]);
  } else {
#pragma unroll
    for (int w = 0; w < C::WPR; ++w) dst[w] = kept[w * NT + t];
  }
}

// ---- host dispatch ----------------------------------------------------------------

static unsigned grid_cap(int64_t work, int threads, int per_sm) {
  int64_t b = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

template <int D>
static void launch_occ_frame(const uint8_t *frames, int64_t hw, int f0, int nf, uint32_t *occ, int group,
                             cudaStream_t st) {
  const int64_t chunk = 256 * 16 * 4;  // pixels per CTA (multiple of 16)
  constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  dim3 grid((unsigned)((hw + chunk - 1) / chunk), (unsigned)nf);
  occ_frame_kernel<D><<<grid, 256, WPR * 4, st>>>(frames, hw, f0, chunk, occ, group);
  count_launch();
}

ocq_status launch_merge_counts(const uint32_t *occ, int N, int64_t nwords, uint32_t T, uint32_t *model,
                               cudaStream_t st) {
  const int P = bit_length((uint32_t)N);
  planes_merge_kernel<<<grid_cap(nwords, 256, 8), 256, 0, st>>>(occ, N, nwords, nullptr, P, 1, 1, T, model);
  count_launch();
  return cuda_status(cudaGetLastError(), "planes_merge_kernel");
}

ocq_status launch_frame_occupancy(const uint8_t *frames, int n, int H, int W, int depth, uint32_t *occ,
                                  cudaStream_t st) {
  const int64_t hw = (int64_t)H * W;
  if (n <= 0 || hw <= 0) return OCQ_OK;
  switch (depth) {
    case 1: launch_occ_frame<1>(frames, hw, 0, n, occ, 1, st); break;
    case 2: launch_occ_frame<2>(frames, hw, 0, n, occ, 1, st); break;
    case 3: launch_occ_frame<3>(frames, hw, 0, n, occ, 1, st); break;
    case 4: launch_occ_frame<4>(frames, hw, 0, n, occ, 1, st); break;
    case 5: launch_occ_frame<5>(frames, hw, 0, n, occ, 1, st); break;
    case 6: launch_occ_frame<6>(frames, hw, 0, n, occ, 1, st); break;
    default:
      occ_global_kernel<<<grid_cap(hw * n, 256, 16), 256, 0, st>>>(frames, H, W, OCQ_REGION_FRAME, 0, depth, 0, n, 1,
                                                                   wpr32(depth), occ, 1);
      count_launch();
  }
  return cuda_status(cudaGetLastError(), "frame occupancy");
}

// Dense path: per-tree leaf bitsets in scratch, folded into bit-sliced
// counters.  One tree per group of `group` consecutive frames (Sec. 3; the
// last group holds the rest); T counts trees.  Scratch is batched by trees.
static ocq_status build_dense(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st, int group = 1) {
  const int G = (N + group - 1) / group;
  const int P = bit_length((uint32_t)G);
  const int64_t nwords = m->R * m->wpr;
  const int64_t hw = (int64_t)m->H * m->W;
  const int64_t budget = (int64_t)512 << 20;
  int nb = G;
  if ((int64_t)G * nwords * 4 > budget) nb = (int)(budget / (nwords * 4) > 0 ? budget / (nwords * 4) : 1);
  if (nb > G) nb = G;
  const bool multi = nb < G;
  uint32_t *occ = nullptr, *planes = nullptr;
  ocq_status rc = cuda_status(malloc_async((void **)&occ, (size_t)nb * nwords * 4, st), "build scratch");
  if (rc != OCQ_OK) return rc;
  if (multi) {
    rc = cuda_status(malloc_async((void **)&planes, (size_t)P * nwords * 4, st), "build counters");
    if (rc != OCQ_OK) {
      cudaFreeAsync(occ, st);
      return rc;
    }
  }
  for (int s0 = 0; s0 < G && rc == OCQ_OK; s0 += nb) {
    const int ns = G - s0 < nb ? G - s0 : nb;
    const int f0 = s0 * group;
    const int f1 = (s0 + ns) * group < N ? (s0 + ns) * group : N;
    const int nf = f1 - f0;
    rc = cuda_status(cudaMemsetAsync(occ, 0, (size_t)ns * nwords * 4, st), "clear occupancy");
    if (rc != OCQ_OK) break;
    if (m->kind == OCQ_REGION_FRAME && m->depth <= 6) {
      switch (m->depth) {
        case 1: launch_occ_frame<1>(frames, hw, f0, nf, occ, group, st); break;
        case 2: launch_occ_frame<2>(frames, hw, f0, nf, occ, group, st); break;
        case 3: launch_occ_frame<3>(frames, hw, f0, nf, occ, group, st); break;
        case 4: launch_occ_frame<4>(frames, hw, f0, nf, occ, group, st); break;
        case 5: launch_occ_frame<5>(frames, hw, f0, nf, occ, group, st); break;
        default: launch_occ_frame<6>(frames, hw, f0, nf, occ, group, st); break;
      }
    } else {
      occ_global_kernel<<<grid_cap(hw * nf, 256, 16), 256, 0, st>>>(frames, m->H, m->W, m->kind, m->block, m->depth,
                                                                     f0, nf, m->R, m->wpr, occ, group);
      count_launch();
    }
    rc = cuda_status(cudaGetLastError(), "occupancy kernel");
    if (rc != OCQ_OK) break;
    planes_merge_kernel<<<grid_cap(nwords, 256, 8), 256, 0, st>>>(occ, ns, nwords, planes, P, s0 == 0,
                                                                   s0 + ns >= G, (uint32_t)m->T, m->bits);
    count_launch();
    rc = cuda_status(cudaGetLastError(), "planes_merge_kernel");
  }
  cudaFreeAsync(occ, st);
  if (planes) cudaFreeAsync(planes, st);
  return rc;
}

template <int D>
static ocq_status launch_block(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  const int P = bit_length((uint32_t)N);
  const size_t smem = (size_t)WPR * (P + 2) * 4;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(build_block_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int bw = (m->W + m->block - 1) / m->block;
  const int threads = m->block * m->block >= 256 ? 256 : (m->block * m->block <= 32 ? 32 : ((m->block * m->block + 31) / 32) * 32);
  build_block_kernel<D><<<(unsigned)m->R, threads, smem, st>>>(frames, N, m->H, m->W, m->block, bw, P, (uint32_t)m->T,
                                                                m->bits, m->R);
  count_launch();
  return cuda_status(cudaGetLastError(), "build_block_kernel");
}

template <int D, int KM, bool GRP>
static ocq_status launch_pixel_mg_km(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st, int group) {
  const size_t smem = (size_t)4 * N * 32 * sizeof(leaf_t<D>);
  auto kern = build_pixel_mg_kernel<D, KM, GRP>;
  if (smem > 48 * 1024) {
    ocq_status rc = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                                "build_pixel_mg_kernel smem");
    if (rc != OCQ_OK) return rc;
  }
  const int64_t hw = (int64_t)m->H * m->W;
  constexpr bool kIndex = D >= 4 && D <= 5 && KM > 0;  // at most 8 kept leaves per location
  if (!kIndex && !m->bits) {
    set_error("internal: a list model needs the candidate build at depth 4-5 with floor(N/T) <= 8");
    return OCQ_EINVAL;
  }
  if (kIndex && !m->kept) {  // the kept-leaf index (16 B per location)
    ocq_status rc = cuda_status(malloc_async((void **)&m->kept, (size_t)hw * 8 * sizeof(uint16_t), st),
                                "kept-leaf index");
    if (rc != OCQ_OK) return rc;
  }
  m->kept_len = kIndex ? (KM < 2 ? 2 : KM) : 0;
  kern<<<(unsigned)((hw + 127) / 128), 128, smem, st>>>(frames, N, hw, (uint32_t)m->T, m->bits, group,
                                                         kIndex ? m->kept : nullptr);
  count_launch();
  return cuda_status(cudaGetLastError(), "build_pixel_mg_kernel");
}

// Candidate counters: the smallest of 1, 2, 4, 8 that is >= floor(N / T);
// beyond 8, every distinct leaf is counted (KM = 0).  group > 1: one tree per
// group of frames (T counts groups; the same bound holds).
template <int D, bool GRP>
static ocq_status launch_pixel_mg_g(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st, int group) {
  const int k = N / m->T;
  if (k <= 1) return launch_pixel_mg_km<D, 1, GRP>(frames, N, m, st, group);
  if (k <= 2) return launch_pixel_mg_km<D, 2, GRP>(frames, N, m, st, group);
  if (k <= 4) return launch_pixel_mg_km<D, 4, GRP>(frames, N, m, st, group);
  if (k <= 8) return launch_pixel_mg_km<D, 8, GRP>(frames, N, m, st, group);
  return launch_pixel_mg_km<D, 0, GRP>(frames, N, m, st, group);
}

template <int D>
static ocq_status launch_pixel_mg(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st, int group = 1) {
  return group > 1 ? launch_pixel_mg_g<D, true>(frames, N, m, st, group)
                   : launch_pixel_mg_g<D, false>(frames, N, m, st, 1);
}

// One warp per block region (b <= 16, N <= 255, frame offsets within 32 bits).
bool block_warp_ok(int N, int H, int W, int b) {
  return b <= 16 && N <= 255 && (int64_t)H * W * 3 <= (int64_t)UINT32_MAX;
}

template <int D, int PPL>
static ocq_status launch_block_warp_ppl(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  constexpr int S = WarpTableCfg<D>::S;
  constexpr size_t smem = (size_t)8 * S * 4;
  auto kern = build_block_warp_kernel<D, PPL>;
  static int cap = 0;
  if (!cap) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, smem);
    cap = (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
  }
  const int bw = (m->W + m->block - 1) / m->block;
  const int64_t ctas = (m->R + 7) / 8;
  kern<<<(unsigned)(ctas < cap ? ctas : cap), 256, smem, st>>>(frames, N, m->H, m->W, m->block, bw,
                                                               (uint32_t)m->T, m->bits, m->R);
  count_launch();
  return cuda_status(cudaGetLastError(), "build_block_warp_kernel");
}

// Block builds for b in {8, 16} (depth 2-5, N <= 255, W % 8 == 0, 8-byte
// aligned frames, frame offsets within 32 bits): warps over 16 x 16 pixel
// tiles, the frames split over the 8 warps of a CTA, or (8 x 8 at depth 5)
// one region per warp with two-level tables.  Form 1 (the default) picks by
// shape and size, from CUDA-event times of 30-frame builds at 320x240 ..
// 1920x1080 (cluster and sway scenes):
//   * 8 x 8 at depth 5: the two-level region tables (1080p 0.168 / 0.198 ms
//     against 0.224 / 0.274 ms one warp per region; 720p 0.106 against 0.133
//     frames split), frames split below 1024 tiles (320x240: 0.025 against
//     0.036 ms);
//   * frames split: 16 x 16 at depth 5 (1080p 0.19 against 0.25 ms for the
//     tiles), 8 x 8 at depth 4 (1080p 0.15 against 0.17 ms), and every frame
//     of fewer than 1024 tiles (320x240: 1.2-2.5x), where the tiles leave most
//     SMs idle;
//   * warp tiles: depth <= 3, and 16 x 16 at depth 4 (1080p 0.12 against
//     0.14 ms).
// Where other streams' kernels share the GPU (the batched forms), form 1
// takes the forms that do the least work per region instead: the tiles, and
// the region tables for 8 x 8 at depth 5 (64-stream mix, 8 x 8 d = 4 class in
// the graph of branches: frames split 0.36, tiles 0.32 ms).
// Forms 0, 2, 3 and 4 force one warp per region, frames split, tiles (8 x 8
// at depth 5: one warp per region) and the region tables (8 x 8 at depth 4
// or 5; at depth 4 they measured 0.17-0.18 ms at 1080p, no faster than the tiles and
// behind the frames split, so the default does not take them there).
static int g_block_form = 1;
static thread_local bool t_shared_gpu = false;
SharedGpuScope::SharedGpuScope() : prev(t_shared_gpu) { t_shared_gpu = true; }
SharedGpuScope::~SharedGpuScope() { t_shared_gpu = prev; }
static bool block_shape_ok(int N, int H, int W, int b, int depth, const void *frames) {
  return (b == 8 || b == 16) && depth >= 2 && depth <= 5 && N <= 255 && W % 8 == 0 &&
         (reinterpret_cast<uintptr_t>(frames) & 7) == 0 && (int64_t)H * W * 3 <= (int64_t)UINT32_MAX;
}
enum BlockBuildKind { BB_WARP = 0, BB_TILE, BB_FS, BB_R8 };
static BlockBuildKind block_build_kind(int N, int H, int W, int b, int depth, const void *frames) {
  if (g_block_form == 0 || !block_shape_ok(N, H, W, b, depth, frames)) return BB_WARP;
  if (g_block_form == 2) return BB_FS;
  if (g_block_form == 4) return b == 8 && depth >= 4 ? BB_R8 : BB_WARP;
  if (g_block_form == 3) return b == 8 && depth == 5 ? BB_WARP : BB_TILE;
  const int64_t tiles = (int64_t)((H + 15) / 16) * ((W + 15) / 16);
  if (b == 8 && depth == 5) return !t_shared_gpu && tiles < 1024 ? BB_FS : BB_R8;
  if (t_shared_gpu) return BB_TILE;
  if (tiles < 1024 || (b == 16 && depth == 5) || (b == 8 && depth == 4)) return BB_FS;
  return BB_TILE;
}
bool block_tile_ok(int N, int H, int W, int b, int depth, const void *frames) {
  return block_build_kind(N, H, W, b, depth, frames) == BB_TILE;
}
bool block_fs_ok(int N, int H, int W, int b, int depth, const void *frames) {
  return block_build_kind(N, H, W, b, depth, frames) == BB_FS;
}
bool block_r8_ok(int N, int H, int W, int b, int depth, const void *frames) {
  return block_build_kind(N, H, W, b, depth, frames) == BB_R8;
}
int block_build_form_count() { return 5; }
int block_build_form_selected() { return g_block_form; }
bool block_build_form_select(int v) {
  if (v < 0 || v > 4) return false;
  g_block_form = v;
  return true;
}

template <int D>
static ocq_status launch_block_r8_d(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  constexpr size_t smem = (size_t)8 * BlockR8CfgD<D>::WARP_SMEM;
  auto kern = build_block_r8_kernel<D>;
  static int cap = 0;
  if (!cap) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, smem);
    cap = (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
  }
  const int bw = m->W / 8;
  const int64_t R = (int64_t)((m->H + 7) / 8) * bw;
  const int64_t ctas = (R + 7) / 8;
  kern<<<(unsigned)(ctas < cap ? ctas : cap), 256, smem, st>>>(frames, N, m->H, m->W, bw, (uint32_t)m->T, m->bits, R);
  count_launch();
  return cuda_status(cudaGetLastError(), "build_block_r8_kernel");
}

static ocq_status launch_block_r8(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  return m->depth == 4 ? launch_block_r8_d<4>(frames, N, m, st) : launch_block_r8_d<5>(frames, N, m, st);
}

template <int D, int B>
static ocq_status launch_block_fs(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  using C = BlockFsCfg<D, B>;
  auto kern = build_block_fs_kernel<D, B>;
  static int cap = 0;
  if (!cap) {
    if (C::SMEM > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, C::SMEM);
    cap = (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
  }
  const int bw = (m->W + m->block - 1) / m->block;
  const int64_t ngroups = C::TILE ? (int64_t)((m->H + 15) / 16) * ((m->W + 15) / 16)
                                  : (int64_t)((m->H + 7) / 8) * (m->W / 8);
  kern<<<(unsigned)(ngroups < cap ? ngroups : cap), 256, C::SMEM, st>>>(frames, N, m->H, m->W, bw, (uint32_t)m->T,
                                                                        m->bits, ngroups);
  count_launch();
  return cuda_status(cudaGetLastError(), "build_block_fs_kernel");
}

template <int D>
static ocq_status launch_block_fs_b(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  return m->block == 8 ? launch_block_fs<D, 8>(frames, N, m, st) : launch_block_fs<D, 16>(frames, N, m, st);
}

template <int D, int B>
static ocq_status launch_block_tile(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  constexpr int PF = BlockTileCfg<D, B>::PF;
  constexpr int WPC = BlockTileCfg<D, B>::WPC;
  constexpr size_t smem = (size_t)WPC * BlockTileCfg<D, B>::WARP_SMEM;
  auto kern = build_block_tile_kernel<D, B, PF>;
  static int cap = 0;
  if (!cap) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, WPC * 32, smem);
    cap = (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
  }
  const int bw = (m->W + m->block - 1) / m->block;
  const int64_t ntiles = (int64_t)((m->H + 15) / 16) * ((m->W + 15) / 16);
  const int64_t ctas = (ntiles + WPC - 1) / WPC;
  kern<<<(unsigned)(ctas < cap ? ctas : cap), WPC * 32, smem, st>>>(frames, N, m->H, m->W, bw, (uint32_t)m->T,
                                                                    m->bits, ntiles);
  count_launch();
  return cuda_status(cudaGetLastError(), "build_block_tile_kernel");
}

template <int D>
static ocq_status launch_block_tile_b(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  return m->block == 8 ? launch_block_tile<D, 8>(frames, N, m, st) : launch_block_tile<D, 16>(frames, N, m, st);
}

template <int D>
static ocq_status launch_block_warp(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  const int npx = m->block * m->block;
  if (npx <= 32) return launch_block_warp_ppl<D, 1>(frames, N, m, st);
  if (npx <= 64) return launch_block_warp_ppl<D, 2>(frames, N, m, st);
  if (npx <= 128) return launch_block_warp_ppl<D, 4>(frames, N, m, st);
  return launch_block_warp_ppl<D, 8>(frames, N, m, st);
}

template <int D, bool WIDE>
static ocq_status launch_pixel_counters(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st,
                                        int64_t p_begin = 0) {
  constexpr int NC = 1 << (3 * D);
  constexpr int CPW = WIDE ? 2 : 4;
  constexpr int NW = (NC + CPW - 1) / CPW;
  const size_t smem = (size_t)NW * 128 * 4;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(build_pixel_counters_kernel<D, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  const int64_t hw = (int64_t)m->H * m->W;
  const int64_t n = hw - p_begin;
  if (n <= 0) return OCQ_OK;
  build_pixel_counters_kernel<D, WIDE>
      <<<(unsigned)((n + 127) / 128), 128, smem, st>>>(frames, N, hw, p_begin, (uint32_t)m->T, m->bits);
  count_launch();
  return cuda_status(cudaGetLastError(), "build_pixel_counters_kernel");
}

// Tensor map of the training frames as a 2-D array of u32: (H*W*3/4) x N,
// rows H*W*3 bytes apart, box (NT*3/4) x FPS.
// The driver's encoder is looked up through the runtime, so the library does
// not link libcuda directly (it loads on machines without a GPU driver).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

static bool encode_frames_map(CUtensorMap *map, const uint8_t *frames, int N, int64_t hw, int nt, int fps) {
  memset(map, 0, sizeof *map);
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(hw * 3 / 4), (cuuint64_t)N};
  const cuuint64_t strides[1] = {(cuuint64_t)(hw * 3)};
  const cuuint32_t box[2] = {(cuuint32_t)(nt * 3 / 4), (cuuint32_t)fps};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, (void *)frames, dims, strides, box, estr,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int D, int CB, int NT, int FPS, int S, bool TENSOR = false>
static ocq_status launch_pixel_staged(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  using C = StagedBuildCfg<D, CB, NT, FPS, S>;
  const int64_t hw = (int64_t)m->H * m->W;
  constexpr bool fits = C::SMEM <= 227 * 1024 && (!TENSOR || (NT * 3 / 4 <= 256 && FPS <= 256));
  const int64_t ntiles = fits ? hw / NT : 0;
  CUtensorMap map;
  memset(&map, 0, sizeof map);
  if (TENSOR && ntiles > 0 && !encode_frames_map(&map, frames, N, hw, NT, FPS)) {
    set_error("cuTensorMapEncodeTiled failed for the training frames");
    return OCQ_ECUDA;
  }
  if (ntiles > 0) {
    auto kern = build_pixel_staged_kernel<D, CB, NT, FPS, S, TENSOR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return cuda_status(e, "build_pixel_staged_kernel smem");
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, C::SMEM);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > ntiles) grid = ntiles;
    kern<<<(unsigned)grid, NT, C::SMEM, st>>>(frames, N, hw, ntiles, (uint32_t)m->T, m->bits, map);
    count_launch();
    ocq_status rc = cuda_status(cudaGetLastError(), "build_pixel_staged_kernel");
    if (rc != OCQ_OK) return rc;
  }
  if (N > 255) return launch_pixel_counters<D, true>(frames, N, m, st, ntiles * NT);
  return launch_pixel_counters<D, false>(frames, N, m, st, ntiles * NT);
}

template <int D>
static ocq_status launch_pixel_chunked(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  constexpr int NCH = 1 << (3 * D - 9);
  const int64_t hw = (int64_t)m->H * m->W;
  ocq_status rc = cuda_status(cudaMemsetAsync(m->bits, 0, m->bytes, st), "clear model");
  if (rc != OCQ_OK) return rc;
  uint32_t *touched = nullptr;
  if (NCH > 64) {
    const size_t tb = (size_t)hw * (NCH / 32) * 4;
    rc = cuda_status(malloc_async((void **)&touched, tb, st), "chunk bitmap");
    if (rc != OCQ_OK) return rc;
    rc = cuda_status(cudaMemsetAsync(touched, 0, tb, st), "clear chunk bitmap");
  }
  if (rc == OCQ_OK) {
    const size_t smem = 256 * 64 * 4;
    cudaFuncSetAttribute(build_pixel_chunked_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    build_pixel_chunked_kernel<D><<<(unsigned)((hw + 63) / 64), 64, smem, st>>>(frames, N, hw, (uint32_t)m->T,
                                                                                 m->bits, touched);
    count_launch();
    rc = cuda_status(cudaGetLastError(), "build_pixel_chunked_kernel");
  }
  if (touched) cudaFreeAsync(touched, st);
  return rc;
}

template <int D, int CB, int NT, int PF>
static ocq_status launch_pixel_direct(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  using C = DirectBuildCfg<D, CB, NT, PF>;
  const int64_t hw = (int64_t)m->H * m->W;
  auto kern = build_pixel_direct_kernel<D, CB, NT, PF>;
  if (C::SMEM > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return cuda_status(e, "build_pixel_direct_kernel smem");
  }
  kern<<<(unsigned)((hw + NT - 1) / NT), NT, C::SMEM, st>>>(frames, N, hw, 0, (uint32_t)m->T, m->bits);
  count_launch();
  return cuda_status(cudaGetLastError(), "build_pixel_direct_kernel");
}

template <int D, int NT, int FPS, int S, bool TENSOR, bool KEPT>
static ocq_status launch_pixel_ws(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  using C = WsBuildCfg<D, NT, FPS, S, KEPT>;
  if (N > 255) return launch_pixel_counters<D, true>(frames, N, m, st, 0);
  const int64_t hw = (int64_t)m->H * m->W;
  constexpr bool fits = C::SMEM <= 227 * 1024 && (!TENSOR || (NT * 3 / 4 <= 256 && FPS <= 256));
  const int64_t ntiles = fits ? hw / NT : 0;
  CUtensorMap map;
  memset(&map, 0, sizeof map);
  if (TENSOR && ntiles > 0 && !encode_frames_map(&map, frames, N, hw, NT, FPS)) {
    set_error("cuTensorMapEncodeTiled failed for the training frames");
    return OCQ_ECUDA;
  }
  if (ntiles > 0) {
    auto kern = build_pixel_ws_kernel<D, NT, FPS, S, TENSOR, KEPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return cuda_status(e, "build_pixel_ws_kernel smem");
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT + 32, C::SMEM);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > ntiles) grid = ntiles;
    kern<<<(unsigned)grid, NT + 32, C::SMEM, st>>>(frames, N, hw, ntiles, (uint32_t)m->T, m->bits, map);
    count_launch();
    ocq_status rc = cuda_status(cudaGetLastError(), "build_pixel_ws_kernel");
    if (rc != OCQ_OK) return rc;
  }
  return launch_pixel_counters<D, false>(frames, N, m, st, ntiles * NT);
}

template <int D, int NT, int FPS, int S>
static ocq_status launch_pixel_red(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  using C = RedBuildCfg<D, NT, FPS, S>;
  if (N > 255) return launch_pixel_counters<D, true>(frames, N, m, st, 0);
  const int64_t hw = (int64_t)m->H * m->W;
  constexpr bool fits = C::SMEM <= 227 * 1024;
  const int64_t ntiles = fits ? hw / NT : 0;
  if (ntiles > 0) {
    auto kern = build_pixel_red_kernel<D, NT, FPS, S>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return cuda_status(e, "build_pixel_red_kernel smem");
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, C::SMEM);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > ntiles) grid = ntiles;
    kern<<<(unsigned)grid, NT, C::SMEM, st>>>(frames, N, hw, ntiles, (uint32_t)m->T, m->bits);
    count_launch();
    ocq_status rc = cuda_status(cudaGetLastError(), "build_pixel_red_kernel");
    if (rc != OCQ_OK) return rc;
  }
  return launch_pixel_counters<D, false>(frames, N, m, st, ntiles * NT);
}

// ---- tunable variants ------------------------------------------------------------
using BuildFn = ocq_status (*)(const uint8_t *, int, ocq_model *, cudaStream_t);
struct BuildVariant {
  int nt, fps, stages, tensor;
  BuildFn fn[2][3];  // [4-bit, 8-bit counters][depth 1, 2, 3]
};
#define OCQ_BV(NT, F, S, TS)                                                                          \
  {                                                                                                  \
    NT, F, S, TS, {                                                                                  \
      {launch_pixel_staged<1, 4, NT, F, S, TS>, launch_pixel_staged<2, 4, NT, F, S, TS>,             \
       launch_pixel_staged<3, 4, NT, F, S, TS>},                                                     \
          {launch_pixel_staged<1, 8, NT, F, S, TS>, launch_pixel_staged<2, 8, NT, F, S, TS>,         \
           launch_pixel_staged<3, 8, NT, F, S, TS>}                                                  \
    }                                                                                                \
  }
#define OCQ_RV(NT, F, S)                                                                              \
  {                                                                                                  \
    NT, F, S, 2, {                                                                                   \
      {launch_pixel_red<1, NT, F, S>, launch_pixel_red<2, NT, F, S>, launch_pixel_red<3, NT, F, S>}, \
          {launch_pixel_red<1, NT, F, S>, launch_pixel_red<2, NT, F, S>, launch_pixel_red<3, NT, F, S>} \
    }                                                                                                \
  }
#define OCQ_DV(NT, PF)                                                                                 \
  {                                                                                                   \
    NT, PF, 0, 3, {                                                                                   \
      {launch_pixel_direct<1, 4, NT, PF>, launch_pixel_direct<2, 4, NT, PF>,                          \
       launch_pixel_direct<3, 4, NT, PF>},                                                            \
          {launch_pixel_direct<1, 8, NT, PF>, launch_pixel_direct<2, 8, NT, PF>,                      \
           launch_pixel_direct<3, 8, NT, PF>}                                                         \
    }                                                                                                 \
  }
// kind (4th field): 0 row copies, 1 2-D tensor copies, 2 byte counters bumped
// by shared reductions, 3 direct loads (frames per stage = prefetched frames)
#define OCQ_WV(NT, F, S, KIND, TS, KP)                                                                \
  {                                                                                                  \
    NT, F, S, KIND, {                                                                                \
      {launch_pixel_ws<1, NT, F, S, TS, KP>, launch_pixel_ws<2, NT, F, S, TS, KP>,                   \
       launch_pixel_ws<3, NT, F, S, TS, KP>},                                                        \
          {launch_pixel_ws<1, NT, F, S, TS, KP>, launch_pixel_ws<2, NT, F, S, TS, KP>,               \
           launch_pixel_ws<3, NT, F, S, TS, KP>}                                                     \
    }                                                                                                \
  }
// kind 4: copy warp + row copies; 5: copy warp + one tensor copy per stage;
// 6: as 4 with kept bits set as counts reach T; 7: as 5 with kept bits
// kind 8: frequent-leaf candidates per pixel (build_pixel_mg_kernel: no shared
// counters, frames read once with direct loads); beyond 255 frames it falls
// back to the first variant.
template <int D>
static ocq_status launch_pixel_candidates(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  if (N > 255) return launch_pixel_ws<D, 128, 8, 3, true, false>(frames, N, m, st);
  return launch_pixel_mg<D>(frames, N, m, st);
}
#define OCQ_MV                                                                                            \
  {                                                                                                       \
    128, 8, 0, 8, {                                                                                       \
      {launch_pixel_candidates<1>, launch_pixel_candidates<2>, launch_pixel_candidates<3>},               \
          {launch_pixel_candidates<1>, launch_pixel_candidates<2>, launch_pixel_candidates<3>}            \
    }                                                                                                     \
  }
static const BuildVariant kBuildVariants[] = {
    OCQ_WV(128, 8, 3, 5, true, false),  OCQ_WV(128, 8, 3, 4, false, false), OCQ_WV(128, 4, 5, 5, true, false),
    OCQ_WV(128, 8, 3, 7, true, true),   OCQ_RV(128, 8, 3),                   OCQ_BV(128, 16, 2, false),
    OCQ_MV};
#undef OCQ_MV
#undef OCQ_WV
#undef OCQ_DV
#undef OCQ_BV
#undef OCQ_RV
static int g_build_variant = 0;

int build_variant_count() { return (int)(sizeof kBuildVariants / sizeof kBuildVariants[0]); }
int build_variant_selected() { return g_build_variant; }
bool build_variant_select(int v) {
  if (v < 0 || v >= build_variant_count()) return false;
  g_build_variant = v;
  return true;
}
void build_variant_describe(int v, int *nt, int *fps, int *stages, int *tensor) {
  *nt = kBuildVariants[v].nt;
  *fps = kBuildVariants[v].fps;
  *stages = kBuildVariants[v].stages;
  *tensor = kBuildVariants[v].tensor;
}

// 4-bit counters saturating at T when T <= 15, else 8-bit (T <= 255).
static ocq_status launch_build_pixel_staged(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  return kBuildVariants[g_build_variant].fn[m->T <= 15 ? 0 : 1][m->depth - 1](frames, N, m, st);
}

bool build_take_timeout() {
  unsigned int flag = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&flag, g_build_timeout, sizeof flag) != cudaSuccess) return false;
  if (flag) cudaMemcpyToSymbol(g_build_timeout, &zero, sizeof zero);
  return flag != 0;
}

static int g_list_models = 1;
bool list_model_applies(int kind, int depth, int N, int T) {
  return g_list_models && kind == OCQ_REGION_PIXEL && (depth == 4 || depth == 5) && N <= 255 && T >= 1 && N / T <= 8;
}
int list_model_form() { return g_list_models; }
bool list_model_select(int v) {
  if (v < 0 || v > 1) return false;
  g_list_models = v;
  return true;
}

ocq_status launch_build_groups(const uint8_t *frames, int N, int group, ocq_model *m, cudaStream_t st) {
  if (group == 1) return launch_build(frames, N, m, st);
  m->kept_len = 0;  // until a candidate build writes the kept-leaf index
  if (m->kind == OCQ_REGION_PIXEL && N <= 255) {  // per pixel location: candidates over group-distinct leaves
    switch (m->depth) {
      case 1: return launch_pixel_mg<1>(frames, N, m, st, group);
      case 2: return launch_pixel_mg<2>(frames, N, m, st, group);
      case 3: return launch_pixel_mg<3>(frames, N, m, st, group);
      case 4: return launch_pixel_mg<4>(frames, N, m, st, group);
      case 5: return launch_pixel_mg<5>(frames, N, m, st, group);
      case 6: return launch_pixel_mg<6>(frames, N, m, st, group);
      case 7: return launch_pixel_mg<7>(frames, N, m, st, group);
      default: return launch_pixel_mg<8>(frames, N, m, st, group);
    }
  }
  return build_dense(frames, N, m, st, group);
}

ocq_status launch_build(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st) {
  const int d = m->depth;
  m->kept_len = 0;  // until a candidate build writes the kept-leaf index
  if (m->kind == OCQ_REGION_FRAME || (m->kind == OCQ_REGION_BLOCK && d >= 6)) return build_dense(frames, N, m, st);
  if (m->kind == OCQ_REGION_BLOCK && block_r8_ok(N, m->H, m->W, m->block, d, frames))
    return launch_block_r8(frames, N, m, st);
  if (m->kind == OCQ_REGION_BLOCK && block_fs_ok(N, m->H, m->W, m->block, d, frames)) {
    switch (d) {
      case 2: return launch_block_fs_b<2>(frames, N, m, st);
      case 3: return launch_block_fs_b<3>(frames, N, m, st);
      case 4: return launch_block_fs_b<4>(frames, N, m, st);
      default: return launch_block_fs_b<5>(frames, N, m, st);
    }
  }
  if (m->kind == OCQ_REGION_BLOCK && block_tile_ok(N, m->H, m->W, m->block, d, frames)) {
    switch (d) {
      case 2: return launch_block_tile_b<2>(frames, N, m, st);
      case 3: return launch_block_tile_b<3>(frames, N, m, st);
      case 4: return launch_block_tile_b<4>(frames, N, m, st);
      default: return launch_block_tile_b<5>(frames, N, m, st);
    }
  }
  if (m->kind == OCQ_REGION_BLOCK && block_warp_ok(N, m->H, m->W, m->block)) {
    switch (d) {
      case 1: return launch_block_warp<1>(frames, N, m, st);
      case 2: return launch_block_warp<2>(frames, N, m, st);
      case 3: return launch_block_warp<3>(frames, N, m, st);
      case 4: return launch_block_warp<4>(frames, N, m, st);
      default: return launch_block_warp<5>(frames, N, m, st);
    }
  }
  if (m->kind == OCQ_REGION_BLOCK) {
    switch (d) {
      case 1: return launch_block<1>(frames, N, m, st);
      case 2: return launch_block<2>(frames, N, m, st);
      case 3: return launch_block<3>(frames, N, m, st);
      case 4: return launch_block<4>(frames, N, m, st);
      default: return launch_block<5>(frames, N, m, st);
    }
  }
  const bool wide = N > 255;
  const bool staged_ok = m->T <= 255 && ((reinterpret_cast<uintptr_t>(frames) & 15) == 0) &&
                         ((int64_t)m->H * m->W) % 16 == 0;
  if (staged_ok && d <= 3) return launch_build_pixel_staged(frames, N, m, st);
  if (d >= 4 && N <= 255) {
    switch (d) {
      case 4: return launch_pixel_mg<4>(frames, N, m, st);
      case 5: return launch_pixel_mg<5>(frames, N, m, st);
      case 6: return launch_pixel_mg<6>(frames, N, m, st);
      case 7: return launch_pixel_mg<7>(frames, N, m, st);
      default: return launch_pixel_mg<8>(frames, N, m, st);
    }
  }
  switch (d) {
    case 1: return wide ? launch_pixel_counters<1, true>(frames, N, m, st) : launch_pixel_counters<1, false>(frames, N, m, st);
    case 2: return wide ? launch_pixel_counters<2, true>(frames, N, m, st) : launch_pixel_counters<2, false>(frames, N, m, st);
    case 3: return wide ? launch_pixel_counters<3, true>(frames, N, m, st) : launch_pixel_counters<3, false>(frames, N, m, st);
    case 4: return launch_pixel_chunked<4>(frames, N, m, st);
    case 5: return launch_pixel_chunked<5>(frames, N, m, st);
    case 6: return launch_pixel_chunked<6>(frames, N, m, st);
    case 7: return launch_pixel_chunked<7>(frames, N, m, st);
    default: return launch_pixel_chunked<8>(frames, N, m, st);
  }
}

// ---- whole-frame build that allocates nothing ------------------------------------
//
// ocq_build_model allocates the model and its scratch with cudaMallocAsync.
// Some callers cannot allocate device memory at call time: camera pipelines
// that reserve all memory at start-up and must never block on the allocator,
// or hosts that hand the library a fixed budget and forbid allocation on the
// processing path.  For them ocq_build_frame_noalloc builds a whole-frame
// model into a buffer the caller owns, using as scratch one statically sized
// device array of this file (kNoAllocScratchBytes on every GPU that loads the
// library, held until the process exits).  All calls on one device share that
// device's array, so calls on the same device whose work may overlap
// (different streams or host threads) must be ordered by the caller; calls on
// different devices use separate arrays.  Each call clears what it needs.

static constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocScratchBytes / 4];

static std::mutex g_noalloc_mu;
static uint32_t *g_noalloc_ptr[256];  // device address of the array, per device ordinal

// Device address of the scratch array on the current device.  The host-side
// symbol g_noalloc_scratch is not a device address, so it is resolved once per
// device (with that device current) and cached for the life of the process;
// a reset of the device's primary context (cudaDeviceReset) invalidates the
// cached address, so the entry point is not to be used after one.
static ocq_status noalloc_scratch(uint32_t **out) {
  int dev = 0;
  ocq_status rc = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc != OCQ_OK) return rc;
  if (dev < 0 || dev >= 256) {
    set_error("device ordinal %d out of range", dev);
    return OCQ_ENOTSUP;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    rc = cuda_status(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(no-alloc scratch)");
    if (rc != OCQ_OK) return rc;
    g_noalloc_ptr[dev] = static_cast<uint32_t *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return OCQ_OK;
}

}  // namespace ocq

using namespace ocq;

extern "C" ocq_status ocq_build_frame_noalloc(const uint8_t *frames, int N, int H, int W, int depth, int T,
                                              uint64_t *model, void *stream) {
  clear_error();
  if (!frames || !model || H < 1 || W < 1 || depth < 1 || depth > 8 || N < 1 || N > 65535 || T < 1 || T > N ||
      (int64_t)N * H * W >= ((int64_t)1 << 40)) {
    set_error("ocq_build_frame_noalloc: need frames, model != NULL, H, W >= 1, 1 <= depth <= 8, "
              "1 <= T <= N <= 65535 (N=%d, T=%d, depth=%d)", N, T, depth);
    return OCQ_EINVAL;
  }
  const int64_t wpr = wpr32(depth);
  const int P = bit_length((uint32_t)N);
  const int64_t cap = (int64_t)(kNoAllocScratchBytes / 4);
  // scratch rows: the merged row, P counter planes, at least one frame's leaf set
  if ((int64_t)(P + 2) * wpr > cap) {
    set_error("ocq_build_frame_noalloc: depth %d with N = %d needs %lld bytes of scratch; the maximum is %zu bytes",
              depth, N, (long long)((int64_t)(P + 2) * wpr * 4), kNoAllocScratchBytes);
    return OCQ_EINVAL;
  }
  uint32_t *scratch = nullptr;
  ocq_status rc = noalloc_scratch(&scratch);
  if (rc != OCQ_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t *row = scratch;                  // [wpr] merged row (internal order)
  uint32_t *planes = scratch + wpr;         // [P][wpr]
  uint32_t *occ = planes + (int64_t)P * wpr; // [nb][wpr]
  int64_t nb64 = cap / wpr - P - 1;
  const int nb = (int)(nb64 < N ? nb64 : N);
  const int64_t hw = (int64_t)H * W;
  for (int f0 = 0; f0 < N && rc == OCQ_OK; f0 += nb) {
    const int nf = N - f0 < nb ? N - f0 : nb;
    rc = cuda_status(cudaMemsetAsync(occ, 0, (size_t)nf * wpr * 4, st), "clear occupancy");
    if (rc != OCQ_OK) break;
    if (depth <= 6) {
      switch (depth) {
        case 1: launch_occ_frame<1>(frames, hw, f0, nf, occ, 1, st); break;
        case 2: launch_occ_frame<2>(frames, hw, f0, nf, occ, 1, st); break;
        case 3: launch_occ_frame<3>(frames, hw, f0, nf, occ, 1, st); break;
        case 4: launch_occ_frame<4>(frames, hw, f0, nf, occ, 1, st); break;
        case 5: launch_occ_frame<5>(frames, hw, f0, nf, occ, 1, st); break;
        default: launch_occ_frame<6>(frames, hw, f0, nf, occ, 1, st); break;
      }
    } else {
      occ_global_kernel<<<grid_cap(hw * nf, 256, 16), 256, 0, st>>>(frames, H, W, OCQ_REGION_FRAME, 0, depth, f0, nf, 1,
                                                                     wpr, occ, 1);
      count_launch();
    }
    rc = cuda_status(cudaGetLastError(), "occupancy kernel");
    if (rc != OCQ_OK) break;
    planes_merge_kernel<<<grid_cap(wpr, 256, 8), 256, 0, st>>>(occ, nf, wpr, planes, P, f0 == 0, f0 + nf >= N,
                                                                (uint32_t)T, row);
    count_launch();
    rc = cuda_status(cudaGetLastError(), "planes_merge_kernel");
  }
  if (rc == OCQ_OK) rc = launch_export(row, 1, depth, model, st);
  return rc;
}

