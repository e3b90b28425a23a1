// Serving window (the update of the octree that the Sec. 4 title names; the
// procedure is not given, so the window semantics of the served form are the
// reading taken here): a camera keeps, instead of its last N frames, the
// per-frame occupancy those frames' trees need (Alg. 1 per frame) and merges
// it again every K frames (Alg. 2) without re-reading any frame.
//
//   * whole-frame regions: a ring of N leaf bitsets (8^d bits, internal planar
//     order) and resident u16 counts, one per leaf, of the frames in the
//     window holding it.  Each frame: its bitset (occupancy kernel), then
//     counts += new - evicted and the slot is overwritten
//     (window_count_update_kernel).  A re-merge is a threshold pass over the
//     counts (window_threshold_kernel): count >= T keeps the leaf.
//   * pixel and block regions (depth <= 5): a ring of N planes of per-pixel
//     u16 leaf codes (the region's code list is its pixels' codes), written by
//     window_codes_kernel.  A re-merge counts, per region, the frames holding
//     each leaf straight from the codes: per pixel location with the
//     frequent-leaf candidate build, per block with the warp leaf tables.
#include "build_bodies.cuh"

namespace ocq {

// Leaf codes of npix consecutive pixels (RGB8) as u16, 16 pixels per step
// when the source is 16-byte aligned.
template <int D>
__global__ void __launch_bounds__(256) window_codes_kernel(const uint8_t *__restrict__ frames, int64_t npix,
                                                           uint16_t *__restrict__ codes) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  int64_t tail = 0;
  if ((reinterpret_cast<uintptr_t>(frames) & 15) == 0) {
    const int64_t ng = npix >> 4;
    for (int64_t g = tid; g < ng; g += nth) {
      uint32_t w[12];
      load_group_masked<D, true>(frames + g * 48, w);
      uint32_t c[8];
      static_for<0, 8>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        c[k] = planar_from_masked<D>(group_pixel<2 * k>(w)) | (planar_from_masked<D>(group_pixel<2 * k + 1>(w)) << 16);
      });
      uint16_t *dst = codes + g * 16;
      if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        reinterpret_cast<uint4 *>(dst)[0] = make_uint4(c[0], c[1], c[2], c[3]);
        reinterpret_cast<uint4 *>(dst)[1] = make_uint4(c[4], c[5], c[6], c[7]);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) dst[2 * k] = (uint16_t)c[k], dst[2 * k + 1] = (uint16_t)(c[k] >> 16);
      }
    }
    tail = ng << 4;
  }
  for (int64_t p = tail + tid; p < npix; p += nth) {
    const uint8_t *px = frames + p * 3;
    codes[p] = (uint16_t)planar_code_rt(px[0], px[1], px[2], D);
  }
}

// One frame enters a whole-frame window: slot (the evicted frame's bitset)
// becomes fresh (the new frame's), each leaf's count follows, and fresh is
// cleared for the next frame's occupancy.
__global__ void __launch_bounds__(256) window_count_update_kernel(uint32_t *__restrict__ slot,
                                                                  uint32_t *__restrict__ fresh,
                                                                  uint16_t *__restrict__ counts, int64_t nwords,
                                                                  int nleaves_in_word) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t old = slot[w], nw = fresh[w];
    uint32_t diff = old ^ nw;
    while (diff) {
      const int i = __ffs(diff) - 1;
      diff &= diff - 1;
      if (i < nleaves_in_word) counts[w * 32 + i] += ((nw >> i) & 1u) ? (uint16_t)1 : (uint16_t)0xFFFFu;
    }
    slot[w] = nw;
    fresh[w] = 0u;
  }
}

// counts[leaf] = number of the N ring bitsets holding the leaf.
__global__ void __launch_bounds__(256) window_counts_init_kernel(const uint32_t *__restrict__ ring, int N,
                                                                 int64_t nwords, int64_t nleaves,
                                                                 uint16_t *__restrict__ counts) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nleaves; q += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c = 0;
    for (int s = 0; s < N; ++s) c += (ring[(int64_t)s * nwords + (q >> 5)] >> (q & 31)) & 1u;
    counts[q] = (uint16_t)c;
  }
}

// Merged row of a whole-frame window: bit q = counts[q] >= T (Alg. 2 keeps a
// leaf held by at least T of the window's trees).
__global__ void __launch_bounds__(256) window_threshold_kernel(const uint16_t *__restrict__ counts, int64_t nwords,
                                                               int nleaves_in_word, uint32_t T,
                                                               uint32_t *__restrict__ bits) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t v = 0;
    for (int i = 0; i < nleaves_in_word; ++i) v |= (uint32_t)(counts[w * 32 + i] >= T) << i;
    bits[w] = v;
  }
}

// Pixel regions: the candidate build over the window's codes.
template <int D, int KM>
__global__ void __launch_bounds__(128) remerge_pixel_codes_kernel(const uint16_t *__restrict__ ring, int N,
                                                                  int64_t hw, uint32_t T,
                                                                  uint32_t *__restrict__ model,
                                                                  uint16_t *__restrict__ kept) {
  extern __shared__ __align__(16) uint8_t rm_smem[];
  leaf_t<D> *codes = reinterpret_cast<leaf_t<D> *>(rm_smem) + (size_t)(threadIdx.x >> 5) * N * 32;
  const int64_t tile = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  if (tile * 32 >= hw) return;
  build_pixel_mg_body<D, KM, false, true>(reinterpret_cast<const uint8_t *>(ring), N, hw, T, model, tile, codes, 1,
                                          kept);
}

// Block regions (b <= 16): one warp per region counts its leaves over the
// window's code planes in a shared table (the table and the chunked fallback
// of the one-warp-per-region build).
template <int D, int PPL>
__device__ __forceinline__ void remerge_block_codes_body(const uint16_t *__restrict__ ring, int N, int H, int W,
                                                         int b, int bw, uint32_t T, uint32_t *__restrict__ model,
                                                         int64_t r_first, int64_t r_end, int64_t r_step,
                                                         uint32_t *tab) {
  using C = WarpTableCfg<D>;
  constexpr int PF = PPL >= 8 ? 2 : 16 / PPL;
  const int lane = threadIdx.x & 31;
  const int64_t hw = (int64_t)H * W;
  for (int64_t r = r_first; r < r_end; r += r_step) {
    const int y0 = (int)(r / bw) * b, x0 = (int)(r % bw) * b;
    const int h = min(b, H - y0), w = min(b, W - x0);
    const int npx = h * w;
    uint32_t off[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      const int i = lane + 32 * k;
      off[k] = i < npx ? (uint32_t)((int64_t)(y0 + i / w) * W + x0 + i % w) : 0u;
    }
    uint32_t *row = model + r * C::WPR;
    warp_zero_row<D>(row);
    if (warp_region_pass<D, PPL, PF, false, uint16_t>(ring, N, hw, off, npx, tab, -1)) {
      warp_emit<D>(tab, row, T);
    } else {
      for (int s = lane; s < C::S; s += 32) tab[s] = 0u;
      for (int c = 0; c < C::NC / C::S; ++c) {
        __syncwarp();
        warp_region_pass<D, PPL, PF, true, uint16_t>(ring, N, hw, off, npx, tab, c);
        warp_emit<D>(tab, row, T);
      }
    }
  }
}

template <int D, int PPL>
__global__ void __launch_bounds__(256) remerge_block_codes_kernel(const uint16_t *__restrict__ ring, int N, int H,
                                                                  int W, int b, int bw, uint32_t T,
                                                                  uint32_t *__restrict__ model, int64_t R) {
  extern __shared__ uint32_t rb_tabs[];
  constexpr int S = WarpTableCfg<D>::S;
  uint32_t *tab = rb_tabs + (threadIdx.x >> 5) * S;
  for (int i = threadIdx.x & 31; i < S; i += 32) tab[i] = 0u;
  __syncwarp();
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  remerge_block_codes_body<D, PPL>(ring, N, H, W, b, bw, T, model,
                                   (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), R, nw, tab);
}

// 8 x 8 blocks at depth 5: one region per warp with two-level tables over the
// window's code planes (build_block_r8_body reading codes).
__global__ void __launch_bounds__(256, 4) remerge_block_r8_kernel(const uint16_t *__restrict__ ring, int N, int H,
                                                                int W, int bw, uint32_t T,
                                                                uint32_t *__restrict__ model, int64_t R) {
  extern __shared__ __align__(16) uint8_t rr_smem[];
  constexpr int WB = BlockR8Cfg::WARP_SMEM;
  uint8_t *wsm = rr_smem + (threadIdx.x >> 5) * WB;
  for (int i = threadIdx.x & 31; i < WB / 4; i += 32) reinterpret_cast<uint32_t *>(wsm)[i] = 0u;
  __syncwarp();
  build_block_r8_body<5, uint16_t>(ring, N, H, W, bw, T, model, (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5), R,
                                   (int64_t)gridDim.x * 8, wsm);
}

static unsigned window_grid(int64_t work, int threads, int per_sm) {
  int64_t b = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

ocq_status launch_window_codes(const uint8_t *frames, int64_t npix, int depth, uint16_t *codes, cudaStream_t st) {
  if (npix <= 0) return OCQ_OK;
  const unsigned grid = window_grid((npix + 15) / 16, 256, 8);
  switch (depth) {
    case 1: window_codes_kernel<1><<<grid, 256, 0, st>>>(frames, npix, codes); break;
    case 2: window_codes_kernel<2><<<grid, 256, 0, st>>>(frames, npix, codes); break;
    case 3: window_codes_kernel<3><<<grid, 256, 0, st>>>(frames, npix, codes); break;
    case 4: window_codes_kernel<4><<<grid, 256, 0, st>>>(frames, npix, codes); break;
    case 5: window_codes_kernel<5><<<grid, 256, 0, st>>>(frames, npix, codes); break;
    default:
      set_error("internal: code windows hold depth <= 5");
      return OCQ_EINVAL;
  }
  count_launch();
  return cuda_status(cudaGetLastError(), "window_codes_kernel");
}

static int leaves_in_word(int depth) { return depth == 1 ? 8 : 32; }

ocq_status launch_window_count_update(uint32_t *slot, uint32_t *fresh, uint16_t *counts, int depth,
                                      cudaStream_t st) {
  const int64_t nw = wpr32(depth);
  window_count_update_kernel<<<window_grid(nw, 256, 4), 256, 0, st>>>(slot, fresh, counts, nw, leaves_in_word(depth));
  count_launch();
  return cuda_status(cudaGetLastError(), "window_count_update_kernel");
}

ocq_status launch_window_counts_init(const uint32_t *ring, int N, int depth, uint16_t *counts, cudaStream_t st) {
  const int64_t nw = wpr32(depth), nl = (int64_t)1 << (3 * depth);
  window_counts_init_kernel<<<window_grid(nl, 256, 8), 256, 0, st>>>(ring, N, nw, nl, counts);
  count_launch();
  return cuda_status(cudaGetLastError(), "window_counts_init_kernel");
}

ocq_status launch_window_threshold(const uint16_t *counts, int depth, uint32_t T, uint32_t *bits, cudaStream_t st) {
  const int64_t nw = wpr32(depth);
  window_threshold_kernel<<<window_grid(nw, 256, 4), 256, 0, st>>>(counts, nw, leaves_in_word(depth), T, bits);
  count_launch();
  return cuda_status(cudaGetLastError(), "window_threshold_kernel");
}

template <int D, int KM>
static ocq_status launch_remerge_pixel_km(const uint16_t *ring, int N, ocq_model *m, cudaStream_t st) {
  const size_t smem = (size_t)4 * N * 32 * sizeof(leaf_t<D>);
  auto kern = remerge_pixel_codes_kernel<D, KM>;
  if (smem > 48 * 1024) {
    ocq_status rc = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                                "remerge_pixel_codes_kernel smem");
    if (rc != OCQ_OK) return rc;
  }
  const int64_t hw = (int64_t)m->H * m->W;
  uint16_t *kept = (KM > 0 && m->kept_len > 0) ? m->kept : nullptr;
  kern<<<(unsigned)((hw + 127) / 128), 128, smem, st>>>(ring, N, hw, (uint32_t)m->T, m->bits, kept);
  count_launch();
  return cuda_status(cudaGetLastError(), "remerge_pixel_codes_kernel");
}

template <int D>
static ocq_status launch_remerge_pixel(const uint16_t *ring, int N, ocq_model *m, cudaStream_t st) {
  const int k = N / m->T;
  if (k <= 1) return launch_remerge_pixel_km<D, 1>(ring, N, m, st);
  if (k <= 2) return launch_remerge_pixel_km<D, 2>(ring, N, m, st);
  if (k <= 4) return launch_remerge_pixel_km<D, 4>(ring, N, m, st);
  if (k <= 8) return launch_remerge_pixel_km<D, 8>(ring, N, m, st);
  return launch_remerge_pixel_km<D, 0>(ring, N, m, st);
}

template <int D, int PPL>
static ocq_status launch_remerge_block_ppl(const uint16_t *ring, int N, ocq_model *m, cudaStream_t st) {
  constexpr size_t smem = (size_t)8 * WarpTableCfg<D>::S * 4;
  const int bw = (m->W + m->block - 1) / m->block;
  const int64_t ctas = (m->R + 7) / 8;
  const unsigned grid = (unsigned)(ctas < (int64_t)sm_count() * 8 ? ctas : (int64_t)sm_count() * 8);
  remerge_block_codes_kernel<D, PPL><<<grid, 256, smem, st>>>(ring, N, m->H, m->W, m->block, bw, (uint32_t)m->T,
                                                              m->bits, m->R);
  count_launch();
  return cuda_status(cudaGetLastError(), "remerge_block_codes_kernel");
}

template <int D>
static ocq_status launch_remerge_block(const uint16_t *ring, int N, ocq_model *m, cudaStream_t st) {
  if (D == 5 && m->block == 8 && m->W % 8 == 0 && (reinterpret_cast<uintptr_t>(ring) & 3) == 0) {
    constexpr size_t smem = (size_t)8 * BlockR8Cfg::WARP_SMEM;
    static int cap = 0;
    if (!cap) {
      cudaFuncSetAttribute(remerge_block_r8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      int per = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, remerge_block_r8_kernel, 256, smem);
      cap = sm_count() * (per > 0 ? per : 1);
    }
    const int bw = m->W / 8;
    const int64_t ctas = (m->R + 7) / 8;
    remerge_block_r8_kernel<<<(unsigned)(ctas < cap ? ctas : cap), 256, smem, st>>>(ring, N, m->H, m->W, bw,
                                                                                   (uint32_t)m->T, m->bits, m->R);
    count_launch();
    return cuda_status(cudaGetLastError(), "remerge_block_r8_kernel");
  }
  const int npx = m->block * m->block;
  if (npx <= 32) return launch_remerge_block_ppl<D, 1>(ring, N, m, st);
  if (npx <= 64) return launch_remerge_block_ppl<D, 2>(ring, N, m, st);
  if (npx <= 128) return launch_remerge_block_ppl<D, 4>(ring, N, m, st);
  return launch_remerge_block_ppl<D, 8>(ring, N, m, st);
}

bool window_codes_apply(int kind, int block, int depth, int N, int H, int W) {
  if (depth > 5 || N > 255 || (int64_t)H * W > (int64_t)UINT32_MAX) return false;
  if (kind == OCQ_REGION_PIXEL) return true;
  return kind == OCQ_REGION_BLOCK && block <= 16;
}

ocq_status launch_remerge_codes(const uint16_t *ring, int N, ocq_model *m, cudaStream_t st) {
  if (!window_codes_apply(m->kind, m->block, m->depth, N, m->H, m->W)) {
    set_error("internal: no code window for this camera");
    return OCQ_EINVAL;
  }
  if (m->kind == OCQ_REGION_PIXEL) {
    switch (m->depth) {
      case 1: return launch_remerge_pixel<1>(ring, N, m, st);
      case 2: return launch_remerge_pixel<2>(ring, N, m, st);
      case 3: return launch_remerge_pixel<3>(ring, N, m, st);
      case 4: return launch_remerge_pixel<4>(ring, N, m, st);
      default: return launch_remerge_pixel<5>(ring, N, m, st);
    }
  }
  switch (m->depth) {
    case 1: return launch_remerge_block<1>(ring, N, m, st);
    case 2: return launch_remerge_block<2>(ring, N, m, st);
    case 3: return launch_remerge_block<3>(ring, N, m, st);
    case 4: return launch_remerge_block<4>(ring, N, m, st);
    default: return launch_remerge_block<5>(ring, N, m, st);
  }
}

}  // namespace ocq
