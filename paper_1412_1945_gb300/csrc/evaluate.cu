// Redraw (Sec. 2, Fig. 2) and evaluation against ground truth (Sec. 5).
//
//   redraw_kernel     each colour becomes the colour of its leaf in a tree
//                     pruned at depth d: the d most significant bits of each
//                     channel, zeros below.  One byte mask on every byte, in
//                     16-byte vectors: 6 bytes of HBM traffic per pixel.
//   confusion_kernel  per frame, true/false positives and negatives of a
//                     foreground mask against ground truth (non-zero byte =
//                     foreground in both); spans of 32 KB of each input per
//                     CTA item, 8 16-byte vectors of both in flight per thread,
//                     per-byte flags counted with popc, one 64-bit atomic per
//                     counter and item.  2 bytes of HBM traffic per pixel.
#include <cstdint>

#include "ocq_internal.cuh"

namespace ocq {

__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t w) {  // 0x01 in each non-zero byte
  w |= w >> 4;
  w |= w >> 2;
  w |= w >> 1;
  return w & 0x01010101u;
}

__global__ void redraw_kernel(const uint8_t *__restrict__ in, int64_t nbytes, uint32_t keep,
                              uint8_t *__restrict__ out, int vec) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t tail = 0;
  if (vec) {
    const int64_t nv = nbytes >> 4;
    for (int64_t i = t0; i < nv; i += stride) {
      uint4 v = ld_stream16(in + (i << 4));
      v.x &= keep, v.y &= keep, v.z &= keep, v.w &= keep;
      st_stream16(out + (i << 4), v);
    }
    tail = nv << 4;
  }
  for (int64_t i = tail + t0; i < nbytes; i += stride) out[i] = in[i] & (uint8_t)keep;
}

// Work item = (frame f, span j): 256 threads x VPT 16-byte vectors of frame f
// (or, without vectors, 256 x VPT x 16 bytes one at a time).  CTAs stride over
// items; each item's counts are reduced in the CTA and added to counts[f].
constexpr int kConfVpt = 8;

__global__ void __launch_bounds__(256, 2) confusion_kernel(const uint8_t *__restrict__ mask,
                                                        const uint8_t *__restrict__ gt, int F, int64_t npix,
                                                        unsigned long long *__restrict__ counts, int vec) {
  __shared__ unsigned long long part[3][8];
  constexpr int64_t kSpan = 256 * kConfVpt * 16;  // pixels per item
  const int64_t spans = (npix + kSpan - 1) / kSpan;
  const int64_t items = spans * F;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int f = (int)(it / spans);
    const int64_t p0 = (it - (int64_t)f * spans) * kSpan;
    const int64_t p1 = p0 + kSpan < npix ? p0 + kSpan : npix;
    const uint8_t *m = mask + (int64_t)f * npix;
    const uint8_t *g = gt + (int64_t)f * npix;
    uint32_t tp = 0, pm = 0, pg = 0;  // both, predicted foreground, actual foreground
    if (vec && p1 - p0 == kSpan) {
      uint4 a[kConfVpt], b[kConfVpt];
#pragma unroll
      for (int k = 0; k < kConfVpt; ++k) {
        const int64_t o = p0 + ((int64_t)k * 256 + threadIdx.x) * 16;
        a[k] = __ldcs(reinterpret_cast<const uint4 *>(m + o));
        b[k] = __ldcs(reinterpret_cast<const uint4 *>(g + o));
      }
#pragma unroll
      for (int k = 0; k < kConfVpt; ++k) {
        const uint32_t am[4] = {a[k].x, a[k].y, a[k].z, a[k].w}, bg[4] = {b[k].x, b[k].y, b[k].z, b[k].w};
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const uint32_t x = nonzero_bytes(am[w]), y = nonzero_bytes(bg[w]);
          tp += __popc(x & y), pm += __popc(x), pg += __popc(y);
        }
      }
    } else {
      for (int64_t i = p0 + threadIdx.x; i < p1; i += 256) {
        const uint32_t x = m[i] != 0, y = g[i] != 0;
        tp += x & y, pm += x, pg += y;
      }
    }
    unsigned long long v[3] = {tp, pm, pg};
#pragma unroll
    for (int k = 0; k < 3; ++k)
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xFFFFFFFFu, v[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
      for (int k = 0; k < 3; ++k) part[k][warp] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long s3[3] = {0, 0, 0};
      for (int w = 0; w < 8; ++w)
        for (int k = 0; k < 3; ++k) s3[k] += part[k][w];
      atomicAdd(&counts[4 * f + 0], s3[0]);          // Tp
      atomicAdd(&counts[4 * f + 1], s3[1] - s3[0]);  // Fp = predicted - Tp
      atomicAdd(&counts[4 * f + 3], s3[2] - s3[0]);  // Fn = actual - Tp
    }
    __syncthreads();
  }
}

// Tn = pixels - Tp - Fp - Fn, once every CTA has added its counts.
__global__ void confusion_finish_kernel(int F, int64_t npix, unsigned long long *counts) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F; f += gridDim.x * blockDim.x)
    counts[4 * f + 2] = (unsigned long long)npix - counts[4 * f] - counts[4 * f + 1] - counts[4 * f + 3];
}

}  // namespace ocq

using namespace ocq;

extern "C" {

ocq_status ocq_redraw(const uint8_t *rgb, int64_t npix, int depth, uint8_t *out, void *stream) {
  if (depth < 1 || depth > 8 || npix < 0 || (npix > 0 && (!rgb || !out))) {
    set_error("ocq_redraw: need 1 <= depth <= 8, npix >= 0 and device buffers");
    return OCQ_EINVAL;
  }
  if (npix == 0) return OCQ_OK;
  const int64_t nbytes = npix * 3;
  const uint32_t keep = ((0xFFu << (8 - depth)) & 0xFFu) * 0x01010101u;
  const int vec = ((reinterpret_cast<uintptr_t>(rgb) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  int64_t blocks = (nbytes / (vec ? 16 : 1) + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  redraw_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(rgb, nbytes, keep, out, vec);
  count_launch();
  return cuda_status(cudaGetLastError(), "redraw_kernel");
}

ocq_status ocq_confusion(const uint8_t *mask, const uint8_t *gt, int F, int64_t npix, uint64_t *counts,
                         void *stream) {
  if (F < 0 || npix < 0 || !counts || (F > 0 && npix > 0 && (!mask || !gt))) {
    set_error("ocq_confusion: need F >= 0, npix >= 0 and device buffers");
    return OCQ_EINVAL;
  }
  if (F == 0) return OCQ_OK;
  cudaStream_t st = (cudaStream_t)stream;
  ocq_status rc = cuda_status(cudaMemsetAsync(counts, 0, (size_t)F * 4 * sizeof(uint64_t), st), "clear counts");
  if (rc != OCQ_OK || npix == 0) return rc;
  const int vec = ((reinterpret_cast<uintptr_t>(mask) | reinterpret_cast<uintptr_t>(gt)) & 15) == 0 &&
                  npix % 16 == 0;
  const int64_t span = 256 * kConfVpt * 16;
  const int64_t items = (npix + span - 1) / span * F;
  const int64_t cap = (int64_t)sm_count() * 8;
  const unsigned grid = (unsigned)(items < cap ? items : cap);
  confusion_kernel<<<grid, 256, 0, st>>>(mask, gt, F, npix, reinterpret_cast<unsigned long long *>(counts), vec);
  count_launch();
  rc = cuda_status(cudaGetLastError(), "confusion_kernel");
  if (rc != OCQ_OK) return rc;
  confusion_finish_kernel<<<(unsigned)((F + 255) / 256), 256, 0, st>>>(F, npix,
                                                                      reinterpret_cast<unsigned long long *>(counts));
  count_launch();
  return cuda_status(cudaGetLastError(), "confusion_finish_kernel");
}

ocq_status ocq_f_scores(const uint64_t *counts, double *out) {
  if (!counts || !out) {
    set_error("ocq_f_scores: NULL argument");
    return OCQ_EINVAL;
  }
  const double tp = (double)counts[0], fp = (double)counts[1], tn = (double)counts[2], fn = (double)counts[3];
  const double p0 = tn + fn > 0 ? tn / (tn + fn) : 1.0;
  const double r0 = tn + fp > 0 ? tn / (tn + fp) : 1.0;
  out[0] = p0;
  out[1] = r0;
  out[2] = p0 + r0 > 0 ? 2.0 * p0 * r0 / (p0 + r0) : 0.0;
  out[3] = 2 * tp + fp + fn > 0 ? 2.0 * tp / (2.0 * tp + fp + fn) : 1.0;
  return OCQ_OK;
}

}  // extern "C"
