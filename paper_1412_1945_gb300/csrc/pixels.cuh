// Pixel-stream helpers: walk a contiguous pixel range of one frame and hand
// each pixel's planar leaf code to a callback, with 16-byte vector loads of
// 16-pixel (48-byte) groups when the range is 16-byte aligned.
#pragma once

#include <type_traits>

#include "ocq_internal.cuh"

namespace ocq {

template <int K, int N, typename Fn>
__device__ __forceinline__ void static_for(Fn &&fn) {
  if constexpr (K < N) {
    fn(std::integral_constant<int, K>{});
    static_for<K + 1, N>(fn);
  }
}

// Loads 48 bytes (16 pixels) and pre-masks every byte to its top D bits,
// moved to the bottom (r_d, g_d, b_d bytes).
template <int D, bool STREAM>
__device__ __forceinline__ void load_group_masked(const uint8_t *src, uint32_t (&w)[12]) {
  const uint4 *s = reinterpret_cast<const uint4 *>(src);
  uint4 a, b, c;
  if constexpr (STREAM) {
    a = ld_stream16(s), b = ld_stream16(s + 1), c = ld_stream16(s + 2);
  } else {
    a = __ldg(s), b = __ldg(s + 1), c = __ldg(s + 2);
  }
  w[0] = a.x, w[1] = a.y, w[2] = a.z, w[3] = a.w;
  w[4] = b.x, w[5] = b.y, w[6] = b.z, w[7] = b.w;
  w[8] = c.x, w[9] = c.y, w[10] = c.z, w[11] = c.w;
#pragma unroll
  for (int i = 0; i < 12; ++i) w[i] = (w[i] >> (8 - D)) & byte_mask(D);
}

// Calls fn(q, p) for every pixel p in [p0, p1) of frame `fr`, the CTA's
// threads striding over 16-pixel groups, then over the ragged tail.
template <int D, typename Fn>
__device__ __forceinline__ void cta_for_codes(const uint8_t *__restrict__ fr, int64_t p0, int64_t p1, Fn &&fn) {
  int64_t tail = p0;
  if ((reinterpret_cast<uintptr_t>(fr + p0 * 3) & 15) == 0) {
    const int64_t ng = (p1 - p0) >> 4;
    for (int64_t g = threadIdx.x; g < ng; g += blockDim.x) {
      uint32_t w[12];
      const int64_t pb = p0 + (g << 4);
      load_group_masked<D, false>(fr + pb * 3, w);
      static_for<0, 16>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        fn(planar_from_masked<D>(group_pixel<k>(w)), pb + k);
      });
    }
    tail = p0 + (ng << 4);
  }
  for (int64_t p = tail + threadIdx.x; p < p1; p += blockDim.x) {
    const uint8_t *px = fr + p * 3;
    fn(planar_code_rt(__ldg(px), __ldg(px + 1), __ldg(px + 2), D), p);
  }
}

}  // namespace ocq
