/* Host generator: fills frames [frame0, frame0+nframes) of a scene on the CPU.
 * Input generation only; see synth_pixel.h. */
#include <stddef.h>
#include "synth_pixel.h"

int ocq_synth_fill_host(const int32_t *scene, int64_t frame0, int64_t nframes,
                        uint8_t *rgb, uint8_t *gt) {
  if (!scene || !rgb || scene[SY_MAGIC] != SY_MAGIC_VALUE || nframes < 0) return 1;
  const int H = scene[SY_H], W = scene[SY_W];
  const uint64_t seed = synth_seed(scene);
  const int64_t rows = nframes * (int64_t)H;
#pragma omp parallel for schedule(static)
  for (int64_t fr = 0; fr < rows; ++fr) {
    const int64_t fl = fr / H;
    const int y = (int)(fr % H);
    uint8_t *o = rgb + (size_t)fr * (size_t)W * 3u;
    uint8_t *m = gt ? gt + (size_t)fr * (size_t)W : NULL;
    for (int x = 0; x < W; ++x) {
      uint8_t g;
      synth_pixel(scene, seed, frame0 + fl, y, x, o + 3 * x, &g);
      if (m) m[x] = g;
    }
  }
  return 0;
}

/* Fills rgb[f][k][3] for frames [frame0, frame0+nframes) at the k pixel
 * locations idx[0..k) (row-major indices y*W + x). */
int ocq_synth_fill_pixels_host(const int32_t *scene, int64_t frame0, int64_t nframes, const int64_t *idx,
                               int64_t k, uint8_t *rgb) {
  if (!scene || !idx || !rgb || scene[SY_MAGIC] != SY_MAGIC_VALUE || nframes < 0 || k < 0) return 1;
  const int W = scene[SY_W];
  const uint64_t seed = synth_seed(scene);
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < nframes; ++f)
    for (int64_t j = 0; j < k; ++j) {
      uint8_t g;
      synth_pixel(scene, seed, frame0 + f, (int)(idx[j] / W), (int)(idx[j] % W), rgb + (f * k + j) * 3, &g);
    }
  return 0;
}
