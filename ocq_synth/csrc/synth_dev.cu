/* Device generator: fills frames [frame0, frame0+nframes) of a scene on the GPU,
 * byte-identical to the host generator (same synth_pixel.h source).
 * Input generation only; none of the method's arithmetic lives here. */
#include <cuda_runtime.h>
#include "synth_pixel.h"

__global__ void synth_fill_kernel(const int32_t *__restrict__ scene, int64_t frame0,
                                  int64_t npix, int H, int W, uint8_t *__restrict__ rgb,
                                  uint8_t *__restrict__ gt) {
  const uint64_t seed = synth_seed(scene);
  const int64_t hw = (int64_t)H * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = i / hw;
    const int64_t p = i - f * hw;
    uint8_t c[3], g;
    synth_pixel(scene, seed, frame0 + f, (int)(p / W), (int)(p % W), c, &g);
    rgb[3 * i + 0] = c[0];
    rgb[3 * i + 1] = c[1];
    rgb[3 * i + 2] = c[2];
    if (gt) gt[i] = g;
  }
}

/* scene_dev: device copy of the scene blob; H, W: its frame size (also in the
 * blob, passed here so the host needs no device read).  Returns a cudaError_t. */
extern "C" int ocq_synth_fill_device(const int32_t *scene_dev, int H, int W, int64_t frame0,
                                     int64_t nframes, uint8_t *rgb_dev, uint8_t *gt_dev,
                                     void *stream) {
  const int64_t npix = nframes * (int64_t)H * W;
  if (npix <= 0) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (npix + 255) / 256;
  if (blocks > (int64_t)sms * 32) blocks = (int64_t)sms * 32;
  synth_fill_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(scene_dev, frame0, npix, H, W,
                                                                       rgb_dev, gt_dev);
  return (int)cudaGetLastError();
}
