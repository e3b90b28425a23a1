// End-to-end detection from host memory: copies training frames in, builds
// the model, then streams test frames through a ring of device chunk buffers
// (copy in / classify / copy masks out overlap on three streams), and copies
// the masks back.  All compute runs in the library's kernels.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "ocq_internal.cuh"

namespace ocq {

struct Chunks {
  uint8_t *in[3] = {nullptr, nullptr, nullptr};
  uint8_t *out[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_in[3] = {}, ev_cls[3] = {}, ev_out[3] = {};
};

}  // namespace ocq

using namespace ocq;

// Staging buffers (training frames, chunk ring) come from a pool of this
// pipeline that keeps freed memory mapped, so repeated calls do not map and
// unmap a gigabyte each time; one pool per device, created on first use.
static cudaMemPool_t pipeline_pool(int dev) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

extern "C" ocq_status ocq_detect_host(const uint8_t *train, int N, const uint8_t *test, int F, int H, int W,
                                      ocq_region region, int depth, int T, uint8_t *mask, void *stream,
                                      ocq_model **out_model) {
  if (out_model) *out_model = nullptr;
  if (!train || F < 0 || (F > 0 && (!test || !mask)) || H < 1 || W < 1) {
    set_error("ocq_detect_host: bad arguments");
    return OCQ_EINVAL;
  }
  cudaStream_t s0 = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  PoolScope scope(pipeline_pool(dev));
  const size_t hw = (size_t)H * (size_t)W;
  uint8_t *train_d = nullptr;
  ocq_status rc = cuda_status(malloc_async((void **)&train_d, (size_t)N * hw * 3, s0), "training frames");
  if (rc != OCQ_OK) return rc;
  rc = cuda_status(cudaMemcpyAsync(train_d, train, (size_t)N * hw * 3, cudaMemcpyHostToDevice, s0), "copy in");
  ocq_model *m = nullptr;
  if (rc == OCQ_OK) rc = ocq_build_model(train_d, N, H, W, region, depth, T, s0, &m);
  cudaFreeAsync(train_d, s0);
  if (rc != OCQ_OK) return rc;

  // ~192 MiB of input per chunk, at least one frame
  const int per = std::max<int>(1, (int)std::min<size_t>((size_t)F, ((size_t)192 << 20) / (hw * 3)));
  const int nchunks = F > 0 ? (F + per - 1) / per : 0;
  Chunks c;
  cudaStream_t s_in = nullptr, s_out = nullptr;
  rc = cuda_status(cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking), "stream");
  if (rc == OCQ_OK) rc = cuda_status(cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking), "stream");
  const int nb = std::min(3, std::max(1, nchunks));
  for (int b = 0; b < nb && rc == OCQ_OK; ++b) {
    rc = cuda_status(malloc_async((void **)&c.in[b], (size_t)per * hw * 3, s0), "chunk buffer");
    if (rc == OCQ_OK) rc = cuda_status(malloc_async((void **)&c.out[b], (size_t)per * hw, s0), "chunk buffer");
    if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&c.ev_in[b], cudaEventDisableTiming), "event");
    if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&c.ev_cls[b], cudaEventDisableTiming), "event");
    if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&c.ev_out[b], cudaEventDisableTiming), "event");
  }
  cudaEvent_t ready = nullptr;
  if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming), "event");
  if (rc == OCQ_OK) {
    // buffers and model are ready on s0; the copy streams start after that
    cudaEventRecord(ready, s0);
    cudaStreamWaitEvent(s_in, ready, 0);
    cudaStreamWaitEvent(s_out, ready, 0);
  }
  for (int k = 0; k < nchunks && rc == OCQ_OK; ++k) {
    const int b = k % nb;
    const int f0 = k * per, nf = std::min(per, F - f0);
    if (k >= nb) cudaStreamWaitEvent(s_in, c.ev_cls[b], 0);  // input buffer consumed
    rc = cuda_status(cudaMemcpyAsync(c.in[b], test + (size_t)f0 * hw * 3, (size_t)nf * hw * 3,
                                     cudaMemcpyHostToDevice, s_in),
                     "copy in");
    if (rc != OCQ_OK) break;
    cudaEventRecord(c.ev_in[b], s_in);
    cudaStreamWaitEvent(s0, c.ev_in[b], 0);
    if (k >= nb) cudaStreamWaitEvent(s0, c.ev_out[b], 0);  // output buffer drained
    rc = ocq_classify(m, c.in[b], nf, c.out[b], s0);
    if (rc != OCQ_OK) break;
    cudaEventRecord(c.ev_cls[b], s0);
    cudaStreamWaitEvent(s_out, c.ev_cls[b], 0);
    rc = cuda_status(cudaMemcpyAsync(mask + (size_t)f0 * hw, c.out[b], (size_t)nf * hw, cudaMemcpyDeviceToHost, s_out),
                     "copy out");
    if (rc != OCQ_OK) break;
    cudaEventRecord(c.ev_out[b], s_out);
  }
  // everything lands before the call returns
  cudaError_t e1 = s_in ? cudaStreamSynchronize(s_in) : cudaSuccess;
  cudaError_t e2 = s_out ? cudaStreamSynchronize(s_out) : cudaSuccess;
  cudaError_t e3 = cudaStreamSynchronize(s0);
  if (rc == OCQ_OK) rc = cuda_status(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "pipeline");
  for (int b = 0; b < 3; ++b) {
    if (c.in[b]) cudaFreeAsync(c.in[b], s0);
    if (c.out[b]) cudaFreeAsync(c.out[b], s0);
    if (c.ev_in[b]) cudaEventDestroy(c.ev_in[b]);
    if (c.ev_cls[b]) cudaEventDestroy(c.ev_cls[b]);
    if (c.ev_out[b]) cudaEventDestroy(c.ev_out[b]);
  }
  if (ready) cudaEventDestroy(ready);
  if (s_in) cudaStreamDestroy(s_in);
  if (s_out) cudaStreamDestroy(s_out);
  if (rc == OCQ_OK && out_model)
    *out_model = m;
  else
    ocq_model_free(m);
  return rc;
}
