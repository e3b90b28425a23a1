// Served form: camera streams join and leave while frames arrive; each
// camera's model and its sliding window of the last N frames stay resident
// in HBM.  The title of the paper's Sec. 4 mentions updating the octree but
// gives no procedure; the window semantics here are:
//   * the N training frames build M_0 (Sec. 3, Alg. 1-2);
//   * test frame t (t = 0, 1, ...) is classified against M_floor(t/K) (Alg. 3);
//   * after classification frame t enters a ring of the last N frames;
//   * when (t+1) % K == 0 the ring is merged again: M_(t+1)/K = merge(ring).
// So M_k is the merged model of global frames [kK, kK+N-1] (training frames
// first).  A camera's per-frame work (classify, ring copy) is ordered on its
// own high-priority CUDA stream and its builds on a low-priority one, joined
// by events: a re-merge starts once the window's last frame is in the ring,
// and the camera's next frame waits for it.  Cameras run concurrently, so work
// of frames that arrive while others are on the GPU overlaps on the device,
// and one camera's long re-merge yields the SMs to other cameras' frames.
// The window keeps what the merge needs of those frames, not the frames
// (window.cu): whole-frame cameras a ring of N leaf bitsets plus resident
// per-leaf counts, updated as each frame enters (re-merge = a threshold pass);
// pixel and block cameras of depth <= 5 a ring of per-pixel u16 leaf codes
// (re-merge = counting the codes, no frame is read again).  Both re-merge the
// model in place on the camera stream, after the frames that read the old one.
// Cameras outside those forms (deeper, N > 255, blocks wider than 16, or a
// whole-frame bitset larger than a frame) keep the N frames and rebuild with
// ocq_build_model on a low-priority stream.
// Admission reserves a camera's footprint (window, model, build scratch; the
// frame ring also a second model) against an HBM budget and returns OCQ_EBUSY
// when it does not fit; released cameras return their share.  A frame's
// completion time is taken by a host function enqueued right after its mask.
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <vector>

#include "ocq_internal.cuh"

namespace ocq {

static double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Camera;

struct Pending {
  struct ocq_server *srv;
  int camera;
  int64_t frame;
  uint64_t tag;
  double arrival;
};

enum WindowForm { WIN_FRAMES = 0, WIN_BITS = 1, WIN_CODES = 2 };

static int window_form(const ocq_camera_desc &d) {
  if (d.region.kind == OCQ_REGION_FRAME)
    return (size_t)wpr32(d.depth) * 4 <= (size_t)d.H * d.W * 3 ? WIN_BITS : WIN_FRAMES;
  return window_codes_apply(d.region.kind, d.region.block, d.depth, d.N, d.H, d.W) ? WIN_CODES : WIN_FRAMES;
}

// Bytes of one window slot (one frame's entry) of each form.
static size_t window_slot_bytes(const ocq_camera_desc &d, int form) {
  const size_t hw = (size_t)d.H * d.W;
  return form == WIN_BITS ? (size_t)wpr32(d.depth) * 4 : form == WIN_CODES ? hw * 2 : hw * 3;
}

struct Camera {
  int id = -1;
  ocq_camera_desc d;
  size_t footprint = 0;
  int win = WIN_FRAMES;
  // slot = frame % N: WIN_FRAMES N frames (HWC RGB8); WIN_BITS N leaf bitsets
  // (wpr32(depth) u32 words, internal order); WIN_CODES N planes of H*W u16
  // leaf codes
  uint8_t *ring = nullptr;
  uint32_t *fresh = nullptr;   // WIN_BITS: the entering frame's bitset
  uint16_t *counts = nullptr;  // WIN_BITS: per leaf, window frames holding it
  ocq_model *model = nullptr;
  cudaStream_t stream = nullptr;  // high priority: classify, ring copies, completions
  cudaStream_t merge = nullptr;   // low priority: builds (M_0 and re-merges)
  cudaEvent_t ring_ready = nullptr, merged = nullptr;
  int64_t submitted = 0;          // test frames submitted so far
  bool live = false;
};

}  // namespace ocq

using namespace ocq;

struct ocq_server {
  size_t budget = 0, used = 0;
  cudaMemPool_t pool = nullptr;  // the cameras' rings, models and scratch
  int max_cameras = 0;
  std::mutex mu;
  std::vector<Camera> cams;
  std::deque<ocq_completion> done;
  int64_t completed = 0;
};

static size_t camera_footprint(const ocq_camera_desc &d) {
  const size_t hw = (size_t)d.H * d.W;
  const size_t model = model_bytes(d.H, d.W, d.region, d.depth, d.N, d.T);
  const int form = window_form(d);
  const size_t ring = (size_t)d.N * window_slot_bytes(d, form);
  size_t scratch = 0;  // what a build of the model allocates beside it
  if (d.region.kind == OCQ_REGION_FRAME) scratch = (size_t)d.N * wpr32(d.depth) * 4;
  if (d.region.kind == OCQ_REGION_PIXEL && d.depth >= 6) scratch = hw * ((size_t)1 << (3 * d.depth - 9)) / 8;
  if (form == WIN_BITS)  // the entering frame's bitset and the u16 counts; re-merged in place
    return model + ring + (size_t)wpr32(d.depth) * 4 + ((size_t)1 << (3 * d.depth)) * 2 + scratch;
  if (form == WIN_CODES) return model + ring + scratch;
  return 2 * model + ring + scratch;  // the model being rebuilt lives beside the current one
}

// Allocates the camera's window on its build stream and fills it from the N
// frames `src` (frame i = global frame i into slot i).
static ocq_status window_fill(Camera &c, const uint8_t *src) {
  const ocq_camera_desc &d = c.d;
  const size_t slot = window_slot_bytes(d, c.win);
  ocq_status rc = cuda_status(malloc_async((void **)&c.ring, (size_t)d.N * slot, c.merge), "camera window");
  if (rc != OCQ_OK) return rc;
  if (c.win == WIN_FRAMES)
    return cuda_status(cudaMemcpyAsync(c.ring, src, (size_t)d.N * slot, cudaMemcpyDeviceToDevice, c.merge),
                       "ring fill");
  if (c.win == WIN_CODES)
    return launch_window_codes(src, (int64_t)d.N * d.H * d.W, d.depth, reinterpret_cast<uint16_t *>(c.ring), c.merge);
  rc = cuda_status(malloc_async((void **)&c.fresh, slot, c.merge), "window bitset");
  if (rc == OCQ_OK)
    rc = cuda_status(malloc_async((void **)&c.counts, ((size_t)1 << (3 * d.depth)) * 2, c.merge), "window counts");
  if (rc == OCQ_OK) rc = cuda_status(cudaMemsetAsync(c.ring, 0, (size_t)d.N * slot, c.merge), "clear window");
  if (rc == OCQ_OK) rc = cuda_status(cudaMemsetAsync(c.fresh, 0, slot, c.merge), "clear window");
  if (rc == OCQ_OK)
    rc = launch_frame_occupancy(src, d.N, d.H, d.W, d.depth, reinterpret_cast<uint32_t *>(c.ring), c.merge);
  if (rc == OCQ_OK)
    rc = launch_window_counts_init(reinterpret_cast<uint32_t *>(c.ring), d.N, d.depth, c.counts, c.merge);
  return rc;
}

static void window_free(Camera &c, cudaStream_t st) {
  if (c.ring) cudaFreeAsync(c.ring, st);
  if (c.fresh) cudaFreeAsync(c.fresh, st);
  if (c.counts) cudaFreeAsync(c.counts, st);
  c.ring = nullptr, c.fresh = nullptr, c.counts = nullptr;
}

static void CUDART_CB on_frame_done(void *arg) {
  Pending *p = static_cast<Pending *>(arg);
  {
    std::lock_guard<std::mutex> lock(p->srv->mu);
    ocq_completion c;
    c.camera = p->camera;
    c.frame = p->frame;
    c.tag = p->tag;
    c.arrival_s = p->arrival;
    c.done_s = now_s();
    p->srv->done.push_back(c);
    p->srv->completed++;
  }
  delete p;
}

extern "C" {

ocq_status ocq_server_create(size_t hbm_budget, int max_cameras, ocq_server **out) {
  if (!out || max_cameras < 1) {
    set_error("ocq_server_create: need out and max_cameras >= 1");
    return OCQ_EINVAL;
  }
  ocq_server *s = new (std::nothrow) ocq_server();
  if (!s) return OCQ_ENOMEM;
  s->budget = hbm_budget;
  s->max_cameras = max_cameras;
  s->cams.resize(max_cameras);
  // A pool of its own that keeps up to the budget mapped after frees, so a
  // camera's release and the next admission do not unmap and map gigabytes
  // (the default pool returns freed memory at every synchronisation, which
  // blocks the calling thread for every camera it serves).
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPoolProps props;
  memset(&props, 0, sizeof props);
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  ocq_status rc = cuda_status(cudaMemPoolCreate(&s->pool, &props), "server memory pool");
  if (rc == OCQ_OK) {
    uint64_t keep = hbm_budget;
    rc = cuda_status(cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep), "pool threshold");
  }
  // Map the whole budget now: growing the pool later maps memory on the
  // thread that admits or submits, in the middle of serving.
  if (rc == OCQ_OK && hbm_budget > 0) {
    cudaStream_t st = nullptr;
    void *p = nullptr;
    rc = cuda_status(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "reserve stream");
    if (rc == OCQ_OK) rc = cuda_status(cudaMallocFromPoolAsync(&p, hbm_budget, s->pool, st), "reserving the budget");
    if (p) cudaFreeAsync(p, st);
    if (st) {
      cudaError_t e = cudaStreamSynchronize(st);
      if (rc == OCQ_OK) rc = cuda_status(e, "reserving the budget");
      cudaStreamDestroy(st);
    }
  }
  if (rc != OCQ_OK) {
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return rc;
  }
  *out = s;
  return OCQ_OK;
}

size_t ocq_server_camera_footprint(const ocq_camera_desc *d) {
  if (!d || ocq_model_footprint(d->H, d->W, d->region, d->depth) == 0 || d->N < 1) return 0;
  return camera_footprint(*d);
}

size_t ocq_server_window_bytes(const ocq_camera_desc *d) {
  if (!d || ocq_model_footprint(d->H, d->W, d->region, d->depth) == 0 || d->N < 1) return 0;
  return (size_t)d->N * window_slot_bytes(*d, window_form(*d));
}

ocq_status ocq_server_admit(ocq_server *s, const ocq_camera_desc *d, const uint8_t *train, int *camera) {
  if (!s || !d || !train || !camera || d->N < 1 || d->N > 65535 || d->T < 1 || d->T > d->N || d->K < 1 ||
      ocq_model_footprint(d->H, d->W, d->region, d->depth) == 0) {
    set_error("ocq_server_admit: bad camera description");
    return OCQ_EINVAL;
  }
  const size_t fp = camera_footprint(*d);
  int slot = -1;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (int i = 0; i < s->max_cameras; ++i)
      if (!s->cams[i].live) {
        slot = i;
        break;
      }
    if (slot < 0 || s->used + fp > s->budget) {
      set_error("ocq_server_admit: no room (slots or HBM budget) for %zu bytes", fp);
      return OCQ_EBUSY;
    }
    s->used += fp;
    s->cams[slot].live = true;
  }
  PoolScope scope(s->pool);
  Camera &c = s->cams[slot];
  c.id = slot;
  c.d = *d;
  c.footprint = fp;
  c.submitted = 0;
  c.win = window_form(*d);
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);  // lo = least urgent, hi = most urgent
  ocq_status rc = cuda_status(cudaStreamCreateWithPriority(&c.stream, cudaStreamNonBlocking, hi), "camera stream");
  if (rc == OCQ_OK) rc = cuda_status(cudaStreamCreateWithPriority(&c.merge, cudaStreamNonBlocking, lo), "merge stream");
  if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&c.ring_ready, cudaEventDisableTiming), "event");
  if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&c.merged, cudaEventDisableTiming), "event");
  if (rc == OCQ_OK) rc = window_fill(c, train);
  if (rc == OCQ_OK) rc = ocq_build_model(train, d->N, d->H, d->W, d->region, d->depth, d->T, c.merge, &c.model);
  if (rc == OCQ_OK) rc = cuda_status(cudaEventRecord(c.merged, c.merge), "merged");
  if (rc == OCQ_OK) rc = cuda_status(cudaStreamWaitEvent(c.stream, c.merged, 0), "wait for M_0");
  if (rc != OCQ_OK) {
    if (c.model) ocq_model_free(c.model);
    c.model = nullptr;
    window_free(c, c.merge);
    if (c.merge) cudaStreamSynchronize(c.merge), cudaStreamDestroy(c.merge);
    if (c.stream) cudaStreamSynchronize(c.stream), cudaStreamDestroy(c.stream);
    if (c.ring_ready) cudaEventDestroy(c.ring_ready);
    if (c.merged) cudaEventDestroy(c.merged);
    c.ring = nullptr, c.stream = nullptr, c.merge = nullptr, c.ring_ready = nullptr, c.merged = nullptr;
    std::lock_guard<std::mutex> lock(s->mu);
    s->used -= fp;
    c.live = false;
    return rc;
  }
  *camera = slot;
  return OCQ_OK;
}

ocq_status ocq_server_submit(ocq_server *s, int camera, const uint8_t *frame, uint8_t *mask, uint64_t tag) {
  if (!s || camera < 0 || camera >= s->max_cameras || !s->cams[camera].live || !frame || !mask) {
    set_error("ocq_server_submit: bad camera or buffers");
    return OCQ_EINVAL;
  }
  PoolScope scope(s->pool);
  Camera &c = s->cams[camera];
  const double arrival = now_s();
  const int64_t t = c.submitted++;
  const size_t fbytes = (size_t)c.d.H * c.d.W * 3;
  ocq_status rc = ocq_classify(c.model, frame, 1, mask, c.stream);
  if (rc != OCQ_OK) return rc;
  Pending *p = new (std::nothrow) Pending{s, camera, t, tag, arrival};
  if (!p) return OCQ_ENOMEM;
  rc = cuda_status(cudaLaunchHostFunc(c.stream, on_frame_done, p), "completion callback");
  if (rc != OCQ_OK) {
    delete p;
    return rc;
  }
  const int64_t slot = (c.d.N + t) % c.d.N;
  if (c.win == WIN_BITS) {
    // the frame's leaf bitset enters the window; every K frames the counts
    // are thresholded into the model (in place: later frames read it)
    uint32_t *ring = reinterpret_cast<uint32_t *>(c.ring) + slot * wpr32(c.d.depth);
    rc = launch_frame_occupancy(frame, 1, c.d.H, c.d.W, c.d.depth, c.fresh, c.stream);
    if (rc == OCQ_OK) rc = launch_window_count_update(ring, c.fresh, c.counts, c.d.depth, c.stream);
    if (rc == OCQ_OK && (t + 1) % c.d.K == 0)
      rc = launch_window_threshold(c.counts, c.d.depth, (uint32_t)c.d.T, c.model->bits, c.stream);
    return rc;
  }
  if (c.win == WIN_CODES) {
    uint16_t *ring = reinterpret_cast<uint16_t *>(c.ring);
    rc = launch_window_codes(frame, (int64_t)c.d.H * c.d.W, c.d.depth, ring + slot * c.d.H * c.d.W, c.stream);
    if (rc == OCQ_OK && (t + 1) % c.d.K == 0) rc = launch_remerge_codes(ring, c.d.N, c.model, c.stream);
    return rc;
  }
  rc = cuda_status(cudaMemcpyAsync(c.ring + (size_t)slot * fbytes, frame, fbytes, cudaMemcpyDeviceToDevice, c.stream),
                   "ring push");
  if (rc == OCQ_OK && (t + 1) % c.d.K == 0) {
    // Re-merge on the low-priority stream once the ring holds frame t; the
    // camera's later frames wait for the new model.  The old model is freed
    // on the camera stream after the last frame that reads it.
    rc = cuda_status(cudaEventRecord(c.ring_ready, c.stream), "ring ready");
    if (rc == OCQ_OK) rc = cuda_status(cudaStreamWaitEvent(c.merge, c.ring_ready, 0), "merge wait");
    ocq_model *next = nullptr;
    if (rc == OCQ_OK) rc = ocq_build_model(c.ring, c.d.N, c.d.H, c.d.W, c.d.region, c.d.depth, c.d.T, c.merge, &next);
    if (rc == OCQ_OK) rc = cuda_status(cudaEventRecord(c.merged, c.merge), "merged");
    if (rc == OCQ_OK) rc = cuda_status(cudaStreamWaitEvent(c.stream, c.merged, 0), "wait for the new model");
    if (rc == OCQ_OK) {
      c.model->stream = c.stream;  // freed in camera-stream order, after the frames that used it
      ocq_model_free(c.model);
      c.model = next;
    } else if (next) {
      ocq_model_free(next);
    }
  }
  return rc;
}

ocq_status ocq_server_poll(ocq_server *s, ocq_completion *out, int max, int *n) {
  if (!s || !n || max < 0 || (max > 0 && !out)) {
    set_error("ocq_server_poll: bad arguments");
    return OCQ_EINVAL;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  int k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n = k;
  return OCQ_OK;
}

ocq_status ocq_server_release(ocq_server *s, int camera) {
  if (!s || camera < 0 || camera >= s->max_cameras || !s->cams[camera].live) {
    set_error("ocq_server_release: bad camera");
    return OCQ_EINVAL;
  }
  Camera &c = s->cams[camera];
  // Builds and frames both finish before the memory goes back to the pool.
  cudaStreamWaitEvent(c.stream, c.merged, 0);
  c.model->stream = c.stream;
  ocq_model_free(c.model);
  window_free(c, c.stream);
  cudaError_t e = cudaStreamSynchronize(c.stream);
  cudaError_t e2 = cudaStreamSynchronize(c.merge);
  if (e == cudaSuccess) e = e2;
  cudaStreamDestroy(c.stream);
  cudaStreamDestroy(c.merge);
  cudaEventDestroy(c.ring_ready);
  cudaEventDestroy(c.merged);
  c.model = nullptr, c.ring = nullptr, c.stream = nullptr, c.merge = nullptr;
  c.ring_ready = nullptr, c.merged = nullptr;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->used -= c.footprint;
    c.live = false;
  }
  return cuda_status(e, "camera release");
}

ocq_status ocq_server_snapshot(ocq_server *s, int camera, uint64_t *model_words, size_t words, uint8_t *ring_out,
                               int64_t *submitted, void *stream) {
  if (!s || camera < 0 || camera >= s->max_cameras || !s->cams[camera].live || !model_words || !ring_out ||
      !submitted) {
    set_error("ocq_server_snapshot: bad camera or buffers");
    return OCQ_EINVAL;
  }
  Camera &c = s->cams[camera];
  const int64_t t = c.submitted;
  const size_t fbytes = window_slot_bytes(c.d, c.win);
  // After t test frames the window holds global frames t .. t + N - 1
  // (training frames are 0 .. N - 1), frame g in slot g mod N: copy the slots
  // oldest first.
  ocq_status rc = cuda_status(cudaStreamWaitEvent(c.stream, c.merged, 0), "snapshot wait");
  if (rc == OCQ_OK) rc = ocq_model_export(c.model, model_words, words, c.stream);
  for (int i = 0; i < c.d.N && rc == OCQ_OK; ++i)
    rc = cuda_status(cudaMemcpyAsync(ring_out + (size_t)i * fbytes, c.ring + (size_t)((t + i) % c.d.N) * fbytes,
                                     fbytes, cudaMemcpyDeviceToDevice, c.stream),
                     "snapshot ring");
  cudaEvent_t done = nullptr;
  if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&done, cudaEventDisableTiming), "event");
  if (rc == OCQ_OK) rc = cuda_status(cudaEventRecord(done, c.stream), "snapshot done");
  if (rc == OCQ_OK) rc = cuda_status(cudaStreamWaitEvent((cudaStream_t)stream, done, 0), "snapshot join");
  if (done) cudaEventDestroy(done);
  if (rc == OCQ_OK) *submitted = t;
  return rc;
}

ocq_status ocq_server_resume(ocq_server *s, const ocq_camera_desc *d, const uint64_t *model_words,
                             const uint8_t *ring, int64_t submitted, int *camera) {
  if (!s || !d || !model_words || !ring || !camera || submitted < 0 || d->N < 1 || d->N > 65535 || d->T < 1 ||
      d->T > d->N || d->K < 1 || ocq_model_footprint(d->H, d->W, d->region, d->depth) == 0) {
    set_error("ocq_server_resume: bad camera description or snapshot");
    return OCQ_EINVAL;
  }
  const size_t fp = camera_footprint(*d);
  int slot = -1;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (int i = 0; i < s->max_cameras; ++i)
      if (!s->cams[i].live) {
        slot = i;
        break;
      }
    if (slot < 0 || s->used + fp > s->budget) {
      set_error("ocq_server_resume: no room (slots or HBM budget) for %zu bytes", fp);
      return OCQ_EBUSY;
    }
    s->used += fp;
    s->cams[slot].live = true;
  }
  PoolScope scope(s->pool);
  Camera &c = s->cams[slot];
  c.id = slot;
  c.d = *d;
  c.footprint = fp;
  c.submitted = submitted;
  c.win = window_form(*d);
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  ocq_status rc = cuda_status(cudaStreamCreateWithPriority(&c.stream, cudaStreamNonBlocking, hi), "camera stream");
  if (rc == OCQ_OK) rc = cuda_status(cudaStreamCreateWithPriority(&c.merge, cudaStreamNonBlocking, lo), "merge stream");
  if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&c.ring_ready, cudaEventDisableTiming), "event");
  if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&c.merged, cudaEventDisableTiming), "event");
  const size_t fbytes = window_slot_bytes(*d, c.win);
  if (rc == OCQ_OK) rc = cuda_status(malloc_async((void **)&c.ring, (size_t)d->N * fbytes, c.merge), "camera window");
  for (int i = 0; i < d->N && rc == OCQ_OK; ++i)  // snapshot slot i is global frame submitted + i
    rc = cuda_status(cudaMemcpyAsync(c.ring + (size_t)((submitted + i) % d->N) * fbytes, ring + (size_t)i * fbytes,
                                     fbytes, cudaMemcpyDeviceToDevice, c.merge),
                     "window restore");
  if (rc == OCQ_OK && c.win == WIN_BITS) {  // the counts follow from the bitsets
    rc = cuda_status(malloc_async((void **)&c.fresh, fbytes, c.merge), "window bitset");
    if (rc == OCQ_OK)
      rc = cuda_status(malloc_async((void **)&c.counts, ((size_t)1 << (3 * d->depth)) * 2, c.merge), "window counts");
    if (rc == OCQ_OK) rc = cuda_status(cudaMemsetAsync(c.fresh, 0, fbytes, c.merge), "clear window");
    if (rc == OCQ_OK)
      rc = launch_window_counts_init(reinterpret_cast<uint32_t *>(c.ring), d->N, d->depth, c.counts, c.merge);
  }
  if (rc == OCQ_OK) {
    ocq_model_info info;
    memset(&info, 0, sizeof info);
    info.H = d->H, info.W = d->W, info.region_kind = d->region.kind, info.block = d->region.block;
    info.depth = d->depth, info.T = d->T, info.N = d->N;
    rc = ocq_model_import(model_words, &info, c.merge, &c.model);
  }
  if (rc == OCQ_OK) rc = cuda_status(cudaEventRecord(c.merged, c.merge), "merged");
  if (rc == OCQ_OK) rc = cuda_status(cudaStreamWaitEvent(c.stream, c.merged, 0), "wait for the model");
  if (rc != OCQ_OK) {
    if (c.model) ocq_model_free(c.model);
    window_free(c, c.merge);
    if (c.merge) cudaStreamSynchronize(c.merge), cudaStreamDestroy(c.merge);
    if (c.stream) cudaStreamSynchronize(c.stream), cudaStreamDestroy(c.stream);
    if (c.ring_ready) cudaEventDestroy(c.ring_ready);
    if (c.merged) cudaEventDestroy(c.merged);
    c.model = nullptr, c.ring = nullptr, c.stream = nullptr, c.merge = nullptr, c.ring_ready = nullptr;
    c.merged = nullptr;
    std::lock_guard<std::mutex> lock(s->mu);
    s->used -= fp;
    c.live = false;
    return rc;
  }
  *camera = slot;
  return OCQ_OK;
}

ocq_status ocq_server_camera_model(const ocq_server *s, int camera, const ocq_model **out) {
  if (!s || !out || camera < 0 || camera >= s->max_cameras || !s->cams[camera].live) {
    set_error("ocq_server_camera_model: bad camera");
    return OCQ_EINVAL;
  }
  *out = s->cams[camera].model;
  return OCQ_OK;
}

ocq_status ocq_server_usage(ocq_server *s, size_t *used, size_t *budget, int64_t *completed) {
  if (!s) {
    set_error("ocq_server_usage: NULL server");
    return OCQ_EINVAL;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  if (used) *used = s->used;
  if (budget) *budget = s->budget;
  if (completed) *completed = s->completed;
  return OCQ_OK;
}

ocq_status ocq_server_sync(ocq_server *s) {
  if (!s) {
    set_error("ocq_server_sync: NULL server");
    return OCQ_EINVAL;
  }
  for (Camera &c : s->cams)
    if (c.live) {
      cudaError_t e = cudaStreamSynchronize(c.stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c.merge);
      if (e != cudaSuccess) return cuda_status(e, "server sync");
    }
  return OCQ_OK;
}

void ocq_server_destroy(ocq_server *s) {
  if (!s) return;
  for (int i = 0; i < s->max_cameras; ++i)
    if (s->cams[i].live) ocq_server_release(s, i);
  if (s->pool) cudaMemPoolDestroy(s->pool);  // every camera's memory was freed and its stream synchronised
  delete s;
}

}  // extern "C"
