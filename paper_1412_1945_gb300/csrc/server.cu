// Served form: camera streams join and leave while frames arrive; each
// camera's model and its sliding window of the last N frames stay resident
// in HBM.  The title of the paper's Sec. 4 mentions updating the octree but
// gives no procedure; the window semantics here are:
//   * the N training frames build M_0 (Sec. 3, Alg. 1-2);
//   * test frame t (t = 0, 1, ...) is classified against M_floor(t/K) (Alg. 3);
//   * after classification frame t enters a ring of the last N frames;
//   * when (t+1) % K == 0 the ring is merged again: M_(t+1)/K = merge(ring).
// So M_k is the merged model of global frames [kK, kK+N-1] (training frames
// first).  The window keeps what the merge needs of those frames, not the
// frames (window.cu): whole-frame cameras a ring of N leaf bitsets plus
// resident per-leaf counts, updated as each frame enters (re-merge = a
// threshold pass); pixel and block cameras of depth <= 5 a ring of per-pixel
// u16 leaf codes (re-merge = counting the codes, no frame is read again).
// Frames of those cameras run in ticks on the server's high-priority stream
// (continuous batching): a tick classifies every camera's frames that arrived
// by grouped launches, a camera's frames of the tick against one read of its
// model (the classify also writes a code window's slots), then enters the
// frames into their windows and re-merges in place the cameras whose period
// ends; ticks follow in stream order, so frame t always meets M_floor(t/K).
// Cameras outside those forms (deeper, N > 255, blocks wider than 16, or a
// whole-frame bitset larger than a frame) keep the N frames, classify frame by
// frame on their own high-priority stream and rebuild with ocq_build_model on
// a low-priority one, joined by events.
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

#include "grouped.cuh"
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
  uint32_t *fresh = nullptr;   // WIN_BITS: the entering frames' bitsets (N slots)
  uint16_t *counts = nullptr;  // WIN_BITS: per leaf, window frames holding it
  bool m0_joined = false;      // the server's tick stream waits for M_0 once
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
  // Continuous batching: the frames of cameras with a bitset or code window
  // run in ticks on one high-priority stream; a tick classifies every frame
  // it holds (of every camera) and enters them into their windows with a few
  // grouped launches.
  cudaStream_t tick = nullptr;
  cudaEvent_t tick_ev = nullptr;
  uint8_t *d_tick = nullptr;  // a tick's segments and frame tables on the device
  size_t tick_cap = 0;
  // page-locked staging of the uploads (a ring, so that a tick's copy never
  // waits for the previous one's)
  struct Stage {
    uint8_t *host = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
  };
  Stage stage[4];
  int stage_next = 0;
  std::vector<uint8_t *> retired;  // outgrown staging, freed with the server (freeing syncs the device)
  // frames of cameras whose M_0 is still being built: held on the host (a tick
  // would otherwise wait for the build and hold back every other camera)
  struct Held {
    int camera;
    const uint8_t *frame;
    uint8_t *mask;
    uint64_t tag;
    double arrival;
  };
  std::vector<Held> held;
  // batching (ocq_server_set_batching): seconds a tick frame may wait for
  // others; ticks enqueued and not yet finished (end events, oldest first),
  // beyond which frames wait on the host and join the next, larger tick
  double batch_delay = 0.0;
  int max_in_flight = 2;
  std::deque<cudaEvent_t> in_flight;
  std::vector<cudaEvent_t> spare_events;
};

// Cameras whose frames run in ticks (windows the grouped tick kernels serve).
static bool tick_camera(const Camera &c) {
  return c.win == WIN_CODES || (c.win == WIN_BITS && c.d.depth <= 6);
}

struct TickDone {
  ocq_server *srv;
  std::vector<Pending> frames;
};

static void CUDART_CB on_tick_done(void *arg) {
  TickDone *d = static_cast<TickDone *>(arg);
  {
    std::lock_guard<std::mutex> lock(d->srv->mu);
    const double t = now_s();
    for (const Pending &p : d->frames) {
      ocq_completion c;
      c.camera = p.camera;
      c.frame = p.frame;
      c.tag = p.tag;
      c.arrival_s = p.arrival;
      c.done_s = t;
      d->srv->done.push_back(c);
      d->srv->completed++;
    }
  }
  delete d;
}

static size_t camera_footprint(const ocq_camera_desc &d) {
  const size_t hw = (size_t)d.H * d.W;
  const size_t model = model_bytes(d.H, d.W, d.region, d.depth, d.N, d.T);
  const int form = window_form(d);
  const size_t ring = (size_t)d.N * window_slot_bytes(d, form);
  size_t scratch = 0;  // what a build of the model allocates beside it
  if (d.region.kind == OCQ_REGION_FRAME) scratch = (size_t)d.N * wpr32(d.depth) * 4;
  if (d.region.kind == OCQ_REGION_PIXEL && d.depth >= 6) scratch = hw * ((size_t)1 << (3 * d.depth - 9)) / 8;
  if (form == WIN_BITS)  // N entering-frame bitsets and the u16 counts; re-merged in place
    return model + 2 * ring + ((size_t)1 << (3 * d.depth)) * 2 + scratch;
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
  rc = cuda_status(malloc_async((void **)&c.fresh, (size_t)d.N * slot, c.merge), "window bitsets");
  if (rc == OCQ_OK)
    rc = cuda_status(malloc_async((void **)&c.counts, ((size_t)1 << (3 * d.depth)) * 2, c.merge), "window counts");
  if (rc == OCQ_OK) rc = cuda_status(cudaMemsetAsync(c.ring, 0, (size_t)d.N * slot, c.merge), "clear window");
  if (rc == OCQ_OK) rc = cuda_status(cudaMemsetAsync(c.fresh, 0, (size_t)d.N * slot, c.merge), "clear window");
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
  if (rc == OCQ_OK) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    rc = cuda_status(cudaStreamCreateWithPriority(&s->tick, cudaStreamNonBlocking, hi), "tick stream");
    if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&s->tick_ev, cudaEventDisableTiming), "tick event");
  }
  if (rc != OCQ_OK) {
    if (s->tick_ev) cudaEventDestroy(s->tick_ev);
    if (s->tick) cudaStreamDestroy(s->tick);
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
  c.m0_joined = false;
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

// The per-frame path (cameras that keep their frames): classify on the
// camera's stream, completion callback, ring copy, and every K frames a
// rebuild on the camera's low-priority stream.
static ocq_status submit_frame_path(ocq_server *s, int camera, const uint8_t *frame, uint8_t *mask, uint64_t tag,
                                    double arrival) {
  Camera &c = s->cams[camera];
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

// One tick: the frames `idx` (in submission order, at most N per camera and
// none after a camera's re-merge frame) classified by grouped launches on the
// tick stream, one completion callback when their masks are written, then
// their window entries and the re-merges that fall at the tick's end.
static ocq_status run_tick(ocq_server *s, const std::vector<int> &idx, const int *cameras,
                           const uint8_t *const *frames, uint8_t *const *masks, const uint64_t *tags,
                           const double *arrival) {
  std::vector<GFrameIn> fin;
  std::vector<int> first(s->max_cameras, -1), taken(s->max_cameras, 0);
  TickDone *done = new (std::nothrow) TickDone();
  if (!done) return OCQ_ENOMEM;
  done->srv = s;
  ocq_status rc = OCQ_OK;
  for (int i : idx) {
    Camera &c = s->cams[cameras[i]];
    if (!c.m0_joined) {  // M_0 (admission or resume) is built on the camera's build stream
      rc = cuda_status(cudaStreamWaitEvent(s->tick, c.merged, 0), "wait for M_0");
      if (rc != OCQ_OK) break;
      c.m0_joined = true;
    }
    const int64_t t = c.submitted + taken[c.id];
    GFrameIn f;
    f.frame = frames[i], f.mask = masks[i], f.model = c.model, f.win = c.win == WIN_BITS ? 1 : 2;
    f.ring = c.ring, f.fresh = c.fresh, f.counts = c.counts, f.N = c.d.N;
    f.slot = (c.d.N + t) % c.d.N, f.j = taken[c.id], f.m = 0;
    if (first[c.id] < 0) first[c.id] = (int)fin.size();
    taken[c.id]++;
    fin.push_back(f);
    done->frames.push_back(Pending{s, c.id, t, tags[i], arrival[i]});
  }
  for (GFrameIn &f : fin)
    if (f.j == 0) f.m = taken[done->frames[&f - &fin[0]].camera];
  std::vector<GLaunch> L;
  std::vector<int> single;
  std::vector<const void *> ptrs;
  if (rc == OCQ_OK) rc = grouped_plan_tick(fin, L, single, ptrs);
  size_t nseg = 0;
  for (const GLaunch &x : L) nseg += x.segs.size();
  const size_t seg_bytes = nseg * sizeof(GSeg), bytes = seg_bytes + ptrs.size() * sizeof(void *);
  if (rc == OCQ_OK && bytes > s->tick_cap) {  // stream-ordered: earlier ticks' kernels are done with it
    if (s->d_tick) cudaFreeAsync(s->d_tick, s->tick);
    s->d_tick = nullptr;
    s->tick_cap = std::max(bytes, 2 * s->tick_cap);
    rc = cuda_status(malloc_async((void **)&s->d_tick, s->tick_cap, s->tick), "tick segments");
  }
  if (rc == OCQ_OK && bytes) {
    ocq_server::Stage &sg = s->stage[s->stage_next];
    s->stage_next = (s->stage_next + 1) % 4;
    if (sg.done) rc = cuda_status(cudaEventSynchronize(sg.done), "tick staging");  // that upload has ended
    if (rc == OCQ_OK && sg.cap < bytes) {
      if (sg.host) s->retired.push_back(sg.host);
      sg.host = nullptr, sg.cap = 0;
      const size_t cap = std::max<size_t>(2 * bytes, 256 * 1024);
      rc = cuda_status(cudaHostAlloc((void **)&sg.host, cap, cudaHostAllocDefault), "tick staging");
      if (rc == OCQ_OK) sg.cap = cap;
    }
    if (rc == OCQ_OK && !sg.done) rc = cuda_status(cudaEventCreateWithFlags(&sg.done, cudaEventDisableTiming), "tick staging");
    if (rc == OCQ_OK) {
      GSeg *hs = reinterpret_cast<GSeg *>(sg.host);
      const uint8_t *const *dtab = reinterpret_cast<const uint8_t *const *>(s->d_tick + seg_bytes);
      for (const GLaunch &x : L)
        for (GSeg g : x.segs) {
          if (g.tab >= 0) {
            g.ftab = dtab + g.tab;
            g.mtab = const_cast<uint8_t *const *>(dtab + g.tab + g.F);
            if (g.codes)
              g.ctab = reinterpret_cast<uint16_t *const *>(const_cast<uint8_t *const *>(dtab + g.tab + 2 * g.F));
          }
          *hs++ = g;
        }
      if (!ptrs.empty()) memcpy(sg.host + seg_bytes, ptrs.data(), ptrs.size() * sizeof(void *));
      rc = cuda_status(cudaMemcpyAsync(s->d_tick, sg.host, bytes, cudaMemcpyHostToDevice, s->tick),
                       "upload tick segments");
      if (rc == OCQ_OK) rc = cuda_status(cudaEventRecord(sg.done, s->tick), "tick staging");
    }
  }
  size_t at = 0;
  for (GLaunch &x : L) x.dev = reinterpret_cast<GSeg *>(s->d_tick) + at, at += x.segs.size();
  for (size_t k = 0; k < single.size() && rc == OCQ_OK; ++k)
    rc = ocq_classify(fin[single[k]].model, fin[single[k]].frame, 1, fin[single[k]].mask, s->tick);
  size_t li = 0;
  for (; li < L.size() && rc == OCQ_OK; ++li) {  // classification (window launches follow)
    if (L[li].kind == GK_CODES || L[li].kind == GK_OCC || L[li].kind == GK_COUNT) break;
    rc = grouped_launch(L[li], s->tick);
  }
  if (rc == OCQ_OK) {  // the masks are written: completion time
    rc = cuda_status(cudaLaunchHostFunc(s->tick, on_tick_done, done), "tick completion");
    if (rc == OCQ_OK) done = nullptr;
  }
  for (; li < L.size() && rc == OCQ_OK; ++li) rc = grouped_launch(L[li], s->tick);
  // re-merges: a camera's last frame of the tick closes its window period
  for (int cam = 0; cam < s->max_cameras && rc == OCQ_OK; ++cam) {
    if (!taken[cam]) continue;
    Camera &c = s->cams[cam];
    c.submitted += taken[cam];
    if (c.submitted % c.d.K != 0) continue;
    if (c.win == WIN_BITS)
      rc = launch_window_threshold(c.counts, c.d.depth, (uint32_t)c.d.T, c.model->bits, s->tick);
    else
      rc = launch_remerge_codes(reinterpret_cast<uint16_t *>(c.ring), c.d.N, c.model, s->tick);
  }
  if (rc == OCQ_OK) {  // the tick's end, for the in-flight limit
    cudaEvent_t e = nullptr;
    if (!s->spare_events.empty()) {
      e = s->spare_events.back();
      s->spare_events.pop_back();
    } else {
      rc = cuda_status(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "tick end");
    }
    if (rc == OCQ_OK) rc = cuda_status(cudaEventRecord(e, s->tick), "tick end");
    if (e) s->in_flight.push_back(e);
  }
  delete done;
  return rc;
}

// Runs the frames `pending` (indices into the arrays, submission order) of
// cameras served in ticks as ticks, each holding for every camera its next
// frames up to its next re-merge (and at most N).
static ocq_status run_ticks(ocq_server *s, std::vector<int> pending, const int *cameras, const uint8_t *const *frames,
                            uint8_t *const *masks, const uint64_t *tags, const double *arrival) {
  std::vector<int> take, rest, count(s->max_cameras, 0);
  std::vector<char> closed(s->max_cameras, 0);
  ocq_status rc = OCQ_OK;
  while (rc == OCQ_OK && !pending.empty()) {
    take.clear(), rest.clear();
    std::fill(count.begin(), count.end(), 0);
    std::fill(closed.begin(), closed.end(), 0);
    for (int i : pending) {
      const Camera &c = s->cams[cameras[i]];
      if (closed[c.id]) {
        rest.push_back(i);
        continue;
      }
      const int64_t t = c.submitted + count[c.id];
      take.push_back(i);
      if (++count[c.id] == c.d.N || (t + 1) % c.d.K == 0) closed[c.id] = 1;
    }
    rc = run_tick(s, take, cameras, frames, masks, tags, arrival);
    pending.swap(rest);
  }
  return rc;
}

static bool m0_ready(Camera &c) { return c.m0_joined || cudaEventQuery(c.merged) == cudaSuccess; }

// Moves held frames of cameras whose M_0 is ready (all of them with `wait`)
// into ticks, after first appending `extra` frames; frames of a camera stay
// in submission order (a camera with held frames holds its new ones too).
static ocq_status flush(ocq_server *s, bool wait, int n = 0, const int *cameras = nullptr,
                        const uint8_t *const *frames = nullptr, uint8_t *const *masks = nullptr,
                        const uint64_t *tags = nullptr, double arrival = 0.0) {
  for (int i = 0; i < n; ++i) s->held.push_back({cameras[i], frames[i], masks[i], tags[i], arrival});
  if (s->held.empty()) return OCQ_OK;
  std::vector<char> ready(s->max_cameras, 0), seen(s->max_cameras, 0);
  std::vector<int> cam, idx;
  std::vector<const uint8_t *> fr;
  std::vector<uint8_t *> mk;
  std::vector<uint64_t> tg;
  std::vector<double> ar;
  std::vector<ocq_server::Held> keep;
  double oldest = 1e300;
  for (const ocq_server::Held &h : s->held) {
    Camera &c = s->cams[h.camera];
    if (!seen[h.camera]) {
      seen[h.camera] = 1;
      if (wait && !c.m0_joined) cudaEventSynchronize(c.merged);
      ready[h.camera] = m0_ready(c);
    }
    if (ready[h.camera]) oldest = std::min(oldest, h.arrival);
  }
  // batching window: the frames wait until the oldest ready one is old enough
  if (!wait && s->batch_delay > 0.0 && now_s() - oldest < s->batch_delay) return OCQ_OK;
  // and while the GPU still has max_in_flight ticks to run
  while (!s->in_flight.empty() && cudaEventQuery(s->in_flight.front()) == cudaSuccess) {
    s->spare_events.push_back(s->in_flight.front());
    s->in_flight.pop_front();
  }
  if (!wait && s->max_in_flight > 0 && (int)s->in_flight.size() >= s->max_in_flight) return OCQ_OK;
  for (const ocq_server::Held &h : s->held) {
    if (!ready[h.camera]) {
      keep.push_back(h);
      continue;
    }
    idx.push_back((int)cam.size());
    cam.push_back(h.camera), fr.push_back(h.frame), mk.push_back(h.mask), tg.push_back(h.tag), ar.push_back(h.arrival);
  }
  s->held.swap(keep);
  if (idx.empty()) return OCQ_OK;
  return run_ticks(s, idx, cam.data(), fr.data(), mk.data(), tg.data(), ar.data());
}

// Continuous batching: the frames of cameras served in ticks go into ticks
// (held on the host while a camera's M_0 is being built); the other cameras'
// frames take the per-frame path.
static ocq_status submit_many(ocq_server *s, int n, const int *cameras, const uint8_t *const *frames,
                              uint8_t *const *masks, const uint64_t *tags) {
  for (int i = 0; i < n; ++i)
    if (cameras[i] < 0 || cameras[i] >= s->max_cameras || !s->cams[cameras[i]].live || !frames[i] || !masks[i]) {
      set_error("ocq_server_submit: bad camera or buffers (entry %d)", i);
      return OCQ_EINVAL;
    }
  PoolScope scope(s->pool);
  const double arrival = now_s();
  std::vector<int> cam;
  std::vector<const uint8_t *> fr;
  std::vector<uint8_t *> mk;
  std::vector<uint64_t> tg;
  ocq_status rc = OCQ_OK;
  for (int i = 0; i < n && rc == OCQ_OK; ++i) {
    if (tick_camera(s->cams[cameras[i]]))
      cam.push_back(cameras[i]), fr.push_back(frames[i]), mk.push_back(masks[i]), tg.push_back(tags[i]);
    else
      rc = submit_frame_path(s, cameras[i], frames[i], masks[i], tags[i], arrival);
  }
  if (rc == OCQ_OK) rc = flush(s, false, (int)cam.size(), cam.data(), fr.data(), mk.data(), tg.data(), arrival);
  return rc;
}

ocq_status ocq_server_submit(ocq_server *s, int camera, const uint8_t *frame, uint8_t *mask, uint64_t tag) {
  if (!s) {
    set_error("ocq_server_submit: NULL server");
    return OCQ_EINVAL;
  }
  return submit_many(s, 1, &camera, &frame, &mask, &tag);
}

ocq_status ocq_server_submit_many(ocq_server *s, int n, const int *cameras, const uint8_t *const *frames,
                                  uint8_t *const *masks, const uint64_t *tags) {
  if (!s || n < 0 || (n > 0 && (!cameras || !frames || !masks || !tags))) {
    set_error("ocq_server_submit_many: bad arguments");
    return OCQ_EINVAL;
  }
  return n ? submit_many(s, n, cameras, frames, masks, tags) : OCQ_OK;
}

ocq_status ocq_server_set_batching(ocq_server *s, double seconds, int ticks_in_flight) {
  if (!s || !(seconds >= 0.0 && seconds <= 1.0) || ticks_in_flight < 0) {
    set_error("ocq_server_set_batching: bad arguments");
    return OCQ_EINVAL;
  }
  s->batch_delay = seconds;
  s->max_in_flight = ticks_in_flight;
  if (!s->held.empty()) {
    PoolScope scope(s->pool);
    return flush(s, false);
  }
  return OCQ_OK;
}

ocq_status ocq_server_poll(ocq_server *s, ocq_completion *out, int max, int *n) {
  if (!s || !n || max < 0 || (max > 0 && !out)) {
    set_error("ocq_server_poll: bad arguments");
    return OCQ_EINVAL;
  }
  if (!s->held.empty()) {  // cameras whose M_0 is now built, frames whose batching window ended
    PoolScope scope(s->pool);
    ocq_status rc = flush(s, false);
    if (rc != OCQ_OK) return rc;
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
  if (!s->held.empty()) {  // the camera's held frames run first
    PoolScope scope(s->pool);
    flush(s, true);
  }
  Camera &c = s->cams[camera];
  // Builds and frames both finish before the memory goes back to the pool.
  cudaStreamWaitEvent(c.stream, c.merged, 0);
  if (tick_camera(c)) {  // its frames ran on the tick stream
    cudaEventRecord(s->tick_ev, s->tick);
    cudaStreamWaitEvent(c.stream, s->tick_ev, 0);
  }
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
  if (!s->held.empty()) {  // the camera's held frames run first
    PoolScope scope(s->pool);
    ocq_status rf = flush(s, true);
    if (rf != OCQ_OK) return rf;
  }
  Camera &c = s->cams[camera];
  const int64_t t = c.submitted;
  const size_t fbytes = window_slot_bytes(c.d, c.win);
  // After t test frames the window holds global frames t .. t + N - 1
  // (training frames are 0 .. N - 1), frame g in slot g mod N: copy the slots
  // oldest first.
  ocq_status rc = cuda_status(cudaStreamWaitEvent(c.stream, c.merged, 0), "snapshot wait");
  if (rc == OCQ_OK && tick_camera(c)) {  // after the ticks that hold its frames
    rc = cuda_status(cudaEventRecord(s->tick_ev, s->tick), "snapshot tick");
    if (rc == OCQ_OK) rc = cuda_status(cudaStreamWaitEvent(c.stream, s->tick_ev, 0), "snapshot wait");
  }
  if (rc == OCQ_OK) rc = ocq_model_export(c.model, model_words, words, c.stream);
  for (int i = 0; i < c.d.N && rc == OCQ_OK; ++i)
    rc = cuda_status(cudaMemcpyAsync(ring_out + (size_t)i * fbytes, c.ring + (size_t)((t + i) % c.d.N) * fbytes,
                                     fbytes, cudaMemcpyDeviceToDevice, c.stream),
                     "snapshot ring");
  cudaEvent_t done = nullptr;
  if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&done, cudaEventDisableTiming), "event");
  if (rc == OCQ_OK) rc = cuda_status(cudaEventRecord(done, c.stream), "snapshot done");
  if (rc == OCQ_OK) rc = cuda_status(cudaStreamWaitEvent((cudaStream_t)stream, done, 0), "snapshot join");
  // later ticks rewrite the window and the model: after the copies
  if (rc == OCQ_OK && tick_camera(c)) rc = cuda_status(cudaStreamWaitEvent(s->tick, done, 0), "snapshot tick join");
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
  c.m0_joined = false;
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
    rc = cuda_status(malloc_async((void **)&c.fresh, (size_t)d->N * fbytes, c.merge), "window bitsets");
    if (rc == OCQ_OK)
      rc = cuda_status(malloc_async((void **)&c.counts, ((size_t)1 << (3 * d->depth)) * 2, c.merge), "window counts");
    if (rc == OCQ_OK) rc = cuda_status(cudaMemsetAsync(c.fresh, 0, (size_t)d->N * fbytes, c.merge), "clear window");
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
  if (!s->held.empty()) {
    PoolScope scope(s->pool);
    ocq_status rc = flush(s, true);
    if (rc != OCQ_OK) return rc;
  }
  for (Camera &c : s->cams)
    if (c.live) {
      cudaError_t e = cudaStreamSynchronize(c.stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c.merge);
      if (e != cudaSuccess) return cuda_status(e, "server sync");
    }
  return cuda_status(cudaStreamSynchronize(s->tick), "server sync");
}

void ocq_server_destroy(ocq_server *s) {
  if (!s) return;
  for (int i = 0; i < s->max_cameras; ++i)
    if (s->cams[i].live) ocq_server_release(s, i);
  if (s->tick) {
    if (s->d_tick) cudaFreeAsync(s->d_tick, s->tick);
    cudaStreamSynchronize(s->tick);
    cudaStreamDestroy(s->tick);
  }
  if (s->tick_ev) cudaEventDestroy(s->tick_ev);
  for (uint8_t *h : s->retired) cudaFreeHost(h);
  for (cudaEvent_t e : s->in_flight) cudaEventDestroy(e);
  for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
  for (ocq_server::Stage &sg : s->stage) {  // the tick stream is synchronised: every upload has ended
    if (sg.host) cudaFreeHost(sg.host);
    if (sg.done) cudaEventDestroy(sg.done);
  }
  if (s->pool) cudaMemPoolDestroy(s->pool);  // every camera's memory was freed and its stream synchronised
  delete s;
}

}  // extern "C"
