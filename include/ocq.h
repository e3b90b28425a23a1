/*
 * ocq -- GB300 (sm_103a) library for the octree colour-quantisation background
 * model of "Background Modeling Using Octree Color Quantization" (arXiv 1412.1945).
 *
 * The method (paper Sec. 2-4):
 *   S1  each RGB8 pixel is quantised to its octree path: at level l (bit 7-l)
 *       the child index is (red bit << 2) | (green bit << 1) | blue bit
 *       (Alg. 1, with the printed sum of the three bits read as bit
 *       concatenation); pruning the tree at height d keeps the top d levels
 *       (Sec. 2).  The path code is the d child indices read as base-8 digits
 *       from the root (index of level 0 most significant).
 *   S2  one tree per training frame and region records which leaves occur
 *       (Store Color, Alg. 1; regions Sec. 3 and Sec. 4).
 *   S3  the N per-frame trees are merged keeping the leaves present in at least
 *       T of them (Merge Trees, Alg. 2, with the fraction test count/N >= t
 *       taken as the integer test count >= T, T = ceil(t*N)).
 *   S4  a pixel of an incoming frame is background when its leaf is in its
 *       region's merged tree, else foreground (Check Color, Alg. 3; Sec. 4).
 *
 * Conventions for every entry point:
 *   - Frames are HWC RGB8 with no row padding: byte ((f*H + y)*W + x)*3 + c.
 *     Masks are u8, one byte per pixel, 1 = foreground, 0 = background.
 *   - Buffers called "device" must be device-accessible memory of the current
 *     CUDA device; the caller owns them.  Nothing is retained after the call
 *     except inside an ocq_model (library-owned, freed by ocq_model_free).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued asynchronously on it; argument errors are returned
 *     synchronously before anything is enqueued; errors of enqueued work are
 *     reported by a later call (OCQ_ECUDA) or by the caller's synchronisation.
 *   - Nothing throws across this interface.  ocq_last_error() gives a message
 *     for the calling thread's last failure.
 *   - Domain: 1 <= depth <= 8; 1 <= T <= N <= 65535; H, W >= 1; H*W*N and
 *     H*W*F below 2^40; block >= 1 for block regions (partial edge blocks allowed).
 */
#ifndef OCQ_H
#define OCQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OCQ_OK = 0,
  OCQ_EINVAL = 1,   /* bad argument (null pointer, size or parameter out of domain) */
  OCQ_ENOMEM = 2,   /* device allocation failed or footprint above the budget */
  OCQ_ECUDA = 3,    /* a CUDA call failed (message in ocq_last_error) */
  OCQ_ETIMEOUT = 4, /* a bounded device-side wait gave up */
  OCQ_EBUSY = 5,    /* no capacity right now (serving admission); retry later */
  OCQ_ENOTSUP = 6   /* valid request the library does not handle */
} ocq_status;

/* Region geometry (Sec. 3 splits a video into regions with a tree each; Sec. 4).
 * FRAME: one region.  BLOCK: b x b blocks numbered row-major,
 * r = (y/b)*ceil(W/b) + x/b, partial blocks at the right/bottom edges.
 * PIXEL: one region per pixel location, r = y*W + x. */
typedef enum { OCQ_REGION_FRAME = 0, OCQ_REGION_BLOCK = 1, OCQ_REGION_PIXEL = 2 } ocq_region_kind;

typedef struct {
  int32_t kind;  /* ocq_region_kind */
  int32_t block; /* b for OCQ_REGION_BLOCK, ignored otherwise */
} ocq_region;

/* Opaque, device-resident merged model (library-owned). */
typedef struct ocq_model ocq_model;

/* Header of a model.  The exported bitset holds `regions` rows of
 * `words_per_region` u64 words; leaf path code c of a row is bit c%64 of word
 * c/64 (words_per_region = max(1, 8^depth/64)). */
typedef struct {
  int32_t H, W;
  int32_t region_kind, block;
  int32_t depth, T, N;
  int32_t reserved;
  int64_t regions;
  int64_t words_per_region;
} ocq_model_info;

/* Human-readable name of a status code (static string). */
const char *ocq_status_str(ocq_status s);

/* Message describing the calling thread's most recent failure ("" if none). */
const char *ocq_last_error(void);

/* Library version string (static). */
const char *ocq_version(void);

/* Number of regions of an H x W frame for `region`, or -1 if invalid. */
int64_t ocq_region_count(int H, int W, ocq_region region);

/* Device bytes an ocq_model of this geometry occupies at most (0 if invalid):
 * its leaf bitsets, plus for per-pixel regions of depth 4-5 a kept-leaf index
 * of 16 B per location (built with the model when no location can keep more
 * than 8 leaves, floor(N / T) <= 8; the classify then compares with it). */
size_t ocq_model_footprint(int H, int W, ocq_region region, int depth);

/*
 * S1 alone (Alg. 1 walk, Sec. 2 pruning): path code of each of `npix` pixels.
 * rgb: device, npix*3 bytes.  codes: device, npix u32 (code < 8^depth).
 */
ocq_status ocq_path_code(const uint8_t *rgb, int64_t npix, int depth, uint32_t *codes, void *stream);

/*
 * S2 alone (Alg. 1, one tree per frame and region): the leaf set of every
 * frame's per-region tree, as a bitset in the exported layout.
 * frames: device, n*H*W*3.  occ: device, n * regions * words_per_region u64,
 * frame-major (row index f*regions + r).  Every word is written.
 */
ocq_status ocq_occupancy(const uint8_t *frames, int n, int H, int W, ocq_region region, int depth,
                         uint64_t *occ, void *stream);

/*
 * S3 alone (Alg. 2) over leaf sets given as bitsets: the merged model of N
 * per-frame trees whose regions were each split into `parts` pieces (for
 * example row bands of whole frames held by different GPUs).  A frame's tree
 * of a region holds a leaf iff the tree of some piece does (Alg. 1 inserts
 * every pixel of the region into that one tree), so the pieces' bitsets are
 * ORed, and a leaf is kept when at least T of the N frames hold it.
 * occ: device, parts * N * regions * words_per_region u64 in the exported
 * layout, piece-major, each piece as ocq_occupancy writes it (row f*regions +
 * r).  H, W: the whole frame's size (regions count as for ocq_build_model).
 * The model has leaf bitset rows (no kept-leaf lists).  Scratch is
 * stream-ordered device memory.  Errors as ocq_build_model.
 */
ocq_status ocq_merge_occupancy(const uint64_t *occ, int parts, int N, int H, int W, ocq_region region, int depth,
                               int T, void *stream, ocq_model **out);

/*
 * S1-S3 (Sec. 3, Alg. 1 + Alg. 2): build the merged model of N training
 * frames.  frames: device, N*H*W*3 bytes.  On success *out owns a new
 * device-resident model, ready for use on `stream` once the enqueued work has
 * run.  Allocation uses stream-ordered device memory.
 */
ocq_status ocq_build_model(const uint8_t *frames, int N, int H, int W, ocq_region region, int depth, int T,
                           void *stream, ocq_model **out);

/*
 * S4 (Sec. 4, Alg. 3): classify F frames against `model`.
 * frames: device, F*H*W*3 bytes of the model's H x W.  mask: device, F*H*W
 * bytes, every byte written (1 = foreground).
 */
ocq_status ocq_classify(const ocq_model *model, const uint8_t *frames, int F, uint8_t *mask, void *stream);

/* Header of a model (host struct filled synchronously). */
ocq_status ocq_model_get_info(const ocq_model *model, ocq_model_info *info);

/* Writes the model as a bitset in the exported layout (see ocq_model_info) to
 * device buffer `dst` of `words` u64 (must be >= regions*words_per_region). */
ocq_status ocq_model_export(const ocq_model *model, uint64_t *dst, size_t words, void *stream);

/* Creates a model from an exported bitset `src` (device) and its header
 * (H, W, region_kind, block, depth are required; T and N are recorded).  When
 * the header describes a model ocq_build_model would build as a list model
 * (per-pixel, depth 4-5, 1 <= T <= N <= 255, floor(N/T) <= 8), the bitset is
 * read into lists: the call then waits for `stream` and returns OCQ_EINVAL if
 * a pixel location holds more than floor(N/T) leaves (more than N frames can
 * give leaves kept in T of them). */
ocq_status ocq_model_import(const uint64_t *src, const ocq_model_info *info, void *stream, ocq_model **out);

/* Frees a model (stream-ordered on the stream it was created on); NULL is ignored. */
void ocq_model_free(ocq_model *model);

/* Synchronises `stream`, then reports whether a kernel of this library on the
 * current device gave up a bounded wait (a bulk copy that did not arrive within
 * one second): OCQ_ETIMEOUT if so (the record is cleared), else OCQ_OK. */
ocq_status ocq_device_status(void *stream);

/*
 * End to end from HOST memory (Sec. 3-4: build on the first N frames, then
 * detect foreground in the next F): copies the N training frames to the device,
 * builds the model (as ocq_build_model), streams the F test frames through
 * device chunk buffers with copy-in, classification and mask copy-out
 * overlapped on three streams, and writes the F*H*W mask bytes to `mask`.
 * train: host, N*H*W*3 bytes; test: host, F*H*W*3; mask: host, F*H*W.
 * Page-locked host buffers give full copy bandwidth; pageable ones work too.
 * Synchronous: returns after every mask byte is in host memory.  Its device
 * staging buffers come from a pool of its own that stays mapped between calls
 * (about 1 GB for 1080p frames).  If
 * out_model is not NULL it receives the model (caller frees), else the model
 * is freed.
 */
ocq_status ocq_detect_host(const uint8_t *train, int N, const uint8_t *test, int F, int H, int W, ocq_region region,
                           int depth, int T, uint8_t *mask, void *stream, ocq_model **out_model);

/*
 * One tree per group of `group` consecutive training frames instead of one per
 * frame (Sec. 3 allows either; the last group holds the remaining frames).  A group's tree holds every leaf of any
 * of its frames; T counts trees: 1 <= T <= ceil(N / group).  group = 1 is
 * ocq_build_model.  Same buffers, ownership and errors as ocq_build_model.
 */
ocq_status ocq_build_model_groups(const uint8_t *frames, int N, int H, int W, ocq_region region, int depth, int T,
                                  int group, void *stream, ocq_model **out);

/*
 * Redraw (Sec. 2, Fig. 2): each pixel's colour becomes the colour of its leaf
 * in a tree pruned at `depth` levels, i.e. the depth most significant bits of
 * each channel followed by zeros.  rgb, out: device, npix*3 bytes (HWC RGB8);
 * out may equal rgb (in place).  Asynchronous on `stream`.
 */
ocq_status ocq_redraw(const uint8_t *rgb, int64_t npix, int depth, uint8_t *out, void *stream);

/*
 * Evaluation against ground truth (Sec. 5).  mask, gt: device, F*npix bytes
 * (frame-major; a non-zero byte is foreground in both).  counts: device,
 * F*4 u64 written as {Tp, Fp, Tn, Fn} per frame (foreground = positive).
 * Asynchronous on `stream`.
 */
ocq_status ocq_confusion(const uint8_t *mask, const uint8_t *gt, int F, int64_t npix, uint64_t *counts,
                         void *stream);
/*
 * Host: from counts {Tp, Fp, Tn, Fn} (one frame or their sum), the paper's
 * scores out[0] = P0 = Tn/(Tn+Fn), out[1] = R0 = Tn/(Tn+Fp),
 * out[2] = F0 = 2 P0 R0/(P0+R0), and out[3] = foreground F1 = 2Tp/(2Tp+Fp+Fn);
 * a ratio with a zero denominator is 1.
 */
ocq_status ocq_f_scores(const uint64_t *counts, double *out);

/*
 * Batched form (no counterpart in the paper, which handles one video): many
 * camera streams, each with its own frame size, region kind and depth, are
 * built (S1-S3) and classified (S4) by one CUDA graph, captured once and
 * replayed.  By default the graph holds ONE persistent kernel whose work items
 * are the CTAs of the per-stream kernels (the same code), taken in list order
 * by persistent CTAs; the other form (ocq_batch_set_mode) holds the streams'
 * plain kernels as concurrent branches.  Either way results are identical to
 * ocq_build_model + ocq_classify per stream.
 *   train: device, N*H*W*3; test: device, F*H*W*3; mask: device, F*H*W.
 * Domain per stream: 1 <= T <= N <= 255; depth <= 5 for block and pixel
 * regions (<= 8 for whole-frame); the buffers stay owned by the caller and
 * must stay valid while the batch exists (their addresses are baked in).
 */
typedef struct {
  const uint8_t *train;
  int N, H, W;
  ocq_region region;
  int depth, T;
  const uint8_t *test;
  int F;
  uint8_t *mask;
} ocq_stream_desc;

typedef struct ocq_batch ocq_batch;

/* Plans the work list, allocates the models (one arena) and scratch.  The
 * first ocq_batch_run captures the graph. */
ocq_status ocq_batch_create(const ocq_stream_desc *streams, int n, void *stream, ocq_batch **out);
/* Builds every stream's model and classifies every test frame (graph replay). */
ocq_status ocq_batch_run(ocq_batch *batch, void *stream);
/* Synchronises `stream`; OCQ_ETIMEOUT if an item gave up waiting for its model. */
ocq_status ocq_batch_status(ocq_batch *batch, void *stream);
/* Model of stream i: a view owned by the batch (never pass it to ocq_model_free). */
ocq_status ocq_batch_model(const ocq_batch *batch, int i, const ocq_model **out);
/* Classification work per item for a region kind, in 1024-pixel frame tiles
 * (units >= 1); re-plans the work list.  get_work also returns the number of
 * items in the list. */
ocq_status ocq_batch_set_work(ocq_batch *batch, int region_kind, int units);
ocq_status ocq_batch_get_work(const ocq_batch *batch, int region_kind, int *units, int64_t *items);
/* Form of the batch's graph:
 *   OCQ_BATCH_PERSISTENT  one persistent work-list kernel (the default);
 *   OCQ_BATCH_GRAPH       one branch per camera stream running that stream's
 *                         plain kernels (build, then classify); branches run
 *                         concurrently.
 *   OCQ_BATCH_GROUPED     one launch per kernel body (and depth, block size,
 *                         counter or list length) over all the streams that
 *                         use it, each launch with that body's own CTA shape,
 *                         shared memory and residency; the launches of one
 *                         class of streams (whole frame, blocks, pixels at
 *                         depth <= 3, pixels at depth 4-5) run in order on
 *                         one branch, the classes' branches concurrently;
 *                         streams outside those bodies run their plain kernels.
 * All give results identical to the per-stream calls.  Changing the form
 * drops the captured graph; the next run captures it again. */
enum { OCQ_BATCH_PERSISTENT = 0, OCQ_BATCH_GRAPH = 1, OCQ_BATCH_GROUPED = 2 };
ocq_status ocq_batch_set_mode(ocq_batch *batch, int mode);
int ocq_batch_get_mode(const ocq_batch *batch);
/* Persistent form: whether per-pixel streams of depth <= 3 classify from rows
 * staged in shared memory (on) or through L1 (off, the default).  Staging
 * speeds those streams up but raises every CTA's shared memory; the autotuner
 * times both.  Results are identical either way. */
ocq_status ocq_batch_set_staging(ocq_batch *batch, int on);
int ocq_batch_get_staging(const ocq_batch *batch);
/* Autotuner: times candidate work sizes per region kind on this batch's own
 * inputs (`reps` runs each, on `stream`) and keeps the fastest (results are
 * cached per (region kind, depths, sizes, frames) signature for the process),
 * then times the three forms and keeps the fastest. */
ocq_status ocq_batch_autotune(ocq_batch *batch, int reps, void *stream);
void ocq_batch_destroy(ocq_batch *batch);

/*
 * Served form.  The title of the paper's Sec. 4 names an update of the
 * octree without giving a procedure; this library's reading is a sliding window: the N training
 * frames build M_0; test frame t (t = 0, 1, ...) is classified against
 * M_floor(t/K); after classification it enters a ring of the last N frames;
 * when (t+1) % K == 0 the ring is merged again (Alg. 2) into the next model.
 * M_k therefore equals ocq_build_model over global frames [kK, kK + N - 1].
 * A camera's model and ring stay in HBM from admission to release.  Each
 * camera's work is ordered on its own CUDA stream and cameras run
 * concurrently: frames that arrive while others are on the GPU are enqueued
 * at once and their work overlaps.  Admission reserves the camera's
 * footprint (ocq_server_camera_footprint) against the server's HBM budget and
 * returns OCQ_EBUSY when slots or budget are exhausted; release returns them.
 * One thread submits for a given camera; different cameras may use
 * different threads.  Frame and mask buffers are the caller's (device) and
 * must stay valid until the frame's completion is polled.  The camera's work
 * runs on a stream of its own that does not wait on the caller's streams: a
 * training or test frame must already be complete on the device when it is
 * passed in (synchronise the stream that produced it first).
 */
typedef struct {
  int H, W;
  ocq_region region;
  int depth, T;
  int N; /* training frames = window length */
  int K; /* re-merge period in test frames */
} ocq_camera_desc;

typedef struct {
  int32_t camera;
  int32_t reserved;
  int64_t frame;    /* test frame index t of the camera */
  uint64_t tag;     /* caller's tag from ocq_server_submit */
  double arrival_s; /* host steady clock, seconds, at submit */
  double done_s;    /* host steady clock when the frame's mask (and any re-merge) was done */
} ocq_completion;

typedef struct ocq_server ocq_server;

/* hbm_budget: device bytes the server may hold; they are reserved (mapped in a
 * memory pool of the server's own) at creation, so admission and serving never
 * wait on the allocator.  OCQ_ENOMEM if the device cannot provide them. */
ocq_status ocq_server_create(size_t hbm_budget, int max_cameras, ocq_server **out);
/* Device bytes a camera of this description reserves (0 if invalid): the model
 * in the form ocq_build_model gives the description at admission (for
 * per-pixel regions of depth 4-5 with floor(N/T) <= 8 a list model, 16 B per
 * location; see OCQ_TUNE_PIXEL_MODEL_FORM), build scratch, and the window:
 *   - whole frame, when a leaf bitset (max(1, 8^d/32) u32 words) is no larger
 *     than a frame: N leaf bitsets, N bitsets of entering frames and 8^d u16
 *     counts (frames holding each leaf); a re-merge thresholds the counts in
 *     place;
 *   - pixel regions, and blocks with b <= 16, at depth <= 5 and N <= 255: N
 *     planes of per-pixel u16 leaf codes (2 bytes per pixel and frame); a
 *     re-merge counts the codes into the model in place;
 *   - otherwise the N frames themselves and a second model (the one being
 *     rebuilt from them by ocq_build_model).
 * The window keeps what the update of the model needs of the last N frames
 * (the paper's Sec. 4 names the update but gives no procedure). */
size_t ocq_server_camera_footprint(const ocq_camera_desc *desc);
/* Bytes of a camera's window image (what ocq_server_snapshot writes to
 * ring_out, oldest frame first): N * (leaf-bitset bytes, 2*H*W, or 3*H*W)
 * in the form ocq_server_camera_footprint describes; never more than N*H*W*3.
 * 0 if the description is invalid. */
size_t ocq_server_window_bytes(const ocq_camera_desc *desc);
/* train: device, N*H*W*3 (the window is filled from it and M_0 built from
 * it; read on the device after the call returns, so keep it until the
 * camera's first mask is done). */
ocq_status ocq_server_admit(ocq_server *server, const ocq_camera_desc *desc, const uint8_t *train, int *camera);
/* frame: device, H*W*3; mask: device, H*W (1 = foreground).  Non-blocking.
 * The same as ocq_server_submit_many with one frame. */
ocq_status ocq_server_submit(ocq_server *server, int camera, const uint8_t *frame, uint8_t *mask, uint64_t tag);
/* Continuous batching: n frames (entry i: camera cameras[i], device frame
 * frames[i] and mask masks[i], tag tags[i]; a camera's frames in arrival
 * order) submitted at once.  Frames of cameras with a bitset or code window
 * (ocq_server_camera_footprint) run in ticks on the server's high-priority
 * stream: a tick holds, for every camera, its next frames up to its next
 * re-merge (at most N), classifies all of them with one grouped launch per
 * kernel body (every camera's frames together), records their completion when
 * the masks are written, enters them into their windows and re-merges the
 * cameras whose window period ends; the next tick follows.  Frames of the
 * other cameras run one by one on their cameras' streams.  Every mask is the
 * one the window semantics give, whatever the grouping.  Non-blocking. */
ocq_status ocq_server_submit_many(ocq_server *server, int n, const int *cameras, const uint8_t *const *frames,
                                  uint8_t *const *masks, const uint64_t *tags);
/* Batching of the ticks.  A tick classifies all of a camera's frames in it
 * against one read of the camera's model (a per-pixel model row is 16-64 B per
 * pixel against a frame's 3 B), so larger ticks move fewer bytes per frame.
 * Frames of cameras served in ticks wait on the host
 *   - until the oldest of them has waited `seconds` (0, the default: no wait),
 *   - and while `ticks_in_flight` ticks are enqueued and unfinished (0: no
 *     limit; the default 2 lets one tick run while the next is queued, so that
 *     under load the frames that arrive meanwhile form one larger tick);
 * both are checked at every submit and poll (release, snapshot and sync run
 * held frames at once), so a caller polls regularly.  seconds in [0, 1].  No
 * counterpart in the paper. */
ocq_status ocq_server_set_batching(ocq_server *server, double seconds, int ticks_in_flight);
/* Up to max completed frames, oldest first; *n receives the count (runs the
 * held frames whose batching window ended). */
ocq_status ocq_server_poll(ocq_server *server, ocq_completion *out, int max, int *n);
/* Waits for the camera's frames, frees its window and model, returns its budget. */
ocq_status ocq_server_release(ocq_server *server, int camera);
/* Checkpoint of a camera's serving state, enqueued after its submitted work:
 * the current model in the exported layout (model_words: device, `words` >=
 * regions * words_per_region u64), the window image oldest frame first
 * (ring_out: device, at least ocq_server_window_bytes(desc) bytes; N*H*W*3
 * always suffices; layout internal to this library) and the number of test
 * frames submitted.
 * `stream` waits for the copies; read the buffers after it.  No counterpart
 * in the paper. */
ocq_status ocq_server_snapshot(ocq_server *server, int camera, uint64_t *model_words, size_t words,
                               uint8_t *ring_out, int64_t *submitted, void *stream);
/* Admits a camera from a snapshot (same description, model words, ring and
 * count): its next frame is test frame `submitted` and its re-merges happen
 * exactly as if it had not stopped.  Reserves the footprint like admit
 * (OCQ_EBUSY when it does not fit); the inputs must be complete on the device. */
ocq_status ocq_server_resume(ocq_server *server, const ocq_camera_desc *desc, const uint64_t *model_words,
                             const uint8_t *ring, int64_t submitted, int *camera);
/* The camera's current model (owned by the server; valid until the next re-merge or release). */
ocq_status ocq_server_camera_model(const ocq_server *server, int camera, const ocq_model **out);
ocq_status ocq_server_usage(ocq_server *server, size_t *used, size_t *budget, int64_t *completed);
/* Waits for every live camera's enqueued work. */
ocq_status ocq_server_sync(ocq_server *server);
void ocq_server_destroy(ocq_server *server);

/*
 * Tuning interface (no counterpart in the paper; it selects between kernel
 * variants that compute identical results).  `kernel` names a tunable kernel:
 *   OCQ_TUNE_CLASSIFY_PIXEL  per-pixel classify, depth <= 3; params =
 *                            {warps per CTA, pixels per thread, stages, frames per stage,
 *                             1 if a dedicated copy warp feeds the stages}
 *   OCQ_TUNE_BUILD_PIXEL     per-pixel build, depth <= 3; params =
 *                            {pixels (threads) per CTA, frames per stage, stages,
 *                             kind: 0 saturating counters, row copies; 1 the same with
 *                             one 2-D tensor copy per stage; 2 byte counters bumped
 *                             by shared-memory reductions; 3 saturating counters fed by
 *                             direct loads, frames per stage = frames prefetched;
 *                             4 as 2 with a dedicated copy warp; 5 as 4 with one 2-D
 *                             tensor copy per stage; 6 as 4 setting kept bits as
 *                             counts reach T; 7 as 5 and 6 together; 8 frequent-leaf
 *                             candidates per pixel counted in registers, no shared
 *                             counters (N <= 255, else as variant 0)}
 *   OCQ_TUNE_CLASSIFY_PIXEL_DEEP per-pixel classify, depth >= 4 (a warp walks
 *                            all frames of its pixel locations); params =
 *                            {pixel locations per lane (1 or 4), frames prefetched,
 *                             CTAs of 4 warps resident per SM, 0, 0}
 *   OCQ_TUNE_CLASSIFY_BLOCK_DEEP block classify with b % 4 == 0; params =
 *                            {form: 0 the strip's rows staged in shared memory
 *                             (b % 8 == 0, W % 16 == 0, depth <= 5), 1 L1-cached
 *                             lookups by warps walking all frames at depth >= 4,
 *                             2 the same at depth >= 3, 0, 0, 0}
 *   OCQ_TUNE_CLASSIFY_PIXEL_LIST per-pixel classify at depth 4-5 for models built
 *                            by the candidate build, which also keeps each location's
 *                            kept leaves as a list (16 B per location); variant 0
 *                            looks up the row, 1 compares with the list (one warp
 *                            per 128 locations walking all frames), 2 and up compare
 *                            with the list in the warp-specialised bulk-copy form
 *                            (frames and mask 16-byte aligned, H*W % 16 == 0; else
 *                            variant 1 runs); params = {warps, locations per thread,
 *                            stages, frames per stage, 0} (zeros for 0 and 1); a list
 *                            model (below) has no rows, so variant 0 acts as 1 there
 *   OCQ_TUNE_PIXEL_MODEL_FORM  what ocq_build_model / ocq_build_model_groups build for
 *                            per-pixel regions of depth 4-5 with N <= 255 and
 *                            floor(N / T) <= 8 (no location can keep more than 8
 *                            leaves): 1 (default) a list model, the kept leaves of
 *                            each location as a 16 B list and no leaf bitset (export
 *                            expands it into the bitset layout); 0 the bitset rows
 *                            plus that list; params = {variant, 0, ...}
 *   OCQ_TUNE_BUILD_BLOCK     block build with b <= 16 and N <= 255.  Forms for b
 *                            in {8, 16}, depth 2-5, W % 8 == 0 and 8-byte aligned
 *                            frames: warps over 16 x 16 pixel tiles (four 8 x 8 or
 *                            one 16 x 16 region, 8 pixels per lane; direct leaf
 *                            tables at depth <= 3, two-level prefix tables
 *                            deeper); the N frames split over the 8 warps of a CTA
 *                            (shared u8 counters per region, a leaf bitset per
 *                            warp for the frame it counts); for 8 x 8 at depth 5
 *                            one region per warp with two-level prefix tables;
 *                            every other block build runs one warp per region
 *                            with a hashed leaf table.  1 (default) picks by
 *                            shape and size: the region tables for 8 x 8 at depth
 *                            5 (frames split below 1024 tiles); frames split for
 *                            16 x 16 at depth 5, 8 x 8 at depth 4 and any frame of
 *                            fewer than 1024 tiles; tiles for depth <= 3 and
 *                            16 x 16 at depth 4; inside the batched forms tiles
 *                            and region tables only.  0 one warp per region
 *                            always; 2 frames split wherever they apply; 3 tiles
 *                            wherever they apply (8 x 8 at depth 5: one warp per
 *                            region); 4 the region tables for 8 x 8 at depth 4
 *                            or 5 (else one warp per region); params =
 *                            {variant, 0, ...}
 * ocq_tune_count: number of variants (-1 for an unknown kernel).
 * ocq_tune_select: process-wide choice used by later calls (not thread-safe
 * against concurrent calls of the same kernel).  ocq_tune_describe writes 5
 * int32 parameters (n >= 5).
 */
enum {
  OCQ_TUNE_CLASSIFY_PIXEL = 0,
  OCQ_TUNE_BUILD_PIXEL = 1,
  OCQ_TUNE_CLASSIFY_PIXEL_DEEP = 2,
  OCQ_TUNE_CLASSIFY_BLOCK_DEEP = 3,
  OCQ_TUNE_CLASSIFY_PIXEL_LIST = 4,
  OCQ_TUNE_PIXEL_MODEL_FORM = 5,
  OCQ_TUNE_BUILD_BLOCK = 6
};
int ocq_tune_count(int kernel);
int ocq_tune_selected(int kernel);
ocq_status ocq_tune_select(int kernel, int variant);
ocq_status ocq_tune_describe(int kernel, int variant, int32_t *params, int n);

/*
 * Test hooks (no counterpart in the paper).  They make failures happen on the
 * host side so that the error paths can be tested without faulting a GPU.
 *   ocq_debug_fail_allocations: the next `count` device allocations the library
 *     makes fail as if the device were out of memory (the call returns
 *     OCQ_ENOMEM after releasing what it had allocated); 0 clears.
 *   ocq_debug_async_bytes_in_use: bytes currently allocated from the current
 *     device's default stream-ordered pool (to check for leaks).
 *   ocq_batch_debug_hold_builds: leaves stream `stream`'s build items out of
 *     the persistent work list (-1 restores them); its classify items then wait
 *     for a model that never comes, give up after the bounded wait (1 s) and
 *     ocq_batch_status reports OCQ_ETIMEOUT; the GPU context stays usable.
 */
void ocq_debug_fail_allocations(int count);
ocq_status ocq_debug_async_bytes_in_use(size_t *bytes);
ocq_status ocq_batch_debug_hold_builds(ocq_batch *batch, int stream);

/*
 * Whole-frame build (as ocq_build_model with OCQ_REGION_FRAME) that allocates
 * no memory.  The paper has no counterpart; it serves callers that cannot
 * allocate device memory at call time -- pipelines that reserve every buffer
 * at start-up and must not block on the allocator, or hosts that give the
 * library a fixed memory budget.
 *   frames: device, N*H*W*3 bytes.  model: device, max(1, 8^depth/64) u64
 *   words, written in the exported layout (path code c at bit c%64 of word
 *   c/64) -- the row ocq_model_export writes for a whole-frame model.
 * Scratch is one static 16 MiB device array inside the library, present on
 * every GPU that loads it until the process exits; requests needing more
 * (depth d and N with (bit_length(N) + 2) * max(1, 8^d/32) * 4 bytes above
 * 16 MiB) return OCQ_EINVAL with a message.  It calls no cudaMalloc/cudaFree.
 * The first call on a device resolves the array's device address (with that
 * device current) and keeps it for the life of the process; make that first
 * call before any stream capture, and do not call the entry point on a device
 * after its primary context was reset (cudaDeviceReset), since the kept
 * address is then stale.  All calls on one device share that device's array
 * and each clears what it needs: calls on the same device whose work may
 * overlap (different streams or host threads) race and must be ordered by
 * the caller; calls on different devices use separate arrays.
 */
ocq_status ocq_build_frame_noalloc(const uint8_t *frames, int N, int H, int W, int depth, int T, uint64_t *model,
                                   void *stream);

/* Number of kernels this library has launched in this process (all devices).
 * Lets a caller count the device work a call sequence issued. */
uint64_t ocq_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* OCQ_H */
