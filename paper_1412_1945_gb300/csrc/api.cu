// C-ABI entry points: argument validation, model ownership, dispatch.
// The compute lives in build.cu, classify.cu and transform.cu.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "ocq_internal.cuh"

namespace ocq {

static thread_local char g_err[512];
static std::atomic<uint64_t> g_launches{0};

void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// Stream-ordered allocation from the memory pool the calling thread has
// selected (a server's own pool, see PoolScope), else the device's default.
static thread_local cudaMemPool_t t_pool = nullptr;
static std::atomic<int> g_fail_allocs{0};  // test hook: allocations still to refuse
cudaError_t malloc_async(void **p, size_t bytes, cudaStream_t st) {
  int n = g_fail_allocs.load();
  while (n > 0)
    if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return cudaErrorMemoryAllocation;
  return t_pool ? cudaMallocFromPoolAsync(p, bytes, t_pool, st) : cudaMallocAsync(p, bytes, st);
}
PoolScope::PoolScope(cudaMemPool_t pool) : prev_(t_pool) { t_pool = pool; }
PoolScope::~PoolScope() { t_pool = prev_; }

void clear_error() { g_err[0] = 0; }

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

ocq_status cuda_status(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return OCQ_OK;
  set_error("%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return OCQ_ENOMEM;
  return OCQ_ECUDA;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

int64_t region_count(int H, int W, int kind, int block) {
  if (H < 1 || W < 1) return -1;
  if (kind == OCQ_REGION_FRAME) return 1;
  if (kind == OCQ_REGION_BLOCK) {
    if (block < 1) return -1;
    return (int64_t)((H + block - 1) / block) * ((W + block - 1) / block);
  }
  if (kind == OCQ_REGION_PIXEL) return (int64_t)H * W;
  return -1;
}

static const int64_t kMaxPixels = (int64_t)1 << 40;

static ocq_status check_geometry(int H, int W, ocq_region region, int depth) {
  if (H < 1 || W < 1) {
    set_error("H and W must be >= 1 (got %d x %d)", H, W);
    return OCQ_EINVAL;
  }
  if (depth < 1 || depth > 8) {
    set_error("depth must be in [1, 8] (got %d)", depth);
    return OCQ_EINVAL;
  }
  if (region_count(H, W, region.kind, region.block) < 1) {
    set_error("invalid region (kind %d, block %d)", region.kind, region.block);
    return OCQ_EINVAL;
  }
  return OCQ_OK;
}

// rows = false: a list model (kept-leaf index only), allocated by its build.
static ocq_model *new_model(int H, int W, ocq_region region, int depth, int T, int N, cudaStream_t st,
                            ocq_status *rc, bool rows = true) {
  ocq_model *m = new (std::nothrow) ocq_model();
  if (!m) {
    set_error("host allocation failed");
    *rc = OCQ_ENOMEM;
    return nullptr;
  }
  m->H = H, m->W = W, m->kind = region.kind, m->block = region.kind == OCQ_REGION_BLOCK ? region.block : 0;
  m->depth = depth, m->T = T, m->N = N;
  m->R = region_count(H, W, region.kind, region.block);
  m->wpr = wpr32(depth);
  m->bytes = rows ? (size_t)m->R * (size_t)m->wpr * sizeof(uint32_t) : 0;
  m->stream = st;
  cudaGetDevice(&m->device);
  if (!rows) return m;
  void *p = nullptr;
  *rc = cuda_status(malloc_async(&p, m->bytes, st), "allocating the model");
  if (*rc != OCQ_OK) {
    delete m;
    return nullptr;
  }
  m->bits = (uint32_t *)p;
  return m;
}

size_t model_bytes(int H, int W, ocq_region region, int depth, int N, int T) {
  const size_t rows = (size_t)region_count(H, W, region.kind, region.block) * (size_t)wpr32(depth) * sizeof(uint32_t);
  const size_t index = (size_t)H * W * 8 * sizeof(uint16_t);
  if (list_model_applies(region.kind, depth, N, T)) return index;
  const bool indexed = region.kind == OCQ_REGION_PIXEL && (depth == 4 || depth == 5) && N <= 255 && T >= 1 &&
                       N / T <= 8;
  return rows + (indexed ? index : 0);
}

}  // namespace ocq

using namespace ocq;

extern "C" {

const char *ocq_status_str(ocq_status s) {
  switch (s) {
    case OCQ_OK: return "OCQ_OK";
    case OCQ_EINVAL: return "OCQ_EINVAL";
    case OCQ_ENOMEM: return "OCQ_ENOMEM";
    case OCQ_ECUDA: return "OCQ_ECUDA";
    case OCQ_ETIMEOUT: return "OCQ_ETIMEOUT";
    case OCQ_EBUSY: return "OCQ_EBUSY";
    case OCQ_ENOTSUP: return "OCQ_ENOTSUP";
  }
  return "OCQ_UNKNOWN";
}

const char *ocq_last_error(void) { return g_err; }

uint64_t ocq_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char *ocq_version(void) { return "ocq 0.1 (sm_103a)"; }

int64_t ocq_region_count(int H, int W, ocq_region region) { return region_count(H, W, region.kind, region.block); }

size_t ocq_model_footprint(int H, int W, ocq_region region, int depth) {
  if (check_geometry(H, W, region, depth) != OCQ_OK) return 0;
  const size_t bits = (size_t)region_count(H, W, region.kind, region.block) * (size_t)wpr32(depth) * sizeof(uint32_t);
  const bool indexed = region.kind == OCQ_REGION_PIXEL && (depth == 4 || depth == 5);
  return bits + (indexed ? (size_t)H * W * 8 * sizeof(uint16_t) : 0);
}

ocq_status ocq_path_code(const uint8_t *rgb, int64_t npix, int depth, uint32_t *codes, void *stream) {
  g_err[0] = 0;
  if (npix < 0 || npix >= kMaxPixels || depth < 1 || depth > 8 || (npix > 0 && (!rgb || !codes))) {
    set_error("ocq_path_code: bad arguments");
    return OCQ_EINVAL;
  }
  if (npix == 0) return OCQ_OK;
  return launch_path_code(rgb, npix, depth, codes, (cudaStream_t)stream);
}

ocq_status ocq_occupancy(const uint8_t *frames, int n, int H, int W, ocq_region region, int depth, uint64_t *occ,
                         void *stream) {
  g_err[0] = 0;
  ocq_status rc = check_geometry(H, W, region, depth);
  if (rc != OCQ_OK) return rc;
  if (n < 0 || (n > 0 && (!frames || !occ)) || (int64_t)n * H * W >= kMaxPixels) {
    set_error("ocq_occupancy: bad frame count or pointers");
    return OCQ_EINVAL;
  }
  if (n == 0) return OCQ_OK;
  return launch_occupancy(frames, n, H, W, region.kind, region.kind == OCQ_REGION_BLOCK ? region.block : 0, depth,
                          occ, (cudaStream_t)stream);
}

ocq_status ocq_build_model(const uint8_t *frames, int N, int H, int W, ocq_region region, int depth, int T,
                           void *stream, ocq_model **out) {
  g_err[0] = 0;
  if (!out) {
    set_error("ocq_build_model: out is NULL");
    return OCQ_EINVAL;
  }
  *out = nullptr;
  ocq_status rc = check_geometry(H, W, region, depth);
  if (rc != OCQ_OK) return rc;
  if (!frames || N < 1 || N > 65535 || T < 1 || T > N || (int64_t)N * H * W >= kMaxPixels) {
    set_error("ocq_build_model: need frames != NULL and 1 <= T <= N <= 65535 (N=%d, T=%d)", N, T);
    return OCQ_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  ocq_model *m = new_model(H, W, region, depth, T, N, st, &rc, !list_model_applies(region.kind, depth, N, T));
  if (!m) return rc;
  rc = launch_build(frames, N, m, st);
  if (rc != OCQ_OK) {
    ocq_model_free(m);
    return rc;
  }
  *out = m;
  return OCQ_OK;
}

ocq_status ocq_merge_occupancy(const uint64_t *occ, int parts, int N, int H, int W, ocq_region region, int depth,
                               int T, void *stream, ocq_model **out) {
  g_err[0] = 0;
  if (!out) {
    set_error("ocq_merge_occupancy: out is NULL");
    return OCQ_EINVAL;
  }
  *out = nullptr;
  ocq_status rc = check_geometry(H, W, region, depth);
  if (rc != OCQ_OK) return rc;
  if (!occ || parts < 1 || N < 1 || N > 65535 || T < 1 || T > N) {
    set_error("ocq_merge_occupancy: need occ != NULL, parts >= 1 and 1 <= T <= N <= 65535 (parts=%d, N=%d, T=%d)",
              parts, N, T);
    return OCQ_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  ocq_model *m = new_model(H, W, region, depth, T, N, st, &rc, true);
  if (!m) return rc;
  const int64_t rows = (int64_t)N * m->R;
  const int64_t w64 = rows * wpr64(depth), w32 = rows * m->wpr;
  uint64_t *un = nullptr;
  uint32_t *planar = nullptr;
  if (parts > 1) rc = cuda_status(malloc_async((void **)&un, (size_t)w64 * 8, st), "merge scratch");
  if (rc == OCQ_OK) rc = cuda_status(malloc_async((void **)&planar, (size_t)w32 * 4, st), "merge scratch");
  if (rc == OCQ_OK && parts > 1) rc = launch_or_parts(occ, parts, w64, un, st);
  if (rc == OCQ_OK) rc = launch_import(parts > 1 ? un : occ, rows, depth, planar, st);
  if (rc == OCQ_OK) rc = launch_merge_counts(planar, N, m->R * m->wpr, (uint32_t)T, m->bits, st);
  if (un) cudaFreeAsync(un, st);
  if (planar) cudaFreeAsync(planar, st);
  if (rc != OCQ_OK) {
    ocq_model_free(m);
    return rc;
  }
  *out = m;
  return OCQ_OK;
}

ocq_status ocq_build_model_groups(const uint8_t *frames, int N, int H, int W, ocq_region region, int depth, int T,
                                  int group, void *stream, ocq_model **out) {
  g_err[0] = 0;
  if (!out) {
    set_error("ocq_build_model_groups: out is NULL");
    return OCQ_EINVAL;
  }
  *out = nullptr;
  ocq_status rc = check_geometry(H, W, region, depth);
  if (rc != OCQ_OK) return rc;
  const int G = group >= 1 ? (N + group - 1) / group : 0;
  if (!frames || N < 1 || N > 65535 || group < 1 || T < 1 || T > G || (int64_t)N * H * W >= kMaxPixels) {
    set_error("ocq_build_model_groups: need frames != NULL, 1 <= N <= 65535, group >= 1 and "
              "1 <= T <= ceil(N / group) (N=%d, group=%d, T=%d)", N, group, T);
    return OCQ_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  ocq_model *m = new_model(H, W, region, depth, T, N, st, &rc, !list_model_applies(region.kind, depth, N, T));
  if (!m) return rc;
  rc = launch_build_groups(frames, N, group, m, st);
  if (rc != OCQ_OK) {
    ocq_model_free(m);
    return rc;
  }
  *out = m;
  return OCQ_OK;
}

ocq_status ocq_classify(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask, void *stream) {
  g_err[0] = 0;
  if (!m || F < 0 || (F > 0 && (!frames || !mask)) || (int64_t)F * m->H * m->W >= kMaxPixels) {
    set_error("ocq_classify: bad arguments");
    return OCQ_EINVAL;
  }
  if (F == 0) return OCQ_OK;
  return launch_classify(m, frames, F, mask, (cudaStream_t)stream);
}

ocq_status ocq_model_get_info(const ocq_model *m, ocq_model_info *info) {
  g_err[0] = 0;
  if (!m || !info) {
    set_error("ocq_model_get_info: NULL argument");
    return OCQ_EINVAL;
  }
  memset(info, 0, sizeof *info);
  info->H = m->H, info->W = m->W, info->region_kind = m->kind, info->block = m->block;
  info->depth = m->depth, info->T = m->T, info->N = m->N;
  info->regions = m->R;
  info->words_per_region = wpr64(m->depth);
  return OCQ_OK;
}

ocq_status ocq_model_export(const ocq_model *m, uint64_t *dst, size_t words, void *stream) {
  g_err[0] = 0;
  if (!m || !dst || words < (size_t)m->R * (size_t)wpr64(m->depth)) {
    set_error("ocq_model_export: NULL argument or destination too small");
    return OCQ_EINVAL;
  }
  if (!m->bits) return launch_export_list(m->kept, m->R, m->depth, dst, (cudaStream_t)stream);
  return launch_export(m->bits, m->R, m->depth, dst, (cudaStream_t)stream);
}

ocq_status ocq_model_import(const uint64_t *src, const ocq_model_info *info, void *stream, ocq_model **out) {
  g_err[0] = 0;
  if (!out || !src || !info) {
    set_error("ocq_model_import: NULL argument");
    return OCQ_EINVAL;
  }
  *out = nullptr;
  ocq_region region = {info->region_kind, info->block};
  ocq_status rc = check_geometry(info->H, info->W, region, info->depth);
  if (rc != OCQ_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const bool list = list_model_applies(region.kind, info->depth, info->N, info->T);
  ocq_model *m = new_model(info->H, info->W, region, info->depth, info->T, info->N, st, &rc, !list);
  if (!m) return rc;
  if (list) {  // the form ocq_build_model gives this description: the kept leaves as lists
    unsigned int *flag = nullptr, overflow = 0;
    rc = cuda_status(malloc_async((void **)&m->kept, (size_t)m->R * 8 * sizeof(uint16_t), st), "kept-leaf index");
    if (rc == OCQ_OK) rc = cuda_status(malloc_async((void **)&flag, sizeof *flag, st), "import flag");
    if (rc == OCQ_OK) rc = cuda_status(cudaMemsetAsync(flag, 0, sizeof *flag, st), "import flag");
    if (rc == OCQ_OK) rc = launch_import_list(src, m->R, m->depth, info->N / info->T, m->kept, flag, st);
    if (rc == OCQ_OK) rc = cuda_status(cudaMemcpyAsync(&overflow, flag, sizeof overflow, cudaMemcpyDeviceToHost, st),
                                       "import flag");
    if (flag) cudaFreeAsync(flag, st);
    if (rc == OCQ_OK) rc = cuda_status(cudaStreamSynchronize(st), "import");
    if (rc == OCQ_OK && overflow) {
      set_error("ocq_model_import: a pixel location holds more than floor(N/T) = %d leaves", info->N / info->T);
      rc = OCQ_EINVAL;
    }
    m->kept_len = list_length(info->N, info->T);
  } else {
    rc = launch_import(src, m->R, m->depth, m->bits, st);
  }
  if (rc != OCQ_OK) {
    ocq_model_free(m);
    return rc;
  }
  *out = m;
  return OCQ_OK;
}

void ocq_model_free(ocq_model *m) {
  if (!m) return;
  if (m->bits) cudaFreeAsync(m->bits, m->stream);
  if (m->kept) cudaFreeAsync(m->kept, m->stream);
  delete m;
}

/* Synchronises `stream` and reports (then clears) a bounded-wait timeout
 * recorded by a kernel on the current device: OCQ_ETIMEOUT if one occurred. */
ocq_status ocq_device_status(void *stream) {
  g_err[0] = 0;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_status(e, "stream synchronise");
  const bool c = classify_take_timeout();
  const bool b = build_take_timeout();
  if (c || b) {
    set_error("a bounded device wait timed out (%s)", c ? "classify" : "build");
    return OCQ_ETIMEOUT;
  }
  return OCQ_OK;
}

int ocq_tune_count(int kernel) {
  if (kernel == OCQ_TUNE_CLASSIFY_PIXEL) return classify_variant_count();
  if (kernel == OCQ_TUNE_BUILD_PIXEL) return build_variant_count();
  if (kernel == OCQ_TUNE_CLASSIFY_PIXEL_DEEP) return deep_variant_count();
  if (kernel == OCQ_TUNE_CLASSIFY_BLOCK_DEEP) return block_form_count();
  if (kernel == OCQ_TUNE_CLASSIFY_PIXEL_LIST) return list_form_count();
  if (kernel == OCQ_TUNE_PIXEL_MODEL_FORM) return 2;
  if (kernel == OCQ_TUNE_BUILD_BLOCK) return block_build_form_count();
  return -1;
}

int ocq_tune_selected(int kernel) {
  if (kernel == OCQ_TUNE_CLASSIFY_PIXEL) return classify_variant_selected();
  if (kernel == OCQ_TUNE_BUILD_PIXEL) return build_variant_selected();
  if (kernel == OCQ_TUNE_CLASSIFY_PIXEL_DEEP) return deep_variant_selected();
  if (kernel == OCQ_TUNE_CLASSIFY_BLOCK_DEEP) return block_form_selected();
  if (kernel == OCQ_TUNE_CLASSIFY_PIXEL_LIST) return list_form_selected();
  if (kernel == OCQ_TUNE_PIXEL_MODEL_FORM) return list_model_form();
  if (kernel == OCQ_TUNE_BUILD_BLOCK) return block_build_form_selected();
  return -1;
}

ocq_status ocq_tune_select(int kernel, int variant) {
  g_err[0] = 0;
  bool ok = false;
  if (kernel == OCQ_TUNE_CLASSIFY_PIXEL) ok = classify_variant_select(variant);
  if (kernel == OCQ_TUNE_BUILD_PIXEL) ok = build_variant_select(variant);
  if (kernel == OCQ_TUNE_CLASSIFY_PIXEL_DEEP) ok = deep_variant_select(variant);
  if (kernel == OCQ_TUNE_CLASSIFY_BLOCK_DEEP) ok = block_form_select(variant);
  if (kernel == OCQ_TUNE_CLASSIFY_PIXEL_LIST) ok = list_form_select(variant);
  if (kernel == OCQ_TUNE_PIXEL_MODEL_FORM) ok = list_model_select(variant);
  if (kernel == OCQ_TUNE_BUILD_BLOCK) ok = block_build_form_select(variant);
  if (!ok) {
    set_error("ocq_tune_select: no variant %d of kernel %d", variant, kernel);
    return OCQ_EINVAL;
  }
  return OCQ_OK;
}

void ocq_debug_fail_allocations(int count) { g_fail_allocs.store(count > 0 ? count : 0); }

ocq_status ocq_debug_async_bytes_in_use(size_t *bytes) {
  if (!bytes) return OCQ_EINVAL;
  int dev = 0;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&pool, dev);
  uint64_t used = 0;
  if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
  *bytes = (size_t)used;
  return cuda_status(e, "default pool usage");
}

ocq_status ocq_tune_describe(int kernel, int variant, int32_t *params, int n) {
  g_err[0] = 0;
  if (!params || n < 5 || variant < 0 || variant >= ocq_tune_count(kernel)) {
    set_error("ocq_tune_describe: bad arguments");
    return OCQ_EINVAL;
  }
  params[0] = params[1] = params[2] = params[3] = params[4] = 0;
  if (kernel == OCQ_TUNE_CLASSIFY_PIXEL)
    classify_variant_describe(variant, &params[0], &params[1], &params[2], &params[3], &params[4]);
  else if (kernel == OCQ_TUNE_BUILD_PIXEL)
    build_variant_describe(variant, &params[0], &params[1], &params[2], &params[3]);
  else if (kernel == OCQ_TUNE_CLASSIFY_PIXEL_DEEP)
    deep_variant_describe(variant, &params[0], &params[1], &params[2]);
  else if (kernel == OCQ_TUNE_CLASSIFY_PIXEL_LIST)
    list_form_describe(variant, &params[0], &params[1], &params[2], &params[3]);
  else
    params[0] = variant;
  return OCQ_OK;
}

}  // extern "C"
