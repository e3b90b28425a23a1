// Batched form: many camera streams of uneven size, depth and region kind are
// built (S1-S3, Sec. 3, Alg. 1-2) and classified (S4, Alg. 3) in ONE
// persistent kernel launch, replayed from a CUDA graph.
//
// The host turns the streams into a work list of items; persistent CTAs take
// items in list order from an atomic counter.  Item kinds:
//   OCC      whole-frame stream: leaf bitset of one frame's pixel chunk
//   MERGE    whole-frame stream: bit-sliced count of the frames' bitsets -> model words
//   BLOCK    block-region stream: one block's model row (per-frame bitset, listed words,
//            bit-sliced counters in shared memory)
//   PIXEL    pixel-region stream: 128 pixel locations' rows (byte counters in shared memory)
//   CLASSIFY any stream: a tile of pixels x a run of test frames
// Dependencies are per stream: MERGE waits for the stream's OCC items, CLASSIFY
// for the stream's build items.  Every item a CTA waits on precedes it in the
// list, so it was taken by a running CTA and completes; each wait is still
// bounded (1 s) and records a timeout instead of spinning forever.
// Tile shapes of CLASSIFY items (pixels x frames) are chosen per region kind
// by the autotuner (ocq_batch_autotune), which times candidate work lists.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "async_copy.cuh"
#include "pixels.cuh"

namespace ocq {

enum : int32_t { IT_OCC = 0, IT_MERGE = 1, IT_BLOCK = 2, IT_PIXEL = 3, IT_CLASSIFY = 4 };

struct BStream {
  const uint8_t *train, *test;
  uint8_t *mask;
  uint32_t *model;  // R * wpr words, internal (planar) order
  uint32_t *occ;    // whole-frame streams: N * wpr words of scratch
  int64_t hw, R, wpr;
  int32_t N, F, H, W, kind, block, bw, depth, T, P;
  int32_t n_build;  // items that complete the model (MERGE, BLOCK or PIXEL)
  int32_t n_occ;    // OCC items (whole-frame streams)
};

struct BItem {
  int32_t type, stream;
  int64_t a;     // first pixel / block / word
  int32_t c;     // pixels / words in the item
  int32_t f0;    // first frame
  int32_t nf;    // frames
  int32_t pad;
};

static constexpr int kBatchThreads = 128;

// Counter block: [0] next item, [1] timeout flag, [2..2+S) OCC done, [2+S..2+2S) build done.
__device__ __forceinline__ bool wait_count(const uint32_t *ctr, uint32_t want, uint32_t *err) {
  const volatile uint32_t *p = ctr;
  if (*p >= want) return true;
  if (*(volatile uint32_t *)err) return false;  // an earlier wait already failed: do not wait again
  const uint64_t t0 = global_ns();
  while (*p < want) {
    __nanosleep(256);
    if (global_ns() - t0 > kWaitLimitNs) {
      atomicExch(err, 1u);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ uint32_t planar_q(const uint8_t *px, int d) {
  return planar_code_rt(px[0], px[1], px[2], d);
}

// ---- items --------------------------------------------------------------------

__device__ void item_occ(const BStream &S, const BItem &it, uint32_t *sm) {
  const uint8_t *fr = S.train + ((int64_t)it.f0 * S.hw) * 3;
  uint32_t *dst = S.occ + (int64_t)it.f0 * S.wpr;
  if (S.wpr <= 8192) {
    for (int64_t i = threadIdx.x; i < S.wpr; i += blockDim.x) sm[i] = 0;
    __syncthreads();
    for (int64_t p = it.a + threadIdx.x; p < it.a + it.c; p += blockDim.x) {
      const uint32_t q = planar_q(fr + p * 3, S.depth);
      const uint32_t m = 1u << (q & 31);
      if (!(sm[q >> 5] & m)) atomicOr(&sm[q >> 5], m);
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < S.wpr; i += blockDim.x)
      if (sm[i]) atomicOr(&dst[i], sm[i]);
  } else {
    for (int64_t p = it.a + threadIdx.x; p < it.a + it.c; p += blockDim.x) {
      const uint32_t q = planar_q(fr + p * 3, S.depth);
      const uint32_t m = 1u << (q & 31);
      if (!(*(volatile uint32_t *)&dst[q >> 5] & m)) atomicOr(&dst[q >> 5], m);
    }
  }
}

__device__ void item_merge(const BStream &S, const BItem &it) {
  for (int64_t w = it.a + threadIdx.x; w < it.a + it.c; w += blockDim.x) {
    uint32_t pl[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) pl[k] = 0;
    for (int f = 0; f < S.N; ++f) {
      uint32_t x = *(volatile const uint32_t *)&S.occ[(int64_t)f * S.wpr + w];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (k < S.P) {
          const uint32_t t = pl[k] & x;
          pl[k] ^= x;
          x = t;
        }
      }
    }
    uint32_t gt = 0, eq = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 15; k >= 0; --k) {
      if (k < S.P) {
        const uint32_t c = pl[k];
        if (((uint32_t)S.T >> k) & 1u) {
          eq &= c;
        } else {
          gt |= eq & c;
          eq &= ~c;
        }
      }
    }
    S.model[w] = gt | eq;
  }
}

__device__ void item_block(const BStream &S, const BItem &it, uint32_t *sm, uint32_t *nlist) {
  const int64_t wpr = S.wpr;
  uint32_t *seen = sm, *planes = sm + wpr, *list = planes + (int64_t)S.P * wpr;
  for (int64_t i = threadIdx.x; i < wpr * (S.P + 1); i += blockDim.x) sm[i] = 0;
  if (threadIdx.x == 0) *nlist = 0;
  const int64_t r = it.a;
  const int b = S.block;
  const int y0 = (int)(r / S.bw) * b, x0 = (int)(r % S.bw) * b;
  const int h = min(b, S.H - y0), w = min(b, S.W - x0);
  const int npx = h * w;
  __syncthreads();
  for (int f = 0; f < S.N; ++f) {
    const uint8_t *fr = S.train + (int64_t)f * S.hw * 3;
    for (int i = threadIdx.x; i < npx; i += blockDim.x) {
      const int y = y0 + i / w, x = x0 + i % w;
      const uint32_t q = planar_q(fr + ((int64_t)y * S.W + x) * 3, S.depth);
      const uint32_t m = 1u << (q & 31);
      if (!(seen[q >> 5] & m)) {
        if (atomicOr(&seen[q >> 5], m) == 0) list[atomicAdd(nlist, 1u)] = q >> 5;
      }
    }
    __syncthreads();
    const uint32_t n = *nlist;
    for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
      const uint32_t wd = list[k];
      uint32_t x = seen[wd];
      for (int j = 0; j < S.P && x; ++j) {
        const uint32_t t = planes[j * wpr + wd] & x;
        planes[j * wpr + wd] ^= x;
        x = t;
      }
      seen[wd] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) *nlist = 0;
    __syncthreads();
  }
  for (int64_t wd = threadIdx.x; wd < wpr; wd += blockDim.x) {
    uint32_t gt = 0, eq = 0xFFFFFFFFu;
    for (int k = S.P - 1; k >= 0; --k) {
      const uint32_t c = planes[k * wpr + wd];
      if (((uint32_t)S.T >> k) & 1u) {
        eq &= c;
      } else {
        gt |= eq & c;
        eq &= ~c;
      }
    }
    S.model[r * wpr + wd] = gt | eq;
  }
}

// Per-pixel rows, 128 pixel locations per item, one per thread.  Byte
// counters (N <= 255, checked by the plan) for 512-leaf chunks in a private
// column cnt[k*128 + t]; depth <= 3 is one chunk, deeper rows count only the
// chunks the pixel's training colours touch.
__device__ void item_pixel(const BStream &S, const BItem &it, uint32_t *cnt) {
  const int t = threadIdx.x;
  const int64_t p = it.a + t;
  if (t >= it.c) return;
  const int d = S.depth;
  const uint32_t ncodes = 1u << (3 * d);
  const uint32_t chunk = ncodes < 512 ? ncodes : 512u;
  const int cwords = (int)((chunk + 3) / 4);
  const int nchunks = (int)(ncodes / chunk);
  const uint8_t *px = S.train + p * 3;
  const int64_t fstride = S.hw * 3;
  uint64_t touched = 0;
  if (nchunks > 1) {
    for (int f = 0; f < S.N; ++f) touched |= 1ull << (planar_q(px + f * fstride, d) >> 9);
  } else {
    touched = 1;
  }
  uint32_t *row = S.model + p * S.wpr;
  for (int c = 0; c < nchunks; ++c) {
    uint32_t *dst = row + (int64_t)c * (chunk >= 32 ? chunk / 32 : 1);
    const int ow = chunk >= 32 ? (int)(chunk / 32) : 1;
    if (!((touched >> c) & 1ull)) {
      for (int w = 0; w < ow; ++w) dst[w] = 0;
      continue;
    }
    for (int k = 0; k < cwords; ++k) cnt[k * kBatchThreads + t] = 0;
    for (int f = 0; f < S.N; ++f) {
      const uint32_t q = planar_q(px + f * fstride, d);
      if ((int)(q / chunk) != c) continue;
      const uint32_t l = q % chunk;
      cnt[(l >> 2) * kBatchThreads + t] += 1u << ((l & 3u) * 8);
    }
    for (int w = 0; w < ow; ++w) {
      uint32_t o = 0;
      for (int k = 0; k < 8 && w * 8 + k < cwords; ++k) {
        const uint32_t ge = __vcmpgeu4(cnt[(w * 8 + k) * kBatchThreads + t], (uint32_t)S.T * 0x01010101u);
        o |= (((ge >> 7) & 1u) | ((ge >> 14) & 2u) | ((ge >> 21) & 4u) | ((ge >> 28) & 8u)) << (4 * k);
      }
      if (chunk < 32) o &= (1u << chunk) - 1u;
      dst[w] = o;
    }
  }
}

// A tile of pixels x a run of test frames.  Whole-frame rows and per-pixel
// rows of depth <= 3 are staged in shared memory (word-major for pixel rows,
// so a warp's lookups fall in distinct banks); other rows are read from
// global memory.
__device__ void item_classify(const BStream &S, const BItem &it, uint32_t *sm) {
  const int d = S.depth;
  const int64_t pa = it.a, pc = it.c;
  const bool frame_row = S.kind == OCQ_REGION_FRAME && S.wpr <= 8192;
  const bool pixel_rows = S.kind == OCQ_REGION_PIXEL && d <= 3;
  if (frame_row) {
    for (int64_t i = threadIdx.x; i < S.wpr; i += blockDim.x) sm[i] = *(volatile const uint32_t *)&S.model[i];
  } else if (pixel_rows) {
    for (int64_t i = threadIdx.x; i < pc * S.wpr; i += blockDim.x) {
      const int64_t pl = i / S.wpr, w = i % S.wpr;
      sm[w * pc + pl] = *(volatile const uint32_t *)&S.model[(pa + pl) * S.wpr + w];
    }
  }
  __syncthreads();
  for (int f = it.f0; f < it.f0 + it.nf; ++f) {
    const uint8_t *fr = S.test + (int64_t)f * S.hw * 3;
    uint8_t *mk = S.mask + (int64_t)f * S.hw;
    for (int64_t i = threadIdx.x; i < pc; i += blockDim.x) {
      const int64_t p = pa + i;
      const uint32_t q = planar_q(fr + p * 3, d);
      uint32_t word;
      if (frame_row) {
        word = sm[q >> 5];
      } else if (pixel_rows) {
        word = sm[(q >> 5) * pc + i];
      } else {
        const int y = (int)(p / S.W), x = (int)(p % S.W);
        word = __ldcg(S.model + region_of(y, x, S.W, S.kind, S.block, S.bw) * S.wpr + (q >> 5));
      }
      mk[p] = (uint8_t)(((word >> (q & 31)) & 1u) ^ 1u);
    }
  }
}

__global__ void __launch_bounds__(kBatchThreads) batch_kernel(const BStream *__restrict__ streams,
                                                              const BItem *__restrict__ items, int n_items, int S,
                                                              uint32_t *ctr) {
  extern __shared__ uint32_t sm[];
  __shared__ int cur;
  __shared__ int ok;
  __shared__ uint32_t nlist;
  uint32_t *err = ctr + 1;
  uint32_t *occ_done = ctr + 2;
  uint32_t *build_done = ctr + 2 + S;
  while (true) {
    if (threadIdx.x == 0) cur = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    const int k = cur;
    if (k >= n_items) return;
    const BItem it = items[k];
    const BStream &st = streams[it.stream];
    if (threadIdx.x == 0) {
      ok = 1;
      if (it.type == IT_MERGE) ok = wait_count(&occ_done[it.stream], (uint32_t)st.n_occ, err);
      if (it.type == IT_CLASSIFY) ok = wait_count(&build_done[it.stream], (uint32_t)st.n_build, err);
      __threadfence();
    }
    __syncthreads();
    if (ok) {
      switch (it.type) {
        case IT_OCC: item_occ(st, it, sm); break;
        case IT_MERGE: item_merge(st, it); break;
        case IT_BLOCK: item_block(st, it, sm, &nlist); break;
        case IT_PIXEL: item_pixel(st, it, sm); break;
        default: item_classify(st, it, sm); break;
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && ok) {
      if (it.type == IT_OCC) atomicAdd(&occ_done[it.stream], 1u);
      if (it.type == IT_MERGE || it.type == IT_BLOCK || it.type == IT_PIXEL) atomicAdd(&build_done[it.stream], 1u);
    }
  }
}

}  // namespace ocq

using namespace ocq;

// ---- host plan ------------------------------------------------------------------

struct ocq_batch {
  std::vector<ocq_stream_desc> desc;
  std::vector<BStream> hs;
  std::vector<ocq_model *> models;  // views (bits point into the arena)
  std::vector<BItem> items;
  int tile_px[3] = {2048, 2048, 1024};  // CLASSIFY pixels per item, per region kind
  int tile_frames[3] = {16, 16, 32};    // CLASSIFY frames per item, per region kind
  BStream *d_streams = nullptr;
  BItem *d_items = nullptr;
  size_t items_cap = 0;
  uint32_t *d_ctr = nullptr;
  uint8_t *arena = nullptr;  // models + whole-frame scratch
  size_t arena_bytes = 0;
  size_t smem = 0;
  int grid = 0;
  cudaStream_t owner = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
};

static ocq_status plan_items(ocq_batch *b) {
  b->items.clear();
  const int S = (int)b->hs.size();
  std::vector<BStream> &hs = b->hs;
  auto push = [&](int32_t type, int s, int64_t a, int32_t c, int32_t f0, int32_t nf) {
    BItem it;
    it.type = type, it.stream = s, it.a = a, it.c = c, it.f0 = f0, it.nf = nf, it.pad = 0;
    b->items.push_back(it);
  };
  // 1. whole-frame occupancy, then their merges (so those models are ready early)
  const int64_t occ_chunk = 16384;
  for (int s = 0; s < S; ++s) {
    BStream &st = hs[s];
    st.n_occ = 0, st.n_build = 0;
    if (st.kind != OCQ_REGION_FRAME) continue;
    for (int f = 0; f < st.N; ++f)
      for (int64_t a = 0; a < st.hw; a += occ_chunk, ++st.n_occ)
        push(IT_OCC, s, a, (int32_t)std::min<int64_t>(occ_chunk, st.hw - a), f, 1);
  }
  for (int s = 0; s < S; ++s) {
    BStream &st = hs[s];
    if (st.kind != OCQ_REGION_FRAME) continue;
    for (int64_t a = 0; a < st.wpr; a += 1024, ++st.n_build)
      push(IT_MERGE, s, a, (int32_t)std::min<int64_t>(1024, st.wpr - a), 0, 0);
  }
  // 2. block and pixel builds, larger streams first
  std::vector<int> order(S);
  for (int s = 0; s < S; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return hs[x].hw * hs[x].N > hs[y].hw * hs[y].N; });
  for (int s : order) {
    BStream &st = hs[s];
    if (st.kind == OCQ_REGION_BLOCK) {
      for (int64_t r = 0; r < st.R; ++r, ++st.n_build) push(IT_BLOCK, s, r, 1, 0, 0);
    } else if (st.kind == OCQ_REGION_PIXEL) {
      for (int64_t a = 0; a < st.hw; a += kBatchThreads, ++st.n_build)
        push(IT_PIXEL, s, a, (int32_t)std::min<int64_t>(kBatchThreads, st.hw - a), 0, 0);
    }
  }
  // 3. classification: whole-frame streams first (ready first), then in build order
  std::vector<int> corder;
  for (int s = 0; s < S; ++s)
    if (hs[s].kind == OCQ_REGION_FRAME) corder.push_back(s);
  for (int s : order)
    if (hs[s].kind != OCQ_REGION_FRAME) corder.push_back(s);
  for (int s : corder) {
    BStream &st = hs[s];
    int tp = b->tile_px[st.kind], tf = b->tile_frames[st.kind];
    if (st.kind == OCQ_REGION_PIXEL && st.depth <= 3) {
      const int64_t cap = (int64_t)(b->smem / 4) / st.wpr;  // rows that fit the staging area
      if (tp > cap) tp = (int)cap;
    }
    for (int64_t a = 0; a < st.hw; a += tp)
      for (int f = 0; f < st.F; f += tf)
        push(IT_CLASSIFY, s, a, (int32_t)std::min<int64_t>(tp, st.hw - a), f, std::min(tf, st.F - f));
  }
  return OCQ_OK;
}

static ocq_status upload_plan(ocq_batch *b, cudaStream_t st) {
  ocq_status rc;
  if (b->items.size() > b->items_cap) {
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    b->items_cap = b->items.size();
    rc = cuda_status(cudaMalloc((void **)&b->d_items, b->items_cap * sizeof(BItem)), "batch work list");
    if (rc != OCQ_OK) return rc;
  }
  rc = cuda_status(cudaMemcpyAsync(b->d_items, b->items.data(), b->items.size() * sizeof(BItem),
                                   cudaMemcpyHostToDevice, st),
                   "upload work list");
  if (rc != OCQ_OK) return rc;
  rc = cuda_status(cudaMemcpyAsync(b->d_streams, b->hs.data(), b->hs.size() * sizeof(BStream),
                                   cudaMemcpyHostToDevice, st),
                   "upload streams");
  if (rc != OCQ_OK) return rc;
  return cuda_status(cudaStreamSynchronize(st), "upload plan");
}

static ocq_status enqueue_run(ocq_batch *b, cudaStream_t st) {
  const int S = (int)b->hs.size();
  ocq_status rc = cuda_status(cudaMemsetAsync(b->d_ctr, 0, (size_t)(2 + 2 * S) * 4, st), "reset batch counters");
  if (rc != OCQ_OK) return rc;
  for (int s = 0; s < S; ++s) {
    if (b->hs[s].kind == OCQ_REGION_FRAME) {
      rc = cuda_status(cudaMemsetAsync(b->hs[s].occ, 0, (size_t)b->hs[s].N * b->hs[s].wpr * 4, st), "clear occupancy");
      if (rc != OCQ_OK) return rc;
    }
  }
  batch_kernel<<<b->grid, kBatchThreads, b->smem, st>>>(b->d_streams, b->d_items, (int)b->items.size(), S, b->d_ctr);
  count_launch();
  return cuda_status(cudaGetLastError(), "batch_kernel");
}

static void free_graph(ocq_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr, b->graph = nullptr;
}

static ocq_status capture(ocq_batch *b) {
  free_graph(b);
  cudaStream_t cs = nullptr;
  ocq_status rc = cuda_status(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
  if (rc != OCQ_OK) return rc;
  rc = cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (rc == OCQ_OK) {
    ocq_status r2 = enqueue_run(b, cs);
    cudaGraph_t g = nullptr;
    rc = cuda_status(cudaStreamEndCapture(cs, &g), "end capture");
    if (rc == OCQ_OK) rc = r2;
    if (rc == OCQ_OK) {
      b->graph = g;
      rc = cuda_status(cudaGraphInstantiate(&b->exec, g, 0), "instantiate graph");
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  cudaStreamDestroy(cs);
  return rc;
}

extern "C" {

ocq_status ocq_batch_create(const ocq_stream_desc *streams, int n, void *stream, ocq_batch **out) {
  if (!out || !streams || n < 1) {
    set_error("ocq_batch_create: need streams and n >= 1");
    return OCQ_EINVAL;
  }
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  ocq_batch *b = new (std::nothrow) ocq_batch();
  if (!b) {
    set_error("host allocation failed");
    return OCQ_ENOMEM;
  }
  cudaGetDevice(&b->device);
  b->owner = st;
  b->desc.assign(streams, streams + n);
  size_t bytes = 0;
  size_t smem = 4096 * 4;
  std::vector<size_t> model_off(n), occ_off(n);
  for (int s = 0; s < n; ++s) {
    const ocq_stream_desc &d = streams[s];
    const int64_t R = region_count(d.H, d.W, d.region.kind, d.region.block);
    if (R < 1 || d.depth < 1 || d.depth > 8 || d.N < 1 || d.N > 255 || d.T < 1 || d.T > d.N || d.F < 0 ||
        !d.train || (d.F > 0 && (!d.test || !d.mask))) {
      set_error("ocq_batch_create: stream %d out of the batched domain (needs 1 <= T <= N <= 255, 1 <= depth <= 8, "
                "valid region and buffers)", s);
      delete b;
      return OCQ_EINVAL;
    }
    if (d.region.kind != OCQ_REGION_FRAME && d.depth > 5) {
      set_error("ocq_batch_create: stream %d: block and pixel regions deeper than 5 are not batched", s);
      delete b;
      return OCQ_ENOTSUP;
    }
    BStream h;
    memset(&h, 0, sizeof h);
    h.train = d.train, h.test = d.test, h.mask = d.mask;
    h.hw = (int64_t)d.H * d.W, h.R = R, h.wpr = wpr32(d.depth);
    h.N = d.N, h.F = d.F, h.H = d.H, h.W = d.W, h.kind = d.region.kind;
    h.block = d.region.kind == OCQ_REGION_BLOCK ? d.region.block : 0;
    h.bw = h.block > 0 ? (d.W + h.block - 1) / h.block : 1;
    h.depth = d.depth, h.T = d.T;
    int P = 0;
    for (uint32_t v = (uint32_t)d.N; v; v >>= 1) ++P;
    h.P = P;
    b->hs.push_back(h);
    model_off[s] = bytes;
    bytes += ((size_t)R * h.wpr * 4 + 255) & ~(size_t)255;
    occ_off[s] = bytes;
    if (h.kind == OCQ_REGION_FRAME) bytes += ((size_t)d.N * h.wpr * 4 + 255) & ~(size_t)255;
    // shared memory each item kind needs
    if (h.kind == OCQ_REGION_FRAME) smem = std::max(smem, (size_t)std::min<int64_t>(h.wpr, 8192) * 4);
    if (h.kind == OCQ_REGION_BLOCK) smem = std::max(smem, (size_t)h.wpr * (P + 2) * 4);
    if (h.kind == OCQ_REGION_PIXEL) smem = std::max(smem, (size_t)128 * kBatchThreads * 4);
  }
  b->smem = std::max<size_t>(smem, 64 * 1024);
  if (b->smem > 227 * 1024) {
    set_error("ocq_batch_create: the streams need %zu bytes of shared memory per CTA", b->smem);
    delete b;
    return OCQ_ENOTSUP;
  }
  b->arena_bytes = bytes;
  ocq_status rc = cuda_status(cudaMalloc((void **)&b->arena, bytes), "batch models");
  if (rc == OCQ_OK) rc = cuda_status(cudaMalloc((void **)&b->d_streams, n * sizeof(BStream)), "batch streams");
  if (rc == OCQ_OK) rc = cuda_status(cudaMalloc((void **)&b->d_ctr, (size_t)(2 + 2 * n) * 4), "batch counters");
  if (rc != OCQ_OK) {
    ocq_batch_destroy(b);
    return rc;
  }
  for (int s = 0; s < n; ++s) {
    BStream &h = b->hs[s];
    h.model = reinterpret_cast<uint32_t *>(b->arena + model_off[s]);
    h.occ = h.kind == OCQ_REGION_FRAME ? reinterpret_cast<uint32_t *>(b->arena + occ_off[s]) : nullptr;
    ocq_model *m = new (std::nothrow) ocq_model();
    if (!m) {
      ocq_batch_destroy(b);
      return OCQ_ENOMEM;
    }
    m->H = h.H, m->W = h.W, m->kind = h.kind, m->block = h.block, m->depth = h.depth, m->T = h.T, m->N = h.N;
    m->R = h.R, m->wpr = h.wpr, m->bits = h.model, m->bytes = (size_t)h.R * h.wpr * 4, m->stream = st;
    m->device = b->device;
    b->models.push_back(m);
  }
  cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
  if (e != cudaSuccess) {
    ocq_batch_destroy(b);
    return cuda_status(e, "batch_kernel smem");
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kBatchThreads, b->smem);
  b->grid = sm_count() * std::max(1, per_sm);  // all CTAs resident: every waited-on item is being run
  rc = plan_items(b);
  if (rc == OCQ_OK) rc = upload_plan(b, st);
  if (rc != OCQ_OK) {
    ocq_batch_destroy(b);
    return rc;
  }
  *out = b;
  return OCQ_OK;
}

ocq_status ocq_batch_run(ocq_batch *b, void *stream) {
  if (!b) {
    set_error("ocq_batch_run: NULL batch");
    return OCQ_EINVAL;
  }
  if (!b->exec) {
    ocq_status rc = capture(b);
    if (rc != OCQ_OK) return rc;
  }
  return cuda_status(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "batch graph launch");
}

ocq_status ocq_batch_set_tiles(ocq_batch *b, int region_kind, int pixels, int frames) {
  if (!b || region_kind < 0 || region_kind > 2 || pixels < 32 || pixels % 32 || frames < 1) {
    set_error("ocq_batch_set_tiles: bad arguments");
    return OCQ_EINVAL;
  }
  b->tile_px[region_kind] = pixels;
  b->tile_frames[region_kind] = frames;
  ocq_status rc = plan_items(b);
  if (rc == OCQ_OK) rc = upload_plan(b, b->owner);
  free_graph(b);
  return rc;
}

ocq_status ocq_batch_get_tiles(const ocq_batch *b, int region_kind, int *pixels, int *frames, int64_t *items) {
  if (!b || region_kind < 0 || region_kind > 2) {
    set_error("ocq_batch_get_tiles: bad arguments");
    return OCQ_EINVAL;
  }
  if (pixels) *pixels = b->tile_px[region_kind];
  if (frames) *frames = b->tile_frames[region_kind];
  if (items) *items = (int64_t)b->items.size();
  return OCQ_OK;
}

// Times candidate CLASSIFY tile shapes per region kind (each candidate runs the
// whole batch `reps` times on `stream`) and keeps the fastest.  Results are
// cached per shape signature (kind, depth, resolution) so an equal batch
// later skips the search.
ocq_status ocq_batch_autotune(ocq_batch *b, int reps, void *stream) {
  if (!b || reps < 1) {
    set_error("ocq_batch_autotune: bad arguments");
    return OCQ_EINVAL;
  }
  static std::map<std::string, std::pair<int, int>> cache;
  cudaStream_t st = (cudaStream_t)stream;
  std::string sig[3];
  bool present[3] = {false, false, false};
  for (const BStream &h : b->hs) {
    present[h.kind] = true;
    sig[h.kind] += std::to_string(h.depth) + "x" + std::to_string(h.hw) + ",";
  }
  const int cand_px[] = {512, 1024, 2048, 4096};
  const int cand_f[] = {8, 16, 32, 64};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ocq_status rc = OCQ_OK;
  for (int k = 0; k < 3 && rc == OCQ_OK; ++k) {
    if (!present[k]) continue;
    auto hit = cache.find(std::to_string(k) + ":" + sig[k]);
    if (hit != cache.end()) {
      b->tile_px[k] = hit->second.first, b->tile_frames[k] = hit->second.second;
      continue;
    }
    float best = 1e30f;
    int bp = b->tile_px[k], bf = b->tile_frames[k];
    for (int px : cand_px) {
      for (int fr : cand_f) {
        b->tile_px[k] = px, b->tile_frames[k] = fr;
        rc = plan_items(b);
        if (rc == OCQ_OK) rc = upload_plan(b, st);
        if (rc != OCQ_OK) break;
        enqueue_run(b, st);  // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) rc = enqueue_run(b, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rc != OCQ_OK) break;
        if (ms < best) best = ms, bp = px, bf = fr;
      }
      if (rc != OCQ_OK) break;
    }
    b->tile_px[k] = bp, b->tile_frames[k] = bf;
    cache[std::to_string(k) + ":" + sig[k]] = {bp, bf};
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == OCQ_OK) rc = plan_items(b);
  if (rc == OCQ_OK) rc = upload_plan(b, st);
  free_graph(b);
  return rc;
}

ocq_status ocq_batch_model(const ocq_batch *b, int i, const ocq_model **out) {
  if (!b || !out || i < 0 || i >= (int)b->models.size()) {
    set_error("ocq_batch_model: bad arguments");
    return OCQ_EINVAL;
  }
  *out = b->models[i];
  return OCQ_OK;
}

void ocq_batch_destroy(ocq_batch *b) {
  if (!b) return;
  free_graph(b);
  for (ocq_model *m : b->models) delete m;  // views: the arena owns the bits
  if (b->arena) cudaFree(b->arena);
  if (b->d_streams) cudaFree(b->d_streams);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_ctr) cudaFree(b->d_ctr);
  delete b;
}

ocq_status ocq_batch_status(ocq_batch *b, void *stream) {
  if (!b) {
    set_error("ocq_batch_status: NULL batch");
    return OCQ_EINVAL;
  }
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_status(e, "batch synchronise");
  uint32_t flag = 0;
  e = cudaMemcpy(&flag, b->d_ctr + 1, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e, "batch status");
  if (flag) {
    set_error("a batched item gave up waiting for its stream's model");
    return OCQ_ETIMEOUT;
  }
  return OCQ_OK;
}

}  // extern "C"
