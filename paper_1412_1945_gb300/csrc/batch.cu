// Batched form: many camera streams of uneven size, depth and region kind are
// built (S1-S3, Sec. 3, Alg. 1-2) and classified (S4, Alg. 3) by ONE replay
// of a CUDA graph holding one of three forms: a persistent kernel over a work
// list, the streams' plain kernels as concurrent branches, or grouped
// launches per kernel body (grouped.cu).
//
// The persistent work list holds the CTAs of the plain per-stream kernels as
// "virtual CTAs" (vb of vg) or warp ranges: each item runs a device body the
// plain kernels run (build_bodies.cuh, classify_bodies.cuh), so every stream's
// result is the plain path's result bit for bit.  Persistent CTAs of 256
// threads take items in list order from an atomic counter.  Per stream, a
// merge waits for the stream's occupancy items and classification for its
// build items; every waited-on item precedes the waiter in the list, so it was
// taken by a running CTA, and each wait is bounded (1 s) and records a timeout
// instead of spinning forever.  The classification work per item (in
// 1024-pixel frame tiles) is chosen per region kind by the autotuner
// (ocq_batch_autotune), which also picks the fastest of the three forms.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "build_bodies.cuh"
#include "classify_bodies.cuh"
#include "grouped.cuh"

namespace ocq {

// Operations a work item runs: each is the body of one of the plain kernels,
// run as virtual CTA vb of vg.
enum : int32_t {
  OP_OCC_FRAME = 0,    // occ_frame_body           (whole frame, depth <= 6)
  OP_OCC_GLOBAL,       // occ_global_body          (whole frame, depth >= 7)
  OP_MERGE,            // planes_merge_body        (whole frame)
  OP_BUILD_BLOCK,      // build_block_body         (blocks, depth <= 5, b > 16)
  OP_BUILD_BLOCK_WARP, // build_block_warp_body    (blocks, depth <= 5, b <= 16): regions [vb, aux)
  OP_BUILD_PIXEL_MG,   // build_pixel_mg_body      (pixels): 32-pixel tiles [vb, aux)
  OP_BUILD_BLOCK_TILE, // build_block_tile_body    (blocks, direct tables): 16x16 tiles [vb, aux)
  OP_BUILD_BLOCK_R8,   // build_block_r8_body      (8x8 blocks, depth 5): regions [vb, aux)
  OP_CLS_FRAME,        // classify_frame_body      (whole frame, depth <= 6)
  OP_CLS_PIXEL_TB,     // classify_pixel_tb_body   (pixels, H*W % 4 == 0): 128-pixel tiles [vb, aux)
  OP_CLS_BLOCK_TB,     // classify_block_tb_body   (blocks, b % 4 == 0, W % 4 == 0): tiles [vb, aux)
  OP_CLS_GENERIC       // classify_generic_body    (everything else)
};

struct BStream {
  const uint8_t *train, *test;
  uint8_t *mask;
  uint32_t *model;  // R * wpr words, internal (planar) order
  uint32_t *occ;    // whole-frame streams: N * wpr words of scratch
  int64_t hw, R, wpr;
  int32_t N, F, H, W, kind, block, bw, depth, T, P;
  int32_t n_build;     // items that complete the model
  int32_t n_occ;       // occupancy items (whole frame)
  int32_t occ_nbx;     // pixel chunks per frame in occupancy items
  int32_t ppl;         // block build, one warp per region: pixels per lane (0: CTA per region)
  int32_t km;          // pixel build: candidate counters (0: count every distinct leaf)
  int32_t tb;          // pixel / block classify: 1 if the L1 body applies
  int32_t nseg;        // block classify (L1 body): 128-pixel segments per pixel row
  int32_t stage;       // pixel classify, depth <= 3: rows staged in shared memory (else L1)
  int32_t kl;          // pixel regions, depth 4-5, candidates: kept-leaf list length (0: no index)
  int32_t tile;        // block build over 16x16 warp tiles with direct tables (build_block_tile_body)
  int32_t r8;          // block build, 8x8 at depth 5, one region per warp, two-level tables
  uint16_t *kept;      // kept-leaf index (kl > 0): written by the build, read by the classify
};

struct BItem {
  int32_t op, stream;
  int64_t vb, vg;
  int64_t aux;  // first pixel of a remainder range (CNT / GENERIC)
};

static constexpr int kBatchThreads = 256;
static constexpr int64_t kOccChunk = 16384;

// Counter block: [0] next item, [1] timeout flag, [2..2+S) occupancy done, [2+S..2+2S) build done.
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

// The warp-granular bodies run as calls of their own (one call site each), so
// that their unrolled register arrays do not share one frame with every other
// inlined body.
template <int D, int PPL>
__device__ __noinline__ void block_warp_item(const BStream &S, int64_t r0, int64_t r1, uint32_t *tab) {
  build_block_warp_body<D, PPL>(S.train, S.N, S.H, S.W, S.block, S.bw, (uint32_t)S.T, S.model, r0, r1,
                                kBatchThreads / 32, tab);
}

template <int D>
__device__ __forceinline__ void block_warp_item_d(const BStream &S, int64_t r0, int64_t r1, uint8_t *smem) {
  constexpr int TS = WarpTableCfg<D>::S;
  uint32_t *tab = reinterpret_cast<uint32_t *>(smem) + (threadIdx.x >> 5) * TS;
  for (int i = threadIdx.x & 31; i < TS; i += 32) tab[i] = 0u;
  __syncwarp();
  switch (S.ppl) {
    case 1: block_warp_item<D, 1>(S, r0, r1, tab); break;
    case 2: block_warp_item<D, 2>(S, r0, r1, tab); break;
    case 4: block_warp_item<D, 4>(S, r0, r1, tab); break;
    default: block_warp_item<D, 8>(S, r0, r1, tab); break;
  }
}

__device__ __noinline__ void block_warp_dispatch(const BStream &S, int64_t r0, int64_t r1, uint8_t *smem) {
  switch (S.depth) {
    case 1: block_warp_item_d<1>(S, r0, r1, smem); break;
    case 2: block_warp_item_d<2>(S, r0, r1, smem); break;
    case 3: block_warp_item_d<3>(S, r0, r1, smem); break;
    case 4: block_warp_item_d<4>(S, r0, r1, smem); break;
    default: block_warp_item_d<5>(S, r0, r1, smem); break;
  }
}

// Warp tiles: warp w of the CTA takes tiles t0 + w, t0 + w + 8, ... < t1 with
// its own table (zeroed here: the shared memory held other items' data).
template <int D, int B>
__device__ __noinline__ void block_tile_item(const BStream &S, int64_t t0, int64_t t1, uint8_t *smem) {
  using C = BlockTileCfg<D, B>;
  static_assert(C::DIRECT, "the persistent kernel hosts the direct-table tiles only");
  uint8_t *wsm = smem + (threadIdx.x >> 5) * C::WARP_SMEM;
  for (int i = threadIdx.x & 31; i < C::WARP_SMEM / 4; i += 32) reinterpret_cast<uint32_t *>(wsm)[i] = 0u;
  __syncwarp();
  build_block_tile_body<D, B, C::PF>(S.train, S.N, S.H, S.W, S.bw, (uint32_t)S.T, S.model, t0 + (threadIdx.x >> 5),
                                     t1, kBatchThreads / 32, wsm);
}

template <int D>
__device__ __noinline__ void block_r8_item(const BStream &S, int64_t r0, int64_t r1, uint8_t *smem) {
  uint8_t *wsm = smem + (threadIdx.x >> 5) * BlockR8CfgD<D>::WARP_SMEM;
  for (int i = threadIdx.x & 31; i < BlockR8CfgD<D>::WARP_SMEM / 4; i += 32) reinterpret_cast<uint32_t *>(wsm)[i] = 0u;
  __syncwarp();
  build_block_r8_body<D>(S.train, S.N, S.H, S.W, S.bw, (uint32_t)S.T, S.model, r0 + (threadIdx.x >> 5), r1,
                         kBatchThreads / 32, wsm);
}

__device__ __noinline__ void block_tile_dispatch(const BStream &S, int64_t t0, int64_t t1, uint8_t *smem) {
  if (S.block == 8) {
    if (S.depth == 2) block_tile_item<2, 8>(S, t0, t1, smem);
    else block_tile_item<3, 8>(S, t0, t1, smem);
  } else {
    if (S.depth == 2) block_tile_item<2, 16>(S, t0, t1, smem);
    else if (S.depth == 3) block_tile_item<3, 16>(S, t0, t1, smem);
    else block_tile_item<4, 16>(S, t0, t1, smem);
  }
}

template <int D, int KM>
__device__ __forceinline__ void pixel_mg_item(const BStream &S, int64_t t0, int64_t t1, uint8_t *smem) {
  leaf_t<D> *codes = reinterpret_cast<leaf_t<D> *>(smem) + (size_t)(threadIdx.x >> 5) * S.N * 32;
  for (int64_t t = t0; t < t1; t += kBatchThreads / 32) {
    build_pixel_mg_body<D, KM>(S.train, S.N, S.hw, (uint32_t)S.T, S.model, t, codes, 1, S.kl ? S.kept : nullptr);
    __syncwarp();
  }
}

template <int D>
__device__ __forceinline__ void pixel_mg_item_d(const BStream &S, int64_t t0, int64_t t1, uint8_t *smem) {
  switch (S.km) {
    case 1: pixel_mg_item<D, 1>(S, t0, t1, smem); break;
    case 2: pixel_mg_item<D, 2>(S, t0, t1, smem); break;
    case 4: pixel_mg_item<D, 4>(S, t0, t1, smem); break;
    case 8: pixel_mg_item<D, 8>(S, t0, t1, smem); break;
    default: pixel_mg_item<D, 0>(S, t0, t1, smem); break;
  }
}

__device__ __noinline__ void pixel_mg_dispatch(const BStream &S, int64_t t0, int64_t t1, uint8_t *smem) {
  switch (S.depth) {
    case 1: pixel_mg_item_d<1>(S, t0, t1, smem); break;
    case 2: pixel_mg_item_d<2>(S, t0, t1, smem); break;
    case 3: pixel_mg_item_d<3>(S, t0, t1, smem); break;
    case 4: pixel_mg_item_d<4>(S, t0, t1, smem); break;
    default: pixel_mg_item_d<5>(S, t0, t1, smem); break;
  }
}

__device__ __noinline__ void block_tb_dispatch(const BStream &S, int64_t t0, int64_t t1) {
  for (int64_t t = t0; t < t1; t += kBatchThreads / 32) {
    switch (S.depth) {
      case 1: classify_block_tb_body<1, 4>(S.test, S.F, S.H, S.W, S.block, S.bw, S.nseg, S.model, S.mask, t); break;
      case 2: classify_block_tb_body<2, 4>(S.test, S.F, S.H, S.W, S.block, S.bw, S.nseg, S.model, S.mask, t); break;
      case 3: classify_block_tb_body<3, 4>(S.test, S.F, S.H, S.W, S.block, S.bw, S.nseg, S.model, S.mask, t); break;
      case 4: classify_block_tb_body<4, 4>(S.test, S.F, S.H, S.W, S.block, S.bw, S.nseg, S.model, S.mask, t); break;
      default: classify_block_tb_body<5, 4>(S.test, S.F, S.H, S.W, S.block, S.bw, S.nseg, S.model, S.mask, t); break;
    }
  }
}

// Depth <= 3 with staging on: the warp's rows staged in shared memory (128 x 16
// words at most); otherwise L1 lookups.
__device__ __noinline__ void pixel_tb_dispatch(const BStream &S, int64_t t0, int64_t t1, uint8_t *smem) {
  uint32_t *rows = reinterpret_cast<uint32_t *>(smem) + (threadIdx.x >> 5) * 128 * 16;
  for (int64_t t = t0; t < t1; t += kBatchThreads / 32) {
    if (S.stage) {
      switch (S.depth) {
        case 1: classify_pixel_tbs_body<1, 8>(S.test, S.F, S.hw, S.model, S.mask, t, rows); break;
        case 2: classify_pixel_tbs_body<2, 8>(S.test, S.F, S.hw, S.model, S.mask, t, rows); break;
        default: classify_pixel_tbs_body<3, 8>(S.test, S.F, S.hw, S.model, S.mask, t, rows); break;
      }
    } else {
      switch (S.depth) {
        case 1: classify_pixel_tb_body<1, 8>(S.test, S.F, S.hw, S.model, S.mask, t); break;
        case 2: classify_pixel_tb_body<2, 8>(S.test, S.F, S.hw, S.model, S.mask, t); break;
        case 3: classify_pixel_tb_body<3, 8>(S.test, S.F, S.hw, S.model, S.mask, t); break;
        case 4: classify_pixel_tb_body<4, 8>(S.test, S.F, S.hw, S.model, S.mask, t); break;
        default: classify_pixel_tb_body<5, 8>(S.test, S.F, S.hw, S.model, S.mask, t); break;
      }
    }
  }
}

// Depth 4-5 with a kept-leaf index: the location's kept leaves in registers.
template <int D>
__device__ __forceinline__ void pixel_list_item(const BStream &S, int64_t t) {
  switch (S.kl) {
    case 2: classify_pixel_list_body<D, 4, 2>(S.test, S.F, S.hw, S.kept, S.mask, t); break;
    case 4: classify_pixel_list_body<D, 4, 4>(S.test, S.F, S.hw, S.kept, S.mask, t); break;
    default: classify_pixel_list_body<D, 4, 8>(S.test, S.F, S.hw, S.kept, S.mask, t); break;
  }
}

__device__ __noinline__ void pixel_list_dispatch(const BStream &S, int64_t t0, int64_t t1) {
  for (int64_t t = t0; t < t1; t += kBatchThreads / 32) {
    if (S.depth == 4)
      pixel_list_item<4>(S, t);
    else
      pixel_list_item<5>(S, t);
  }
}

template <int D>
__device__ __forceinline__ void run_item_d(const BStream &S, const BItem &it, uint8_t *smem) {
  const uint32_t T = (uint32_t)S.T;
  switch (it.op) {
    case OP_OCC_FRAME:
      if constexpr (D <= 6) occ_frame_body<D>(S.train, S.hw, 0, kOccChunk, S.occ, it.vb % S.occ_nbx, it.vb / S.occ_nbx);
      break;
    case OP_BUILD_BLOCK:
      if constexpr (D <= 5) build_block_body<D>(S.train, S.N, S.H, S.W, S.block, S.bw, S.P, T, S.model, S.R, it.vb, it.vg);
      break;
    case OP_CLS_FRAME:
      if constexpr (D <= 6) classify_frame_body<D>(S.test, (int64_t)S.F * S.hw, S.model, S.mask, it.vb, it.vg);
      break;
    default:
      break;
  }
}

__device__ void run_item(const BStream &S, const BItem &it, uint8_t *smem) {
  switch (it.op) {
    case OP_OCC_GLOBAL:
      occ_global_body(S.train, S.H, S.W, OCQ_REGION_FRAME, 0, S.depth, 0, S.N, 1, S.wpr, S.occ, it.vb, it.vg);
      return;
    case OP_MERGE:
      planes_merge_body(S.occ, S.N, S.wpr, nullptr, S.P, 1, 1, (uint32_t)S.T, S.model, it.vb, it.vg);
      return;
    case OP_BUILD_BLOCK_WARP:
      block_warp_dispatch(S, it.vb + (threadIdx.x >> 5), it.aux, smem);
      return;
    case OP_BUILD_PIXEL_MG:
      pixel_mg_dispatch(S, it.vb + (threadIdx.x >> 5), it.aux, smem);
      return;
    case OP_BUILD_BLOCK_TILE:
      block_tile_dispatch(S, it.vb, it.aux, smem);
      return;
    case OP_BUILD_BLOCK_R8:
      if (S.depth == 4)
        block_r8_item<4>(S, it.vb, it.aux, smem);
      else
        block_r8_item<5>(S, it.vb, it.aux, smem);
      return;
    case OP_CLS_PIXEL_TB:
      if (S.kl)
        pixel_list_dispatch(S, it.vb + (threadIdx.x >> 5), it.aux);
      else
        pixel_tb_dispatch(S, it.vb + (threadIdx.x >> 5), it.aux, smem);
      return;
    case OP_CLS_BLOCK_TB:
      block_tb_dispatch(S, it.vb + (threadIdx.x >> 5), it.aux);
      return;
    case OP_CLS_GENERIC:
      classify_generic_body(S.test, S.F, S.H, S.W, S.kind, S.block, S.depth, S.wpr, S.model, S.mask, it.aux, S.hw,
                            it.vb, it.vg);
      return;
    default:
      break;
  }
  switch (S.depth) {
    case 1: run_item_d<1>(S, it, smem); break;
    case 2: run_item_d<2>(S, it, smem); break;
    case 3: run_item_d<3>(S, it, smem); break;
    case 4: run_item_d<4>(S, it, smem); break;
    case 5: run_item_d<5>(S, it, smem); break;
    case 6: run_item_d<6>(S, it, smem); break;
    default: break;
  }
}

__global__ void __launch_bounds__(kBatchThreads, 3) batch_kernel(const BStream *__restrict__ streams,
                                                              const BItem *__restrict__ items, int n_items, int S,
                                                              uint32_t *ctr) {
  extern __shared__ __align__(128) uint8_t dsmem[];
  __shared__ int cur;
  __shared__ int ok;
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
      if (it.op == OP_MERGE) ok = wait_count(&occ_done[it.stream], (uint32_t)st.n_occ, err);
      if (it.op >= OP_CLS_FRAME) ok = wait_count(&build_done[it.stream], (uint32_t)st.n_build, err);
      __threadfence();
    }
    __syncthreads();
    if (ok) run_item(st, it, dsmem);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && ok) {
      if (it.op == OP_OCC_FRAME || it.op == OP_OCC_GLOBAL) atomicAdd(&occ_done[it.stream], 1u);
      else if (it.op < OP_CLS_FRAME) atomicAdd(&build_done[it.stream], 1u);
    }
  }
}

// A warp's table bytes of the direct-table tile build (depth <= 3, or 4 with
// 16 x 16 blocks).
static size_t block_tile_warp_smem(int d, int b) {
  if (b == 8) return d == 2 ? BlockTileCfg<2, 8>::WARP_SMEM : BlockTileCfg<3, 8>::WARP_SMEM;
  return d == 2 ? BlockTileCfg<2, 16>::WARP_SMEM : d == 3 ? BlockTileCfg<3, 16>::WARP_SMEM : BlockTileCfg<4, 16>::WARP_SMEM;
}

// Shared memory one item of stream S needs (bytes).
static size_t item_smem(const BStream &h) {
  const int d = h.depth;
  size_t need = 0;
  if (h.kind == OCQ_REGION_FRAME) {
    if (d <= 6) need = std::max<size_t>(need, (size_t)h.wpr * 4 * (d <= 4 ? 32 : 1));  // occ row / replicated row
  } else if (h.kind == OCQ_REGION_BLOCK) {
    if (h.r8)
      need = std::max<size_t>(need, (size_t)(kBatchThreads / 32) *
                                        (d == 4 ? BlockR8CfgD<4>::WARP_SMEM : BlockR8CfgD<5>::WARP_SMEM));
    else if (h.tile)
      need = std::max<size_t>(need, (size_t)(kBatchThreads / 32) * block_tile_warp_smem(d, h.block));
    else if (h.ppl > 0)
      need = std::max<size_t>(need, (size_t)(kBatchThreads / 32) * std::min(1 << (3 * d), 1024) * 4);
    else
      need = std::max<size_t>(need, (size_t)h.wpr * (h.P + 2) * 4);
  } else {
    need = std::max<size_t>(need, (size_t)(kBatchThreads / 32) * h.N * 32 * 2);  // candidate build: leaves
    if (h.stage)
      need = std::max<size_t>(need, (size_t)(kBatchThreads / 32) * 128 * 16 * 4);  // staged rows, 16-word stride
  }
  return need;
}

}  // namespace ocq

using namespace ocq;

// ---- host plan ------------------------------------------------------------------

struct ocq_batch {
  std::vector<ocq_stream_desc> desc;
  std::vector<BStream> hs;
  std::vector<ocq_model *> models;  // views (bits point into the arena)
  std::vector<BItem> items;
  int units[3] = {64, 64, 64};  // classification work per item, per region kind, in 1024-pixel frame tiles
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
  int mode = OCQ_BATCH_PERSISTENT;
  bool stage = false;  // depth <= 3 per-pixel classify rows staged in shared memory
  int hold = -1;  // test hook: stream whose build items are left out of the work list
  std::vector<cudaStream_t> side;  // branch streams of the graph form
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  // grouped form: launches per kernel body over the streams they cover, and
  // the streams left to their plain kernels
  std::vector<GLaunch> glaunch;
  std::vector<int> gfallback;
  GSeg *d_gsegs = nullptr;
  bool gplanned = false;
};

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Shared memory per CTA for the current streams and staging choice, the
// kernel's attribute and the persistent grid (CTAs resident at once).
static ocq_status size_kernel(ocq_batch *b) {
  size_t smem = 16 * 1024;
  for (BStream &h : b->hs) {
    h.stage = b->stage && h.kind == OCQ_REGION_PIXEL && h.depth <= 3 && h.tb;
    smem = std::max(smem, item_smem(h));
  }
  smem = (smem + 127) & ~(size_t)127;
  if (smem > 227 * 1024) {
    set_error("ocq_batch: the streams need %zu bytes of shared memory per CTA", smem);
    return OCQ_ENOTSUP;
  }
  b->smem = smem;
  ocq_status rc = cuda_status(cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)b->smem),
                              "batch_kernel smem");
  if (rc != OCQ_OK) return rc;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kBatchThreads, b->smem);
  b->grid = sm_count() * std::max(1, per_sm);
  return OCQ_OK;
}

// Work list: the virtual CTAs of every stream's plain kernels.  Whole-frame
// occupancy first, then the merges, then block and pixel builds (larger
// streams first), then classification in the order the models become ready.
static ocq_status plan_items(ocq_batch *b) {
  b->items.clear();
  const int S = (int)b->hs.size();
  std::vector<BStream> &hs = b->hs;
  auto push = [&](int32_t op, int s, int64_t vb, int64_t vg, int64_t aux) {
    if (s == b->hold && op < OP_CLS_FRAME) return;  // counted, never run: its classify items time out
    BItem it;
    it.op = op, it.stream = s, it.vb = vb, it.vg = vg, it.aux = aux;
    b->items.push_back(it);
  };
  for (int s = 0; s < S; ++s) {
    BStream &st = hs[s];
    st.n_occ = 0, st.n_build = 0;
    if (st.kind != OCQ_REGION_FRAME) continue;
    if (st.depth <= 6) {
      st.occ_nbx = (int32_t)cdiv(st.hw, kOccChunk);
      for (int64_t v = 0; v < (int64_t)st.occ_nbx * st.N; ++v, ++st.n_occ) push(OP_OCC_FRAME, s, v, 0, 0);
    } else {
      const int64_t vg = std::max<int64_t>(1, std::min<int64_t>(4096, cdiv(st.hw * st.N, (int64_t)kBatchThreads * 256)));
      for (int64_t v = 0; v < vg; ++v, ++st.n_occ) push(OP_OCC_GLOBAL, s, v, vg, 0);
    }
  }
  for (int s = 0; s < S; ++s) {
    BStream &st = hs[s];
    if (st.kind != OCQ_REGION_FRAME) continue;
    const int64_t vg = std::max<int64_t>(1, std::min<int64_t>(64, cdiv(st.wpr, kBatchThreads)));
    for (int64_t v = 0; v < vg; ++v, ++st.n_build) push(OP_MERGE, s, v, vg, 0);
  }
  std::vector<int> order(S);
  for (int s = 0; s < S; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return hs[x].hw * hs[x].N > hs[y].hw * hs[y].N; });
  for (int s : order) {
    BStream &st = hs[s];
    if (st.kind == OCQ_REGION_BLOCK && st.r8) {
      constexpr int64_t kRegionsPerItem = 64;  // 8 per warp
      for (int64_t r = 0; r < st.R; r += kRegionsPerItem, ++st.n_build)
        push(OP_BUILD_BLOCK_R8, s, r, 0, std::min(st.R, r + kRegionsPerItem));
    } else if (st.kind == OCQ_REGION_BLOCK && st.tile) {
      constexpr int64_t kTilesPerItem = 32;  // 4 per warp
      const int64_t tiles = cdiv(st.H, 16) * cdiv(st.W, 16);
      for (int64_t t = 0; t < tiles; t += kTilesPerItem, ++st.n_build)
        push(OP_BUILD_BLOCK_TILE, s, t, 0, std::min(tiles, t + kTilesPerItem));
    } else if (st.kind == OCQ_REGION_BLOCK && st.ppl > 0) {
      constexpr int64_t kRegionsPerItem = 40;
      for (int64_t r = 0; r < st.R; r += kRegionsPerItem, ++st.n_build)
        push(OP_BUILD_BLOCK_WARP, s, r, 0, std::min(st.R, r + kRegionsPerItem));
    } else if (st.kind == OCQ_REGION_BLOCK) {
      const int64_t vg = cdiv(st.R, 8);
      for (int64_t v = 0; v < vg; ++v, ++st.n_build) push(OP_BUILD_BLOCK, s, v, vg, 0);
    } else if (st.kind == OCQ_REGION_PIXEL) {
      constexpr int64_t kTilesPerItem = 64;  // 32-pixel tiles, 8 per warp
      const int64_t tiles = cdiv(st.hw, 32);
      for (int64_t t = 0; t < tiles; t += kTilesPerItem, ++st.n_build)
        push(OP_BUILD_PIXEL_MG, s, t, 0, std::min(tiles, t + kTilesPerItem));
    }
  }
  std::vector<int> corder;
  for (int s = 0; s < S; ++s)
    if (hs[s].kind == OCQ_REGION_FRAME) corder.push_back(s);
  for (int s : order)
    if (hs[s].kind != OCQ_REGION_FRAME) corder.push_back(s);
  for (int s : corder) {
    BStream &st = hs[s];
    const int64_t per = (int64_t)b->units[st.kind];
    auto generic = [&](int64_t p0) {
      const int64_t n = (st.hw - p0) * st.F;
      if (n <= 0) return;
      const int64_t vg = std::max<int64_t>(1, std::min<int64_t>(cdiv(n, per * 1024), cdiv(n, kBatchThreads)));
      for (int64_t v = 0; v < vg; ++v) push(OP_CLS_GENERIC, s, v, vg, p0);
    };
    if (st.F == 0) continue;
    if (st.kind == OCQ_REGION_FRAME && st.depth <= 6) {
      const int64_t vg = std::max<int64_t>(1, cdiv(st.hw * st.F, per * 1024));
      for (int64_t v = 0; v < vg; ++v) push(OP_CLS_FRAME, s, v, vg, 0);
    } else if (st.kind == OCQ_REGION_PIXEL && st.tb) {
      const int64_t tiles = cdiv(st.hw, 128);
      const int64_t nw = kBatchThreads / 32;
      const int64_t k = std::max<int64_t>(1, per * 1024 / (128 * (int64_t)st.F) / nw) * nw;
      for (int64_t t = 0; t < tiles; t += k) push(OP_CLS_PIXEL_TB, s, t, 0, std::min(tiles, t + k));
    } else if (st.kind == OCQ_REGION_BLOCK && st.tb) {
      const int64_t tiles = cdiv(st.H, st.block) * (int64_t)st.nseg * st.block;
      const int64_t nw = kBatchThreads / 32;
      const int64_t k = std::max<int64_t>(1, per * 1024 / (128 * (int64_t)st.F) / nw) * nw;
      for (int64_t t = 0; t < tiles; t += k) push(OP_CLS_BLOCK_TB, s, t, 0, std::min(tiles, t + k));
    } else {
      generic(0);
    }
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
  for (int s = 0; s < S && rc == OCQ_OK; ++s) {
    const BStream &h = b->hs[s];
    if (h.kind == OCQ_REGION_FRAME)
      rc = cuda_status(cudaMemsetAsync(h.occ, 0, (size_t)h.N * h.wpr * 4, st), "clear occupancy");
  }
  if (rc != OCQ_OK) return rc;
  batch_kernel<<<b->grid, kBatchThreads, b->smem, st>>>(b->d_streams, b->d_items, (int)b->items.size(), S, b->d_ctr);
  count_launch();
  return cuda_status(cudaGetLastError(), "batch_kernel");
}

static void free_graph(ocq_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr, b->graph = nullptr;
}

// Graph form: one branch per camera stream (side streams forked from and
// joined back to the capture stream), each running that stream's plain
// kernels, build then classify.  Branches are independent, so the graph runs
// the streams' kernels concurrently; the work is the plain path's, kernel by
// kernel.
static ocq_status enqueue_branches(ocq_batch *b, cudaStream_t cs) {
  const int S = (int)b->hs.size();
  const int NB = std::min(S, 64);
  ocq_status rc = OCQ_OK;
  if (!b->fork) rc = cuda_status(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "fork event");
  while (rc == OCQ_OK && (int)b->side.size() < NB) {
    cudaStream_t s2 = nullptr;
    cudaEvent_t e2 = nullptr;
    rc = cuda_status(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking), "branch stream");
    if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming), "join event");
    if (s2) b->side.push_back(s2);
    if (e2) b->joins.push_back(e2);
  }
  if (rc == OCQ_OK) rc = cuda_status(cudaEventRecord(b->fork, cs), "fork");
  for (int i = 0; i < NB && rc == OCQ_OK; ++i) rc = cuda_status(cudaStreamWaitEvent(b->side[i], b->fork, 0), "fork wait");
  // Larger streams first on each branch stream.
  std::vector<int> order(S);
  for (int s = 0; s < S; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return b->hs[x].hw * (b->hs[x].N + b->hs[x].F) > b->hs[y].hw * (b->hs[y].N + b->hs[y].F);
  });
  for (int k = 0; k < S && rc == OCQ_OK; ++k) {
    const int s = order[k];
    const ocq_stream_desc &d = b->desc[s];
    cudaStream_t st = b->side[k % NB];
    rc = launch_build(d.train, d.N, b->models[s], st);
    if (rc == OCQ_OK && d.F > 0) rc = launch_classify(b->models[s], d.test, d.F, d.mask, st);
  }
  for (int i = 0; i < NB && rc == OCQ_OK; ++i) {
    rc = cuda_status(cudaEventRecord(b->joins[i], b->side[i]), "join");
    if (rc == OCQ_OK) rc = cuda_status(cudaStreamWaitEvent(cs, b->joins[i], 0), "join wait");
  }
  return rc;
}

// Grouped form: one launch per kernel body and template over all streams it
// covers (grouped.cu), chained on one branch (each class's builds before its
// classification); streams outside those bodies run their plain kernels on
// branches of their own.
static ocq_status plan_grouped(ocq_batch *b) {
  if (b->gplanned) return OCQ_OK;
  std::vector<GStreamIn> in;
  for (size_t s = 0; s < b->hs.size(); ++s) {
    const BStream &h = b->hs[s];
    GStreamIn x;
    x.train = h.train, x.test = h.test, x.mask = h.mask, x.model = h.model, x.occ = h.occ, x.kept = h.kept;
    x.N = h.N, x.F = h.F, x.H = h.H, x.W = h.W, x.kind = h.kind, x.block = h.block, x.depth = h.depth, x.T = h.T;
    x.km = h.km, x.kl = h.kl;
    in.push_back(x);
  }
  ocq_status rc = grouped_plan(in, b->glaunch, b->gfallback);
  if (rc != OCQ_OK) return rc;
  size_t nseg = 0;
  for (const GLaunch &L : b->glaunch) nseg += L.segs.size();
  if (nseg > 0) {
    rc = cuda_status(cudaMalloc((void **)&b->d_gsegs, nseg * sizeof(GSeg)), "grouped segments");
    if (rc != OCQ_OK) return rc;
    size_t at = 0;
    for (GLaunch &L : b->glaunch) {
      L.dev = b->d_gsegs + at;
      rc = cuda_status(cudaMemcpy(L.dev, L.segs.data(), L.segs.size() * sizeof(GSeg), cudaMemcpyHostToDevice),
                       "upload grouped segments");
      if (rc != OCQ_OK) return rc;
      at += L.segs.size();
    }
  }
  b->gplanned = true;
  return OCQ_OK;
}

static ocq_status ensure_side_streams(ocq_batch *b, int n) {
  ocq_status rc = OCQ_OK;
  if (!b->fork) rc = cuda_status(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "fork event");
  while (rc == OCQ_OK && (int)b->side.size() < n) {
    cudaStream_t s2 = nullptr;
    cudaEvent_t e2 = nullptr;
    rc = cuda_status(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking), "branch stream");
    if (rc == OCQ_OK) rc = cuda_status(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming), "join event");
    if (s2) b->side.push_back(s2);
    if (e2) b->joins.push_back(e2);
  }
  return rc;
}

static ocq_status enqueue_grouped(ocq_batch *b, cudaStream_t cs) {
  ocq_status rc = plan_grouped(b);
  if (rc != OCQ_OK) return rc;
  const int nfb = std::min<int>((int)b->gfallback.size(), 8);
  const int NB = kGroupBranches + nfb;
  rc = ensure_side_streams(b, NB);
  if (rc == OCQ_OK) rc = cuda_status(cudaEventRecord(b->fork, cs), "fork");
  for (int i = 0; i < NB && rc == OCQ_OK; ++i) rc = cuda_status(cudaStreamWaitEvent(b->side[i], b->fork, 0), "fork wait");
  // whole-frame occupancy is ORed into zeroed scratch: cleared on the branch
  // that builds the stream
  for (const GLaunch &L : b->glaunch) {
    if (L.kind != GK_OCC) continue;
    for (const GSeg &g : L.segs)
      if (rc == OCQ_OK)
        rc = cuda_status(cudaMemsetAsync(g.occ, 0, (size_t)g.N * wpr32(L.a) * 4, b->side[L.branch]), "clear occupancy");
  }
  for (const GLaunch &L : b->glaunch) {
    if (rc != OCQ_OK) break;
    rc = grouped_launch(L, b->side[L.branch]);
  }
  for (size_t k = 0; k < b->gfallback.size() && rc == OCQ_OK; ++k) {
    const int s = b->gfallback[k];
    const ocq_stream_desc &d = b->desc[s];
    cudaStream_t st = b->side[kGroupBranches + (int)(k % (size_t)nfb)];
    rc = launch_build(d.train, d.N, b->models[s], st);
    if (rc == OCQ_OK && d.F > 0) rc = launch_classify(b->models[s], d.test, d.F, d.mask, st);
  }
  for (int i = 0; i < NB && rc == OCQ_OK; ++i) {
    rc = cuda_status(cudaEventRecord(b->joins[i], b->side[i]), "join");
    if (rc == OCQ_OK) rc = cuda_status(cudaStreamWaitEvent(cs, b->joins[i], 0), "join wait");
  }
  return rc;
}

static ocq_status capture(ocq_batch *b) {
  free_graph(b);
  SharedGpuScope shared;  // the streams' builds run beside one another
  if (b->mode == OCQ_BATCH_GROUPED) {  // plan (device tables, kernel attributes) before capturing
    ocq_status rp = plan_grouped(b);
    if (rp != OCQ_OK) return rp;
  }
  cudaStream_t cs = nullptr;
  ocq_status rc = cuda_status(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
  if (rc != OCQ_OK) return rc;
  rc = cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (rc == OCQ_OK) {
    ocq_status r2 = b->mode == OCQ_BATCH_GRAPH     ? enqueue_branches(b, cs)
                    : b->mode == OCQ_BATCH_GROUPED ? enqueue_grouped(b, cs)
                                                   : enqueue_run(b, cs);
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
  size_t smem = 16 * 1024;
  std::vector<size_t> model_off(n), occ_off(n), kept_off(n);
  std::vector<char> list_only(n, 0);
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
    if (h.kind == OCQ_REGION_PIXEL) {
      const int k = d.N / d.T;
      h.km = k <= 1 ? 1 : k <= 2 ? 2 : k <= 4 ? 4 : k <= 8 ? 8 : 0;
      h.kl = (d.depth == 4 || d.depth == 5) && h.km > 0 ? (h.km < 2 ? 2 : h.km) : 0;
      h.tb = d.F > 0 && h.hw % 4 == 0 &&
             ((reinterpret_cast<uintptr_t>(d.test) | reinterpret_cast<uintptr_t>(d.mask)) & 3) == 0;
      // a list model (no rows) where every classify item can read the index
      list_only[s] = h.kl > 0 && h.tb && list_model_applies(h.kind, d.depth, d.N, d.T);
    }
    if (h.kind == OCQ_REGION_BLOCK && h.block % 4 == 0 && d.W % 4 == 0 && d.F > 0 &&
        ((reinterpret_cast<uintptr_t>(d.test) | reinterpret_cast<uintptr_t>(d.mask)) & 3) == 0) {
      h.tb = 1;
      h.nseg = (d.W + 127) / 128;
    }
    if (h.kind == OCQ_REGION_BLOCK && block_warp_ok(d.N, d.H, d.W, h.block)) {
      const int npx = h.block * h.block;
      h.ppl = npx <= 32 ? 1 : npx <= 64 ? 2 : npx <= 128 ? 4 : 8;
    }
    {
      SharedGpuScope shared;  // the form the batched plain kernels take
      h.tile = h.kind == OCQ_REGION_BLOCK && (d.depth <= 3 || (d.depth == 4 && h.block == 16)) &&
               block_tile_ok(d.N, d.H, d.W, h.block, d.depth, d.train);
      h.r8 = h.kind == OCQ_REGION_BLOCK && block_r8_ok(d.N, d.H, d.W, h.block, d.depth, d.train);
    }
    b->hs.push_back(h);
    model_off[s] = bytes;
    if (!list_only[s]) bytes += ((size_t)R * h.wpr * 4 + 255) & ~(size_t)255;
    occ_off[s] = bytes;
    if (h.kind == OCQ_REGION_FRAME) bytes += ((size_t)d.N * h.wpr * 4 + 255) & ~(size_t)255;
    // the kept-leaf index a per-pixel candidate build of depth 4-5 writes:
    // allocated here so that no allocation is captured into the graph
    kept_off[s] = bytes;
    if (h.kl > 0) bytes += ((size_t)R * 16 + 255) & ~(size_t)255;
    smem = std::max(smem, item_smem(h));
  }
  b->smem = (smem + 127) & ~(size_t)127;
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
    h.model = list_only[s] ? nullptr : reinterpret_cast<uint32_t *>(b->arena + model_off[s]);
    h.occ = h.kind == OCQ_REGION_FRAME ? reinterpret_cast<uint32_t *>(b->arena + occ_off[s]) : nullptr;
    ocq_model *m = new (std::nothrow) ocq_model();
    if (!m) {
      ocq_batch_destroy(b);
      return OCQ_ENOMEM;
    }
    m->H = h.H, m->W = h.W, m->kind = h.kind, m->block = h.block, m->depth = h.depth, m->T = h.T, m->N = h.N;
    m->R = h.R, m->wpr = h.wpr, m->bits = h.model, m->bytes = h.model ? (size_t)h.R * h.wpr * 4 : 0, m->stream = st;
    m->device = b->device;
    if (h.kl > 0) {
      h.kept = reinterpret_cast<uint16_t *>(b->arena + kept_off[s]);
      m->kept = h.kept, m->kept_len = h.kl;
    }
    b->models.push_back(m);
  }
  rc = size_kernel(b);
  if (rc == OCQ_OK) rc = plan_items(b);
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

ocq_status ocq_batch_set_work(ocq_batch *b, int region_kind, int units) {
  if (!b || region_kind < 0 || region_kind > 2 || units < 1) {
    set_error("ocq_batch_set_work: bad arguments");
    return OCQ_EINVAL;
  }
  b->units[region_kind] = units;
  ocq_status rc = plan_items(b);
  if (rc == OCQ_OK) rc = upload_plan(b, b->owner);
  free_graph(b);
  return rc;
}

ocq_status ocq_batch_get_work(const ocq_batch *b, int region_kind, int *units, int64_t *items) {
  if (!b || region_kind < 0 || region_kind > 2) {
    set_error("ocq_batch_get_work: bad arguments");
    return OCQ_EINVAL;
  }
  if (units) *units = b->units[region_kind];
  if (items) *items = (int64_t)b->items.size();
  return OCQ_OK;
}

// Autotuner: for each region kind present, times candidate classification
// work sizes per item (the whole batch `reps` times each, on `stream`) and
// keeps the fastest.  Results are cached per signature (kind, depths, sizes)
// so an equal batch later skips the search.
ocq_status ocq_batch_autotune(ocq_batch *b, int reps, void *stream) {
  if (!b || reps < 1) {
    set_error("ocq_batch_autotune: bad arguments");
    return OCQ_EINVAL;
  }
  static std::map<std::string, int> cache;
  cudaStream_t st = (cudaStream_t)stream;
  std::string sig[3];
  bool present[3] = {false, false, false};
  for (const BStream &h : b->hs) {
    present[h.kind] = true;
    sig[h.kind] += std::to_string(h.depth) + "x" + std::to_string(h.hw) + "f" + std::to_string(h.F) + ",";
  }
  const int cand[] = {8, 16, 32, 64, 128, 256};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ocq_status rc = OCQ_OK;
  for (int k = 0; k < 3 && rc == OCQ_OK; ++k) {
    if (!present[k]) continue;
    const std::string key = std::to_string(k) + ":" + sig[k];
    auto hit = cache.find(key);
    if (hit != cache.end()) {
      b->units[k] = hit->second;
      continue;
    }
    float best = 1e30f;
    int bu = b->units[k];
    for (int u : cand) {
      b->units[k] = u;
      rc = plan_items(b);
      if (rc == OCQ_OK) rc = upload_plan(b, st);
      if (rc != OCQ_OK) break;
      rc = enqueue_run(b, st);  // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && rc == OCQ_OK; ++r) rc = enqueue_run(b, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rc != OCQ_OK) break;
      if (ms < best) best = ms, bu = u;
    }
    b->units[k] = bu;
    cache[key] = bu;
  }
  if (rc == OCQ_OK) rc = plan_items(b);
  if (rc == OCQ_OK) rc = upload_plan(b, st);
  // Staging of depth <= 3 per-pixel rows in shared memory: it speeds those
  // streams up but raises every CTA's shared memory (less L1 for the others),
  // so it is timed both ways on this batch.
  bool stageable = false;
  for (const BStream &h : b->hs) stageable |= h.kind == OCQ_REGION_PIXEL && h.depth <= 3 && h.tb;
  if (stageable && rc == OCQ_OK) {
    float ts[2] = {1e30f, 1e30f};
    for (int stg = 0; stg < 2 && rc == OCQ_OK; ++stg) {
      b->stage = stg == 1;
      rc = size_kernel(b);
      if (rc == OCQ_OK) rc = plan_items(b);
      if (rc == OCQ_OK) rc = upload_plan(b, st);
      if (rc != OCQ_OK) break;
      rc = enqueue_run(b, st);  // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && rc == OCQ_OK; ++r) rc = enqueue_run(b, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ts[stg], e0, e1);
    }
    b->stage = ts[1] < ts[0];
    if (rc == OCQ_OK) rc = size_kernel(b);
    if (rc == OCQ_OK) rc = plan_items(b);
    if (rc == OCQ_OK) rc = upload_plan(b, st);
  }
  // Then the form: the persistent kernel with the chosen work sizes against
  // the graph of per-stream branches, each captured and replayed.
  float t[3] = {1e30f, 1e30f, 1e30f};
  for (int mode = 0; mode < 3 && rc == OCQ_OK; ++mode) {
    free_graph(b);
    b->mode = mode;
    rc = capture(b);
    if (rc != OCQ_OK) break;
    rc = cuda_status(cudaGraphLaunch(b->exec, st), "autotune warm-up");
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && rc == OCQ_OK; ++r) rc = cuda_status(cudaGraphLaunch(b->exec, st), "autotune run");
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&t[mode], e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == OCQ_OK) {
    int best = OCQ_BATCH_PERSISTENT;
    for (int mode = 1; mode < 3; ++mode)
      if (t[mode] < t[best]) best = mode;
    if (best != b->mode) free_graph(b);
    b->mode = best;
  }
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
  for (cudaStream_t s2 : b->side) cudaStreamDestroy(s2);
  for (cudaEvent_t e2 : b->joins) cudaEventDestroy(e2);
  if (b->fork) cudaEventDestroy(b->fork);
  for (ocq_model *m : b->models) delete m;  // views: the arena owns the bits
  if (b->arena) cudaFree(b->arena);
  if (b->d_streams) cudaFree(b->d_streams);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_ctr) cudaFree(b->d_ctr);
  if (b->d_gsegs) cudaFree(b->d_gsegs);
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
  const bool ct = classify_take_timeout(), bt = build_take_timeout(), gt = grouped_take_timeout();
  if (ct || bt || gt) {
    set_error("a kernel of the graph form gave up waiting for a copy");
    return OCQ_ETIMEOUT;
  }
  return OCQ_OK;
}

ocq_status ocq_batch_set_mode(ocq_batch *b, int mode) {
  if (!b || (mode != OCQ_BATCH_PERSISTENT && mode != OCQ_BATCH_GRAPH && mode != OCQ_BATCH_GROUPED)) {
    set_error("ocq_batch_set_mode: bad arguments");
    return OCQ_EINVAL;
  }
  if (mode != b->mode) free_graph(b);
  b->mode = mode;
  return OCQ_OK;
}

int ocq_batch_get_mode(const ocq_batch *b) { return b ? b->mode : -1; }

ocq_status ocq_batch_set_staging(ocq_batch *b, int on) {
  if (!b) {
    set_error("ocq_batch_set_staging: NULL batch");
    return OCQ_EINVAL;
  }
  b->stage = on != 0;
  ocq_status rc = size_kernel(b);
  if (rc == OCQ_OK) rc = plan_items(b);
  if (rc == OCQ_OK) rc = upload_plan(b, b->owner);
  free_graph(b);
  return rc;
}

int ocq_batch_get_staging(const ocq_batch *b) { return b ? (int)b->stage : -1; }

ocq_status ocq_batch_debug_hold_builds(ocq_batch *b, int stream) {
  if (!b || stream < -1 || stream >= (int)b->hs.size()) {
    set_error("ocq_batch_debug_hold_builds: bad arguments");
    return OCQ_EINVAL;
  }
  b->hold = stream;
  ocq_status rc = plan_items(b);
  if (rc == OCQ_OK) rc = upload_plan(b, b->owner);
  free_graph(b);
  return rc;
}

}  // extern "C"
