// Grouped launches of the batched form (grouped.cu): shared by the batch
// planner (batch.cu).
#pragma once

#include <vector>

#include "ocq_internal.cuh"

namespace ocq {

constexpr int64_t kGroupOccChunk = 16384;  // pixels per whole-frame occupancy CTA

// One stream's share of a grouped launch: CTAs [cta0, cta0 + vg) of the
// launch run the body for this stream as virtual CTAs 0 .. vg - 1.
struct GSeg {
  const uint8_t *in;  // frames read: training frames (builds) or test frames
  uint8_t *mask;
  uint32_t *model;    // leaf bitset rows, internal order (null for a list model)
  uint32_t *occ;      // whole frame: N per-frame leaf bitsets
  uint16_t *kept;     // kept-leaf lists
  int64_t hw, cta0, vg;
  int64_t units;      // tiles, items or words the body walks
  int64_t aux;        // occupancy: CTAs per frame; block classify: tiles
  int32_t N, F, H, W, block, bw, T, P;
  int32_t aux2, aux3;  // block classify: frames per chunk, 128-pixel segments per row
  // serving ticks: frame f of the segment and its mask at ftab[f] and mtab[f]
  // (device tables; null: in + f*hw*3 and mask + f*hw).  While planning, tab
  // is the index of the segment's first entry in the tick's pointer list
  // (frames, then masks), or -1.
  const uint8_t *const *ftab;
  uint8_t *const *mtab;
  uint16_t *const *ctab;  // frame f's leaf codes into ctab[f] too (a code window's slot), or null
  int64_t tab;
  int32_t codes;  // planning: the segment's table also lists code slots (after the masks)
  int32_t pad;
};

// Kernel kinds (one launch per kind and template arguments a, b).
enum GroupKind : int {
  GK_OCC = 0,      // whole-frame occupancy, a = depth
  GK_MERGE,        // whole-frame merge (any depth)
  GK_CLS_FRAME,    // whole-frame classify, a = depth
  GK_BLOCK_TILE,   // block build over 16 x 16 warp tiles, a = depth, b = block size
  GK_BLOCK_WARP,   // block build, one warp per region, a = depth, b = pixels per lane
  GK_BLOCK_FS,     // block build, frames split over a CTA's warps, a = depth, b = block size
  GK_BLOCK_R8,     // block build, 8 x 8 at depth 5, one region per warp, two-level tables
  GK_BLOCK_TB,     // block classify, warps walking frames, a = depth
  GK_PIX_WS_BUILD, // per-pixel build, depth <= 3, counters + copy warp, a = depth
  GK_PIX_WS_CLS,   // per-pixel classify, depth <= 3, rows staged + copy warp, a = depth
  GK_PIX_MG,       // per-pixel candidate build, a = depth, b = candidate counters
  GK_PIX_LIST,     // per-pixel classify against kept-leaf lists, a = depth, b = list length
  GK_CODES,        // serving window: per-pixel u16 leaf codes of one frame, a = depth
  GK_COUNT         // serving window: a camera's new leaf bitsets into its ring and counts
};

// The grouped launches chain on one branch of the batch graph, in GroupKind
// order (so each class's builds come before its classification).  The
// classes (whole frame, blocks, pixels d <= 3, pixels d = 4-5) on concurrent
// branches measured slower and uneven from run to run (7.7-9.8 ms against
// 7.1 ms on the 64-stream preset): the large grouped kernels of different
// classes contend for the SMs.  Streams no grouped body takes run their plain
// kernels on branches of their own.
constexpr int kGroupBranches = 1;

struct GLaunch {
  int kind = 0, a = 0, b = 0, branch = 0;
  std::vector<GSeg> segs;
  GSeg *dev = nullptr;  // device copy of segs (owned by the batch's upload buffer)
  int threads = 256;
  size_t smem = 0;
  int64_t grid = 0;
};

// What the planner needs to know of a camera stream.
struct GStreamIn {
  const uint8_t *train, *test;
  uint8_t *mask;
  uint32_t *model, *occ;
  uint16_t *kept;
  int N, F, H, W, kind, block, depth, T, km, kl;
};

// Plans grouped launches for the streams they cover, in dependency order per
// branch; streams they do not cover are listed in `fallback` (run by their
// plain kernels).  Sets each launch's CTA shape, shared memory and grid.
ocq_status grouped_plan(const std::vector<GStreamIn> &in, std::vector<GLaunch> &out, std::vector<int> &fallback);
// One frame of a served camera in a serving tick (continuous batching: the
// frames that arrived since the last tick, of every camera, classified and
// entered into their windows by a few grouped launches).
struct GFrameIn {
  const uint8_t *frame;
  uint8_t *mask;
  const ocq_model *model;
  int win;            // 1: leaf bitsets + counts, 2: per-pixel codes
  uint8_t *ring;      // the camera's window
  uint32_t *fresh;    // bits: N bitsets of entering frames
  uint16_t *counts;   // bits
  int N;
  int64_t slot;       // ring slot of this frame
  int j;              // this frame's index among its camera's frames of the tick
  int m;              // the camera's frames in the tick (first frame's record: j == 0)
};
// Plans a tick: grouped classify launches, then window launches.  Frames no
// grouped classify body takes are listed in `single` (classified one by one).
// A camera's frames of the tick share one classify segment (its model read
// once for all of them) where the body takes frame tables: `ptrs` receives the
// tables (each segment's frames, its masks, then for code windows the slots
// its leaf codes go to: that classify writes them, no separate code pass;
// GSeg::tab indexes them).
ocq_status grouped_plan_tick(const std::vector<GFrameIn> &in, std::vector<GLaunch> &out, std::vector<int> &single,
                             std::vector<const void *> &ptrs);
// Enqueues one planned launch (segments already on the device) on `st`.
ocq_status grouped_launch(const GLaunch &L, cudaStream_t st);
// True (and cleared) if a bounded wait of a grouped body gave up.
bool grouped_take_timeout();

}  // namespace ocq
