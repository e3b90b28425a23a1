// Internal declarations shared by the library's translation units.
//
// Device model layout.  Inside the library a region's leaf set is a bitset
// indexed by the *channel-planar* code
//     q = r_d | g_d << d | b_d << 2d,    c_d = c >> (8 - d),
// a fixed permutation of the path code's 3d bits (the path code interleaves
// the same bits level by level, red most significant in each triple).  q is
// cheap to form from packed RGB bytes (mask, then one byte dot product), which
// is what the classify inner loop needs; export and import translate to and
// from the path-code layout of the public interface.  A region row is
// wpr32(d) u32 words, leaf q at bit q%32 of word q/32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ocq.h"

struct ocq_model {
  int H, W, kind, block, depth, T, N;
  int64_t R;           // regions
  int64_t wpr;         // u32 words per region (internal layout)
  uint32_t *bits;      // device, R * wpr words; nullptr for a list model (kept-leaf index only)
  size_t bytes;
  cudaStream_t stream; // stream the model was created on (stream-ordered free)
  int device;
  // Pixel regions, depth 4-5, built by the candidate build with k = floor(N/T)
  // <= 8 (no location keeps more than 8 leaves): per pixel location its kept
  // leaves as 8 u16 planar codes, kKeptNone padding.  Beside the rows it is a
  // derived index for the classify; without rows (bits == nullptr, a "list
  // model") it is the model itself, and export expands it into the bitset
  // layout.  Valid while kept_len > 0.
  uint16_t *kept;
  int kept_len;  // entries of a list that can hold a kept leaf: 2, 4 or 8; 0 = no valid index
};

constexpr uint16_t kKeptNone = 0xFFFFu;  // no planar code of depth <= 5 equals it

namespace ocq {

// ---- host-side helpers (api.cu) --------------------------------------------
void set_error(const char *fmt, ...);
void clear_error();  // empties the calling thread's last-error text
ocq_status cuda_status(cudaError_t e, const char *what);
int sm_count();
// cudaMallocAsync from the pool the calling thread selected with PoolScope
// (else the device's default pool).
cudaError_t malloc_async(void **p, size_t bytes, cudaStream_t st);
struct PoolScope {
  explicit PoolScope(cudaMemPool_t pool);
  ~PoolScope();
  PoolScope(const PoolScope &) = delete;
  PoolScope &operator=(const PoolScope &) = delete;

 private:
  cudaMemPool_t prev_;
};
void count_launch(int n = 1);
int64_t region_count(int H, int W, int kind, int block);

inline int64_t wpr32(int d) { return d == 1 ? 1 : (int64_t)1 << (3 * d - 5); }
inline int64_t wpr64(int d) { return d <= 2 ? 1 : (int64_t)1 << (3 * d - 6); }

// ---- device helpers ----------------------------------------------------------

// Mask selecting the top d bits of each byte after a right shift by 8-d.
__host__ __device__ __forceinline__ constexpr uint32_t byte_mask(int d) { return ((1u << d) - 1u) * 0x01010101u; }

// q from a word whose bytes 0..2 already hold r_d, g_d, b_d (byte 3 ignored).
template <int D>
__device__ __forceinline__ uint32_t planar_from_masked(uint32_t t) {
  if constexpr (D <= 3) {
    return __dp4a(t, 1u | ((1u << D) << 8) | ((1u << (2 * D)) << 16), 0u);
  } else {
    return (t & 0xFFu) | (((t >> 8) & 0xFFu) << D) | (((t >> 16) & 0xFFu) << (2 * D));
  }
}

// q of packed pixel y = r | g << 8 | b << 16 (upper byte ignored).
template <int D>
__device__ __forceinline__ uint32_t planar_code(uint32_t y) {
  return planar_from_masked<D>((y >> (8 - D)) & byte_mask(D));
}

__host__ __device__ __forceinline__ uint32_t planar_code_rt(uint32_t r, uint32_t g, uint32_t b, int d) {
  const int s = 8 - d;
  return (r >> s) | ((g >> s) << d) | ((b >> s) << (2 * d));
}

// Path code (interleaved, Alg. 1 order) -> planar code, and back.
__host__ __device__ __forceinline__ uint32_t path_to_planar(uint32_t c, int d) {
  uint32_t r = 0, g = 0, b = 0;
  for (int l = 0; l < d; ++l) {
    uint32_t digit = (c >> (3 * (d - 1 - l))) & 7u;
    r = (r << 1) | (digit >> 2);
    g = (g << 1) | ((digit >> 1) & 1u);
    b = (b << 1) | (digit & 1u);
  }
  return r | (g << d) | (b << (2 * d));
}

__host__ __device__ __forceinline__ uint32_t planar_to_path(uint32_t q, int d) {
  const uint32_t m = (1u << d) - 1u;
  uint32_t r = q & m, g = (q >> d) & m, b = (q >> (2 * d)) & m;
  uint32_t c = 0;
  for (int l = 0; l < d; ++l) {
    int bit = d - 1 - l;
    c = (c << 3) | (((r >> bit) & 1u) << 2) | (((g >> bit) & 1u) << 1) | ((b >> bit) & 1u);
  }
  return c;
}

// Region of pixel (y, x); bw = ceil(W / block) for block regions.
__host__ __device__ __forceinline__ int64_t region_of(int y, int x, int W, int kind, int block, int bw) {
  if (kind == OCQ_REGION_FRAME) return 0;
  if (kind == OCQ_REGION_BLOCK) return (int64_t)(y / block) * bw + x / block;
  return (int64_t)y * W + x;
}

// Bit-sliced counter: add the 32 one-bit values of `x` into planes[0..P).
__device__ __forceinline__ void planes_add(uint32_t *planes, int P, uint32_t x) {
  for (int k = 0; k < P && x; ++k) {
    uint32_t t = planes[k] & x;
    planes[k] ^= x;
    x = t;
  }
}

// Lanes whose bit-sliced count (planes[0..P)) is >= T (T < 2^P).
__device__ __forceinline__ uint32_t planes_ge(const uint32_t *planes, int P, uint32_t T) {
  uint32_t gt = 0, eq = 0xFFFFFFFFu;
  for (int k = P - 1; k >= 0; --k) {
    uint32_t c = planes[k];
    if ((T >> k) & 1u) {
      eq &= c;
    } else {
      gt |= eq & c;
      eq &= ~c;
    }
  }
  return gt | eq;
}

// Streaming (evict-first) 16-byte global load / store.
__device__ __forceinline__ uint4 ld_stream16(const void *p) {
  uint4 v;
  asm volatile("ld.global.cs.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ void st_stream16(void *p, uint4 v) {
  asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

// Packed pixel k (0..15) of a 48-byte group held as 12 words.
template <int K>
__device__ __forceinline__ uint32_t group_pixel(const uint32_t (&w)[12]) {
  constexpr int o = 3 * K, i = o / 4, s = o % 4;
  constexpr uint32_t sel = (uint32_t)(s | ((s + 1) << 4) | ((s + 2) << 8) | ((s + 2) << 12));
  if constexpr (i + 1 < 12)
    return __byte_perm(w[i], w[i + 1], sel);
  else
    return __byte_perm(w[i], 0u, sel);
}

// ---- kernel launchers (build.cu, classify.cu, transform.cu) -------------------
ocq_status launch_path_code(const uint8_t *rgb, int64_t npix, int depth, uint32_t *codes, cudaStream_t st);
ocq_status launch_build(const uint8_t *frames, int N, ocq_model *m, cudaStream_t st);
ocq_status launch_build_groups(const uint8_t *frames, int N, int group, ocq_model *m, cudaStream_t st);
ocq_status launch_classify(const ocq_model *m, const uint8_t *frames, int F, uint8_t *mask, cudaStream_t st);
ocq_status launch_occupancy(const uint8_t *frames, int n, int H, int W, int kind, int block, int depth,
                            uint64_t *occ, cudaStream_t st);
ocq_status launch_export(const uint32_t *bits, int64_t R, int depth, uint64_t *dst, cudaStream_t st);
ocq_status launch_import(const uint64_t *src, int64_t R, int depth, uint32_t *bits, cudaStream_t st);
// out[w] = OR of occ[p * words + w] over p < parts (exported layout).
ocq_status launch_or_parts(const uint64_t *occ, int parts, int64_t words, uint64_t *out, cudaStream_t st);
// model[w] = (number of the N rows of occ holding bit) >= T, word-wise over
// nwords internal words (occ: N * nwords, N <= 65535).
ocq_status launch_merge_counts(const uint32_t *occ, int N, int64_t nwords, uint32_t T, uint32_t *model,
                               cudaStream_t st);
// Serving windows (window.cu): per-frame occupancy kept in place of frames.
// Leaf bitsets of n whole frames (internal order) ORed into occ[f * wpr32(d)]
// (occ zero beforehand).
ocq_status launch_frame_occupancy(const uint8_t *frames, int n, int H, int W, int depth, uint32_t *occ,
                                  cudaStream_t st);
// Pixel and block regions with depth <= 5, N <= 255 (blocks: b <= 16) keep a
// ring of per-pixel u16 leaf codes.
bool window_codes_apply(int kind, int block, int depth, int N, int H, int W);
ocq_status launch_window_codes(const uint8_t *frames, int64_t npix, int depth, uint16_t *codes, cudaStream_t st);
ocq_status launch_window_count_update(uint32_t *slot, uint32_t *fresh, uint16_t *counts, int depth,
                                      cudaStream_t st);
ocq_status launch_window_counts_init(const uint32_t *ring, int N, int depth, uint16_t *counts, cudaStream_t st);
ocq_status launch_window_threshold(const uint16_t *counts, int depth, uint32_t T, uint32_t *bits, cudaStream_t st);
// Re-merge of a pixel or block model in place from N code planes.
ocq_status launch_remerge_codes(const uint16_t *ring, int N, ocq_model *m, cudaStream_t st);
bool classify_take_timeout();
bool build_take_timeout();
// Block regions that the one-warp-per-region build handles (b <= 16, N <= 255).
bool block_warp_ok(int N, int H, int W, int b);
// Block regions that the 16 x 16 warp-tile build handles (b in {8, 16}, ...),
// and its selection (1: used where it applies; 0: one warp per region).
bool block_tile_ok(int N, int H, int W, int b, int depth, const void *frames);
bool block_fs_ok(int N, int H, int W, int b, int depth, const void *frames);
bool block_r8_ok(int N, int H, int W, int b, int depth, const void *frames);
// While one is alive on this thread, the default block build form picks for
// work per region rather than for filling the GPU (the batched forms, where
// other streams' kernels run beside it).
struct SharedGpuScope {
  SharedGpuScope();
  ~SharedGpuScope();
  SharedGpuScope(const SharedGpuScope &) = delete;
  SharedGpuScope &operator=(const SharedGpuScope &) = delete;
  bool prev;
};
int block_build_form_count();
int block_build_form_selected();
bool block_build_form_select(int v);

// Kernel variants the tuner can choose between (per-pixel tiled classify,
// staged per-pixel build).
int classify_variant_count();
int classify_variant_selected();
bool classify_variant_select(int v);
void classify_variant_describe(int v, int *nw, int *ppt, int *stages, int *fps, int *ws);
int deep_variant_count();
int deep_variant_selected();
bool deep_variant_select(int v);
void deep_variant_describe(int v, int *pxl, int *pf, int *cps);
int list_form_count();
int list_form_selected();
bool list_form_select(int v);
// List models: per-pixel regions of depth 4-5 whose candidate build keeps at
// most 8 leaves per location (N <= 255, floor(N / T) <= 8) are built as the
// kept-leaf index alone, unless switched off (form 0).
bool list_model_applies(int kind, int depth, int N, int T);
int list_model_form();
bool list_model_select(int v);
ocq_status launch_export_list(const uint16_t *kept, int64_t R, int depth, uint64_t *dst, cudaStream_t st);
ocq_status launch_import_list(const uint64_t *src, int64_t R, int depth, int limit, uint16_t *kept,
                              unsigned int *overflow, cudaStream_t st);
// Entries of a list that can hold a kept leaf when floor(N/T) <= 8: 2, 4 or 8.
inline int list_length(int N, int T) {
  const int k = N / T;
  return k <= 2 ? 2 : k <= 4 ? 4 : 8;
}
// Device bytes of a model built from N frames with threshold T (list model,
// rows with or without the index): what ocq_build_model allocates.
size_t model_bytes(int H, int W, ocq_region region, int depth, int N, int T);
void list_form_describe(int v, int *nw, int *ppt, int *stages, int *fps);
int block_form_count();
int block_form_selected();
bool block_form_select(int v);
int build_variant_count();
int build_variant_selected();
bool build_variant_select(int v);
void build_variant_describe(int v, int *nt, int *fps, int *stages, int *tensor);

}  // namespace ocq
