// S1 as a standalone kernel, S2 per-frame occupancy, and the translation
// between the library's planar leaf order and the path-code order of the
// public bitset layout (export / import).
#include "ocq_internal.cuh"

namespace ocq {

// ---- S1: path code per pixel (Alg. 1 walk, pruned at depth d, Sec. 2) --------
__global__ void path_code_kernel(const uint8_t *__restrict__ rgb, int64_t npix, int d, uint32_t *__restrict__ codes) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t r = rgb[3 * i], g = rgb[3 * i + 1], b = rgb[3 * i + 2];
    uint32_t c = 0;
    for (int l = 0; l < d; ++l) {  // level l reads bit 7-l of each channel
      const int bit = 7 - l;
      c = (c << 3) | (((r >> bit) & 1u) << 2) | (((g >> bit) & 1u) << 1) | ((b >> bit) & 1u);
    }
    codes[i] = c;
  }
}

static unsigned grid_for(int64_t work, int threads, int per_sm = 16) {
  int64_t b = (work + threads - 1) / threads;
  int64_t cap = (int64_t)sm_count() * per_sm;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

ocq_status launch_path_code(const uint8_t *rgb, int64_t npix, int depth, uint32_t *codes, cudaStream_t st) {
  path_code_kernel<<<grid_for(npix, 256), 256, 0, st>>>(rgb, npix, depth, codes);
  count_launch();
  return cuda_status(cudaGetLastError(), "path_code_kernel");
}

// ---- planar <-> path translation ------------------------------------------------
// Both orders are permutations of the same 3d bits, so for codes a, b with
// disjoint bits perm(a | b) = perm(a) | perm(b).  A 64-bit output word holds path
// codes 64k | j (j < 64): its planar codes are path_to_planar(64k) | off[j],
// with the 64-entry table off[j] = path_to_planar(j).  Likewise for import.

// Output word k of a region row in the public layout: bits of path codes
// 64k .. 64k+63 (fewer when d <= 1).
__global__ void export_kernel(const uint32_t *__restrict__ bits, int64_t R, int d, int64_t wpr_in, int64_t wpr_out,
                              uint64_t *__restrict__ dst) {
  __shared__ uint32_t off[64];
  const uint32_t ncodes = 1u << (3 * d);
  const uint32_t n = ncodes < 64 ? ncodes : 64;
  if (threadIdx.x < 64) off[threadIdx.x] = threadIdx.x < n ? path_to_planar(threadIdx.x, d) : 0u;
  __syncthreads();
  const int64_t total = R * wpr_out;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / wpr_out, k = i % wpr_out;
    const uint32_t *row = bits + r * wpr_in;
    const uint32_t base = path_to_planar((uint32_t)(k * 64), d);
    uint64_t out = 0;
    for (uint32_t j = 0; j < n; ++j) {
      const uint32_t q = base | off[j];
      out |= (uint64_t)((__ldg(row + (q >> 5)) >> (q & 31)) & 1u) << j;
    }
    dst[i] = out;
  }
}

// Internal word w of a region row: bits of planar codes 32w .. 32w+31.
__global__ void import_kernel(const uint64_t *__restrict__ src, int64_t R, int d, int64_t wpr_in, int64_t wpr_out,
                              uint32_t *__restrict__ bits) {
  __shared__ uint32_t off[32];
  const uint32_t ncodes = 1u << (3 * d);
  const uint32_t n = ncodes < 32 ? ncodes : 32;
  if (threadIdx.x < 32) off[threadIdx.x] = threadIdx.x < n ? planar_to_path(threadIdx.x, d) : 0u;
  __syncthreads();
  const int64_t total = R * wpr_out;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / wpr_out, w = i % wpr_out;
    const uint64_t *row = src + r * wpr_in;
    const uint32_t base = planar_to_path((uint32_t)(w * 32), d);
    uint32_t out = 0;
    for (uint32_t j = 0; j < n; ++j) {
      const uint32_t c = base | off[j];
      out |= (uint32_t)((__ldg(row + (c >> 6)) >> (c & 63)) & 1u) << j;
    }
    bits[i] = out;
  }
}

ocq_status launch_export(const uint32_t *bits, int64_t R, int depth, uint64_t *dst, cudaStream_t st) {
  const int64_t total = R * wpr64(depth);
  export_kernel<<<grid_for(total, 256, 8), 256, 0, st>>>(bits, R, depth, wpr32(depth), wpr64(depth), dst);
  count_launch();
  return cuda_status(cudaGetLastError(), "export_kernel");
}

// List models: a warp per location row.  Lane e < 8 turns list entry e into
// its path code (or an out-of-range value for kKeptNone) and the warp shares
// the 8 codes; then lane l writes the row's output words l, l + 32, .. : word
// k holds the bits of the codes in 64k .. 64k+63.  Stores are coalesced and
// each location's list is read once.
__global__ void export_list_kernel(const uint16_t *__restrict__ kept, int64_t R, int d, int64_t wpr_out,
                                   uint64_t *__restrict__ dst) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < R; r += warps) {
    uint32_t mine = 0xFFFFFFFFu;
    if (lane < 8) {
      const uint32_t q = __ldg(kept + r * 8 + lane);
      if (q != kKeptNone) mine = planar_to_path(q, d);
    }
    uint32_t c[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) c[e] = __shfl_sync(0xFFFFFFFFu, mine, e);
    for (int64_t k = lane; k < wpr_out; k += 32) {
      uint64_t out = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (c[e] != 0xFFFFFFFFu && (int64_t)(c[e] >> 6) == k) out |= 1ull << (c[e] & 63);
      dst[r * wpr_out + k] = out;
    }
  }
}

ocq_status launch_export_list(const uint16_t *kept, int64_t R, int depth, uint64_t *dst, cudaStream_t st) {
  export_list_kernel<<<grid_for(R * 32, 256, 8), 256, 0, st>>>(kept, R, depth, wpr64(depth), dst);
  count_launch();
  return cuda_status(cudaGetLastError(), "export_list_kernel");
}

// Import into a list model: a warp per location row.  Lane l scans the row's
// words l, l + 32, ..; the set bits (path codes) become planar codes, placed by
// a warp prefix sum over the lanes' counts; the rest of the 8 entries are
// kKeptNone.  A row with more than `limit` (<= 8) bits cannot be a list of
// this model: it sets *overflow and its list is left padded.
__global__ void import_list_kernel(const uint64_t *__restrict__ src, int64_t R, int d, int64_t wpr_in, int limit,
                                   uint16_t *__restrict__ kept, unsigned int *overflow) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < R; r += warps) {
    const uint64_t *row = src + r * wpr_in;
    int n = 0;
    for (int64_t k = lane; k < wpr_in; k += 32) n += __popcll(__ldg(row + k));
    int before = n;  // inclusive prefix sum of the counts over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xFFFFFFFFu, before, o);
      if (lane >= o) before += v;
    }
    const int total = __shfl_sync(0xFFFFFFFFu, before, 31);
    uint16_t *list = kept + r * 8;
    if (total > limit) {
      if (lane == 0) atomicExch(overflow, 1u);
      if (lane < 8) list[lane] = kKeptNone;
      continue;
    }
    int at = before - n;  // this lane's first entry
    for (int64_t k = lane; k < wpr_in && at < before; k += 32) {
      uint64_t w = __ldg(row + k);
      while (w) {
        const int b = __ffsll((long long)w) - 1;
        w &= w - 1;
        list[at++] = (uint16_t)path_to_planar((uint32_t)(k * 64 + b), d);
      }
    }
    if (lane >= total && lane < 8) list[lane] = kKeptNone;
  }
}

ocq_status launch_import_list(const uint64_t *src, int64_t R, int depth, int limit, uint16_t *kept,
                              unsigned int *overflow, cudaStream_t st) {
  import_list_kernel<<<grid_for(R * 32, 256, 8), 256, 0, st>>>(src, R, depth, wpr64(depth), limit, kept, overflow);
  count_launch();
  return cuda_status(cudaGetLastError(), "import_list_kernel");
}

// Union of `parts` leaf-set bitsets per row (exported layout): the tree of a
// region whose pixels were split into parts holds a leaf iff some part's tree
// does (Alg. 1 inserts every pixel of the region into one tree).
__global__ void or_parts_kernel(const uint64_t *__restrict__ occ, int parts, int64_t words,
                                uint64_t *__restrict__ out) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
    uint64_t v = 0;
    for (int p = 0; p < parts; ++p) v |= occ[(int64_t)p * words + w];
    out[w] = v;
  }
}

ocq_status launch_or_parts(const uint64_t *occ, int parts, int64_t words, uint64_t *out, cudaStream_t st) {
  or_parts_kernel<<<grid_for(words, 256, 8), 256, 0, st>>>(occ, parts, words, out);
  count_launch();
  return cuda_status(cudaGetLastError(), "or_parts_kernel");
}

ocq_status launch_import(const uint64_t *src, int64_t R, int depth, uint32_t *bits, cudaStream_t st) {
  const int64_t total = R * wpr32(depth);
  import_kernel<<<grid_for(total, 256, 8), 256, 0, st>>>(src, R, depth, wpr64(depth), wpr32(depth), bits);
  count_launch();
  return cuda_status(cudaGetLastError(), "import_kernel");
}

// ---- S2 standalone: per-frame, per-region leaf sets ----------------------------
__global__ void occupancy_kernel(const uint8_t *__restrict__ frames, int64_t npix, int H, int W, int kind, int block,
                                 int d, int64_t R, int64_t wpr, uint32_t *__restrict__ occ) {
  const int64_t hw = (int64_t)H * W;
  const int bw = kind == OCQ_REGION_BLOCK ? (W + block - 1) / block : 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = i / hw, p = i % hw;
    const int y = (int)(p / W), x = (int)(p % W);
    const uint32_t q = planar_code_rt(frames[3 * i], frames[3 * i + 1], frames[3 * i + 2], d);
    uint32_t *word = occ + (f * R + region_of(y, x, W, kind, block, bw)) * wpr + (q >> 5);
    const uint32_t m = 1u << (q & 31);
    if (!(*(volatile uint32_t *)word & m)) atomicOr(word, m);
  }
}

ocq_status launch_occupancy(const uint8_t *frames, int n, int H, int W, int kind, int block, int depth, uint64_t *occ,
                            cudaStream_t st) {
  const int64_t R = region_count(H, W, kind, block);
  const int64_t rows = (int64_t)n * R;
  const size_t bytes = (size_t)rows * (size_t)wpr32(depth) * sizeof(uint32_t);
  uint32_t *tmp = nullptr;
  ocq_status rc = cuda_status(malloc_async((void **)&tmp, bytes, st), "occupancy scratch");
  if (rc != OCQ_OK) return rc;
  rc = cuda_status(cudaMemsetAsync(tmp, 0, bytes, st), "occupancy scratch clear");
  if (rc == OCQ_OK) {
    const int64_t npix = (int64_t)n * H * W;
    occupancy_kernel<<<grid_for(npix, 256), 256, 0, st>>>(frames, npix, H, W, kind, block, depth, R, wpr32(depth),
                                                           tmp);
    count_launch();
    rc = cuda_status(cudaGetLastError(), "occupancy_kernel");
  }
  if (rc == OCQ_OK) rc = launch_export(tmp, rows, depth, occ, st);
  cudaFreeAsync(tmp, st);
  return rc;
}

}  // namespace ocq
