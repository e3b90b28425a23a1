// Grouped launches of the batched form: one launch per kernel body and
// template (depth, block size, counter or list length) over every camera
// stream that uses it.  Each stream owns a contiguous range of the launch's
// CTAs (its virtual grid: CTA vb of vg, found by a binary search on the CTA
// index), and each CTA runs the body the plain per-stream kernel runs, with
// that kernel's CTA shape, shared memory and residency, so a stream's result
// is the plain path's bit for bit.  The launches of one class of streams form
// a chain (builds, then classification) in one branch of the batch's graph;
// the classes' branches run concurrently.
#include <algorithm>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "build_bodies.cuh"
#include "classify_bodies.cuh"
#include "grouped.cuh"

namespace ocq {

// Set when a bounded wait of a grouped body gives up; read and cleared by
// grouped_take_timeout().
__device__ unsigned int g_grouped_timeout;

__device__ __forceinline__ const GSeg &seg_of(const GSeg *__restrict__ g, int n, int64_t &vb) {
  int lo = 0, hi = n - 1;  // the last segment whose first CTA is <= blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g[mid].cta0 <= (int64_t)blockIdx.x)
      lo = mid;
    else
      hi = mid - 1;
  }
  vb = (int64_t)blockIdx.x - g[lo].cta0;
  return g[lo];
}

// ---- whole frame -------------------------------------------------------------------

template <int D>
__global__ void __launch_bounds__(256) g_occ_frame(const GSeg *__restrict__ g, int n) {
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  occ_frame_body<D>(s.in, s.hw, 0, kGroupOccChunk, s.occ, vb % s.aux, vb / s.aux);
}

__global__ void __launch_bounds__(256) g_merge(const GSeg *__restrict__ g, int n) {
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  planes_merge_body(s.occ, s.N, s.units, nullptr, s.P, 1, 1, (uint32_t)s.T, s.model, vb, s.vg);
}

template <int D>
__global__ void __launch_bounds__(256) g_cls_frame(const GSeg *__restrict__ g, int n) {
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  classify_frame_body<D>(s.in, (int64_t)s.F * s.hw, s.model, s.mask, vb, s.vg);
}

// ---- blocks ----------------------------------------------------------------------

template <int D, int B>
__global__ void __launch_bounds__(BlockTileCfg<D, B>::WPC * 32, BlockTileCfg<D, B>::MINB)
    g_block_tile(const GSeg *__restrict__ g, int n) {
  extern __shared__ __align__(16) uint8_t gt_smem[];
  constexpr int WB = BlockTileCfg<D, B>::WARP_SMEM;
  uint8_t *wsm = gt_smem + (threadIdx.x >> 5) * WB;
  for (int i = threadIdx.x & 31; i < WB / 4; i += 32) reinterpret_cast<uint32_t *>(wsm)[i] = 0u;
  __syncwarp();
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  constexpr int WPC = BlockTileCfg<D, B>::WPC;
  build_block_tile_body<D, B, BlockTileCfg<D, B>::PF>(s.in, s.N, s.H, s.W, s.bw, (uint32_t)s.T, s.model,
                                                      vb * WPC + (threadIdx.x >> 5), s.units, s.vg * WPC, wsm);
}

template <int D, int PPL>
__global__ void __launch_bounds__(256) g_block_warp(const GSeg *__restrict__ g, int n) {
  extern __shared__ uint32_t gw_tabs[];
  constexpr int S = WarpTableCfg<D>::S;
  uint32_t *tab = gw_tabs + (threadIdx.x >> 5) * S;
  for (int i = threadIdx.x & 31; i < S; i += 32) tab[i] = 0u;
  __syncwarp();
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  build_block_warp_body<D, PPL>(s.in, s.N, s.H, s.W, s.block, s.bw, (uint32_t)s.T, s.model,
                                vb * 8 + (threadIdx.x >> 5), s.units, s.vg * 8, tab);
}

template <int D, int B>
__global__ void __launch_bounds__(256, BlockFsCfg<D, B>::MINB) g_block_fs(const GSeg *__restrict__ g, int n) {
  extern __shared__ __align__(16) uint32_t gf_smem[];
  for (int i = threadIdx.x; i < BlockFsCfg<D, B>::SMEM / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(gf_smem)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  build_block_fs_body<D, B>(s.in, s.N, s.H, s.W, s.bw, (uint32_t)s.T, s.model, s.units, vb, s.vg, gf_smem);
}

template <int D>
__global__ void __launch_bounds__(256, 4) g_block_r8(const GSeg *__restrict__ g, int n) {
  extern __shared__ __align__(16) uint8_t gr_smem[];
  constexpr int WB = BlockR8CfgD<D>::WARP_SMEM;
  uint8_t *wsm = gr_smem + (threadIdx.x >> 5) * WB;
  for (int i = threadIdx.x & 31; i < WB / 4; i += 32) reinterpret_cast<uint32_t *>(wsm)[i] = 0u;
  __syncwarp();
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  build_block_r8_body<D>(s.in, s.N, s.H, s.W, s.bw, (uint32_t)s.T, s.model, vb * 8 + (threadIdx.x >> 5), s.units,
                         s.vg * 8, wsm);
}

// items u = chunk * tiles + tile over frames [chunk * fchunk, + fchunk)
template <int D>
__global__ void __launch_bounds__(256) g_block_tb(const GSeg *__restrict__ g, int n) {
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  const int64_t tiles = s.aux;
  for (int64_t u = vb * 8 + (threadIdx.x >> 5); u < s.units; u += s.vg * 8) {
    const int64_t c = u / tiles;
    const int f0 = (int)(c * s.aux2);
    classify_block_tb_body<D, 4>(s.in, s.F, s.H, s.W, s.block, s.bw, s.aux3, s.model, s.mask, u - c * tiles, f0,
                                 f0 + s.aux2, s.ftab, s.mtab, s.ctab);
  }
}

// ---- pixel locations ----------------------------------------------------------------

template <int D, int NT, int FPS, int S>
__global__ void __launch_bounds__(NT + 32) g_pixel_ws_build(const GSeg *__restrict__ g, int n) {
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  build_pixel_ws_body<D, NT, FPS, S, false, false>(s.in, s.N, s.hw, s.units, (uint32_t)s.T, s.model, nullptr, vb,
                                                   s.vg, &g_grouped_timeout);
}

template <int D, int NW, int PPT, int S, int FPS>
__global__ void __launch_bounds__(NW * 32 + 32, 1) g_pixel_ws_cls(const GSeg *__restrict__ g, int n) {
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  classify_pixel_ws_body<D, NW, PPT, S, FPS>(s.in, s.F, s.hw, s.units, s.model, s.mask, vb, s.vg,
                                             &g_grouped_timeout, nullptr, s.ftab, s.mtab, s.ctab);
}

template <int D, int KM>
__global__ void __launch_bounds__(128) g_pixel_mg(const GSeg *__restrict__ g, int n) {
  extern __shared__ __align__(16) uint8_t gm_smem[];
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  leaf_t<D> *codes = reinterpret_cast<leaf_t<D> *>(gm_smem) + (size_t)(threadIdx.x >> 5) * s.N * 32;
  const int64_t tile = vb * 4 + (threadIdx.x >> 5);
  if (tile * 32 >= s.hw) return;  // whole warps only
  build_pixel_mg_body<D, KM>(s.in, s.N, s.hw, (uint32_t)s.T, s.model, tile, codes, 1, s.kept);
}

template <int D, int KL>
__global__ void __launch_bounds__(128) g_pixel_list(const GSeg *__restrict__ g, int n) {
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  for (int64_t t = vb * 4 + (threadIdx.x >> 5); t < s.units; t += s.vg * 4)
    classify_pixel_list_body<D, 8, KL>(s.in, s.F, s.hw, s.kept, s.mask, t, s.ftab, s.mtab, s.ctab);
}

// ---- serving ticks ------------------------------------------------------------------

// Per-pixel leaf codes of one frame into its window slot (segment: in = frame,
// kept = the slot's codes, units = pixels).
template <int D>
__global__ void __launch_bounds__(256) g_codes(const GSeg *__restrict__ g, int n) {
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  const int64_t tid = vb * blockDim.x + threadIdx.x, nth = s.vg * blockDim.x;
  const uint8_t *frames = s.in;
  uint16_t *codes = s.kept;
  const int64_t npix = s.units;
  int64_t tail = 0;
  if ((reinterpret_cast<uintptr_t>(frames) & 15) == 0 && (reinterpret_cast<uintptr_t>(codes) & 15) == 0) {
    const int64_t ng = npix >> 4;
    for (int64_t q = tid; q < ng; q += nth) {
      uint32_t w[12];
      load_group_masked<D, true>(frames + q * 48, w);
      uint32_t c[8];
      static_for<0, 8>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        c[k] = planar_from_masked<D>(group_pixel<2 * k>(w)) | (planar_from_masked<D>(group_pixel<2 * k + 1>(w)) << 16);
      });
      reinterpret_cast<uint4 *>(codes + q * 16)[0] = make_uint4(c[0], c[1], c[2], c[3]);
      reinterpret_cast<uint4 *>(codes + q * 16)[1] = make_uint4(c[4], c[5], c[6], c[7]);
    }
    tail = ng << 4;
  }
  for (int64_t p = tail + tid; p < npix; p += nth) {
    const uint8_t *px = frames + p * 3;
    codes[p] = (uint16_t)planar_code_rt(px[0], px[1], px[2], D);
  }
}

// A camera's F entering frames, in order: bitset j (occ + j * units words)
// replaces ring slot (aux + j) mod N and each leaf's count follows; the
// bitsets are cleared for the next tick (segment: model = ring, kept = counts,
// units = words per bitset, aux2 = leaves per word).
__global__ void __launch_bounds__(256) g_count(const GSeg *__restrict__ g, int n) {
  int64_t vb;
  const GSeg &s = seg_of(g, n, vb);
  uint16_t *counts = s.kept;
  for (int64_t w = vb * blockDim.x + threadIdx.x; w < s.units; w += s.vg * blockDim.x)
    for (int j = 0; j < s.F; ++j) {
      uint32_t *slot = s.model + ((s.aux + j) % s.N) * s.units;
      uint32_t *fresh = s.occ + (int64_t)j * s.units;
      const uint32_t old = slot[w], nw = fresh[w];
      uint32_t diff = old ^ nw;
      while (diff) {
        const int i = __ffs(diff) - 1;
        diff &= diff - 1;
        if (i < s.aux2) counts[w * 32 + i] += ((nw >> i) & 1u) ? (uint16_t)1 : (uint16_t)0xFFFFu;
      }
      slot[w] = nw;
      fresh[w] = 0u;
    }
}

// ---- host side ----------------------------------------------------------------------

using GKern = void (*)(const GSeg *, int);

struct KInfo {
  GKern fn = nullptr;
  int threads = 256;
  size_t smem = 0;  // fixed part; GK_PIX_MG adds its per-stream codes
};

template <int D>
static KInfo kinfo_d(int kind, int b) {
  KInfo k;
  constexpr int WPR = D == 1 ? 1 : 1 << (3 * D - 5);
  switch (kind) {
    case GK_OCC:
      if constexpr (D <= 6) k.fn = g_occ_frame<D>, k.smem = (size_t)WPR * 4;
      break;
    case GK_CLS_FRAME:
      if constexpr (D <= 6) k.fn = g_cls_frame<D>, k.smem = (size_t)WPR * (D <= 4 ? 32 : 1) * 4;
      break;
    case GK_BLOCK_TILE:
      if constexpr (D >= 2 && D <= 5) {
        if (b == 16)
          k.fn = g_block_tile<D, 16>, k.threads = BlockTileCfg<D, 16>::WPC * 32,
          k.smem = (size_t)BlockTileCfg<D, 16>::WPC * BlockTileCfg<D, 16>::WARP_SMEM;
        if (b == 8)
          k.fn = g_block_tile<D, 8>, k.threads = BlockTileCfg<D, 8>::WPC * 32,
          k.smem = (size_t)BlockTileCfg<D, 8>::WPC * BlockTileCfg<D, 8>::WARP_SMEM;
      }
      break;
    case GK_BLOCK_FS:
      if constexpr (D >= 2 && D <= 5) {
        if (b == 16) k.fn = g_block_fs<D, 16>, k.smem = BlockFsCfg<D, 16>::SMEM;
        if (b == 8) k.fn = g_block_fs<D, 8>, k.smem = BlockFsCfg<D, 8>::SMEM;
      }
      break;
    case GK_BLOCK_R8:
      if constexpr (D == 4 || D == 5)
        if (b == 8) k.fn = g_block_r8<D>, k.smem = (size_t)8 * BlockR8CfgD<D>::WARP_SMEM;
      break;
    case GK_BLOCK_WARP:
      if constexpr (D <= 5) {
        k.smem = (size_t)8 * WarpTableCfg<D>::S * 4;
        k.fn = b == 1 ? g_block_warp<D, 1> : b == 2 ? g_block_warp<D, 2> : b == 4 ? g_block_warp<D, 4> : g_block_warp<D, 8>;
      }
      break;
    case GK_BLOCK_TB:
      if constexpr (D <= 5) k.fn = g_block_tb<D>;
      break;
    case GK_PIX_WS_BUILD:
      if constexpr (D <= 3) k.fn = g_pixel_ws_build<D, 128, 8, 3>, k.threads = 160,
                            k.smem = WsBuildCfg<D, 128, 8, 3, false>::SMEM;
      break;
    case GK_PIX_WS_CLS:
      if constexpr (D <= 3) k.fn = g_pixel_ws_cls<D, 4, 8, 4, 4>, k.threads = 160,
                            k.smem = TiledCfg<D, 4, 8, 4, 4>::SMEM + 4 * 8;
      break;
    case GK_PIX_MG:
      if constexpr (D == 4 || D == 5) {
        k.threads = 128;
        k.fn = b == 1 ? g_pixel_mg<D, 1> : b == 2 ? g_pixel_mg<D, 2> : b == 4 ? g_pixel_mg<D, 4> : g_pixel_mg<D, 8>;
      }
      break;
    case GK_PIX_LIST:
      if constexpr (D == 4 || D == 5) {
        k.threads = 128;
        k.fn = b == 2 ? g_pixel_list<D, 2> : b == 4 ? g_pixel_list<D, 4> : g_pixel_list<D, 8>;
      }
      break;
    case GK_CODES:
      if constexpr (D <= 5) k.fn = g_codes<D>;
      break;
    default:
      break;
  }
  return k;
}

static KInfo kinfo(int kind, int a, int b) {
  if (kind == GK_MERGE || kind == GK_COUNT) {
    KInfo k;
    k.fn = kind == GK_MERGE ? g_merge : g_count;
    return k;
  }
  switch (a) {
    case 1: return kinfo_d<1>(kind, b);
    case 2: return kinfo_d<2>(kind, b);
    case 3: return kinfo_d<3>(kind, b);
    case 4: return kinfo_d<4>(kind, b);
    case 5: return kinfo_d<5>(kind, b);
    case 6: return kinfo_d<6>(kind, b);
    default: return KInfo();
  }
}

// CTAs of the kernel resident on the whole GPU (at least one per SM).
static int64_t resident(const KInfo &k, size_t smem) {
  if (smem > 48 * 1024) cudaFuncSetAttribute((const void *)k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)k.fn, k.threads, smem);
  return (int64_t)sm_count() * (per > 0 ? per : 1);
}

static int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }


ocq_status grouped_plan(const std::vector<GStreamIn> &in, std::vector<GLaunch> &out, std::vector<int> &fallback) {
  out.clear();
  fallback.clear();
  // launch key -> index in `out`, created in the order the phases run
  std::vector<GLaunch> L;
  auto launch = [&](int kind, int a, int b) -> GLaunch & {
    for (GLaunch &x : L)
      if (x.kind == kind && x.a == a && x.b == b) return x;
    GLaunch x;
    x.kind = kind, x.a = a, x.b = b, x.branch = 0;
    L.push_back(x);
    return L.back();
  };
  auto base = [](const GStreamIn &x, const uint8_t *src) {
    GSeg s;
    memset(&s, 0, sizeof s);
    s.tab = -1;
    s.in = src, s.mask = x.mask, s.model = x.model, s.occ = x.occ, s.kept = x.kept;
    s.hw = (int64_t)x.H * x.W;
    s.N = x.N, s.F = x.F, s.H = x.H, s.W = x.W, s.block = x.block, s.T = x.T;
    s.bw = x.block > 0 ? (x.W + x.block - 1) / x.block : 1;
    int P = 0;
    for (uint32_t v = (uint32_t)x.N; v; v >>= 1) ++P;
    s.P = P;
    return s;
  };
  const int64_t sms = sm_count();
  for (int i = 0; i < (int)in.size(); ++i) {
    const GStreamIn &x = in[i];
    const int64_t hw = (int64_t)x.H * x.W;
    const int d = x.depth;
    const uintptr_t tm = reinterpret_cast<uintptr_t>(x.test) | reinterpret_cast<uintptr_t>(x.mask);
    if (x.kind == OCQ_REGION_FRAME) {
      if (d > 6 || x.N > 255) {
        fallback.push_back(i);
        continue;
      }
      GSeg o = base(x, x.train);
      o.aux = cdiv64(hw, kGroupOccChunk), o.vg = o.aux * x.N;
      launch(GK_OCC, d, 0).segs.push_back(o);
      GSeg m = base(x, x.train);
      m.units = wpr32(d), m.vg = std::max<int64_t>(1, std::min<int64_t>(64, cdiv64(m.units, 256)));
      launch(GK_MERGE, 0, 0).segs.push_back(m);
      if (x.F > 0) {
        GSeg c = base(x, x.test);
        c.units = (int64_t)x.F * hw;
        launch(GK_CLS_FRAME, d, 0).segs.push_back(c);
      }
    } else if (x.kind == OCQ_REGION_BLOCK) {
      const bool cls_ok = x.F == 0 || (x.block % 4 == 0 && x.W % 4 == 0 && (tm & 3) == 0);
      const bool r8 = block_r8_ok(x.N, x.H, x.W, x.block, d, x.train);
      const bool fs = !r8 && block_fs_ok(x.N, x.H, x.W, x.block, d, x.train);
      const bool tile = !r8 && !fs && block_tile_ok(x.N, x.H, x.W, x.block, d, x.train);
      const bool warp = !r8 && !fs && !tile && d <= 5 && block_warp_ok(x.N, x.H, x.W, x.block);
      if (!cls_ok || (!r8 && !fs && !tile && !warp)) {
        fallback.push_back(i);
        continue;
      }
      GSeg bld = base(x, x.train);
      if (r8) {
        bld.units = cdiv64(x.H, 8) * (x.W / 8);
        launch(GK_BLOCK_R8, d, 8).segs.push_back(bld);
      } else if (fs) {
        bld.units = x.block == 8 && d == 5 ? cdiv64(x.H, 8) * (x.W / 8) : cdiv64(x.H, 16) * cdiv64(x.W, 16);
        launch(GK_BLOCK_FS, d, x.block).segs.push_back(bld);
      } else if (tile) {
        bld.units = cdiv64(x.H, 16) * cdiv64(x.W, 16);
        launch(GK_BLOCK_TILE, d, x.block).segs.push_back(bld);
      } else {
        const int npx = x.block * x.block;
        const int ppl = npx <= 32 ? 1 : npx <= 64 ? 2 : npx <= 128 ? 4 : 8;
        bld.units = region_count(x.H, x.W, OCQ_REGION_BLOCK, x.block);
        launch(GK_BLOCK_WARP, d, ppl).segs.push_back(bld);
      }
      if (x.F > 0) {
        GSeg c = base(x, x.test);
        const int bh = (x.H + x.block - 1) / x.block;
        c.aux3 = (x.W + 127) / 128;
        const int64_t tiles = (int64_t)bh * c.aux3 * x.block;
        const int64_t cap = sms * 4 * 8;
        int chunks = 1;
        if (tiles < 2 * cap) chunks = (int)std::min<int64_t>(cdiv64(2 * cap, tiles), (x.F + 15) / 16);
        if (chunks < 1) chunks = 1;
        const int fchunk = (x.F + chunks - 1) / chunks;
        chunks = (x.F + fchunk - 1) / fchunk;
        c.aux = tiles, c.aux2 = fchunk, c.units = tiles * chunks;
        launch(GK_BLOCK_TB, d, 0).segs.push_back(c);
      }
    } else {
      const uintptr_t all = tm | reinterpret_cast<uintptr_t>(x.train);
      if (d <= 3 && x.N <= 255 && x.T <= 255 && hw % 1024 == 0 && (all & 15) == 0 && x.model) {
        GSeg bld = base(x, x.train);
        bld.units = hw / 128;
        launch(GK_PIX_WS_BUILD, d, 0).segs.push_back(bld);
        if (x.F > 0) {
          GSeg c = base(x, x.test);
          c.units = hw / 1024;
          launch(GK_PIX_WS_CLS, d, 0).segs.push_back(c);
        }
      } else if ((d == 4 || d == 5) && x.N <= 255 && x.km > 0 && x.kl > 0 && x.kept &&
                 (x.F == 0 || (hw % 4 == 0 && (tm & 3) == 0))) {
        GSeg bld = base(x, x.train);
        bld.vg = cdiv64(hw, 128);
        launch(GK_PIX_MG, d, x.km).segs.push_back(bld);
        if (x.F > 0) {
          GSeg c = base(x, x.test);
          c.units = cdiv64(hw, 128);
          launch(GK_PIX_LIST, d, x.kl).segs.push_back(c);
        }
      } else {
        fallback.push_back(i);
        continue;
      }
    }
  }
  // Phase order inside each branch follows the GroupKind order (builds before
  // classification); launches of one kind keep ascending template arguments.
  std::stable_sort(L.begin(), L.end(), [](const GLaunch &p, const GLaunch &q) {
    if (p.branch != q.branch) return p.branch < q.branch;
    if (p.kind != q.kind) return p.kind < q.kind;
    return p.a != q.a ? p.a < q.a : p.b < q.b;
  });
  for (GLaunch &x : L) {
    KInfo k = kinfo(x.kind, x.a, x.b);
    if (!k.fn) {
      set_error("internal: no grouped kernel for kind %d (%d, %d)", x.kind, x.a, x.b);
      return OCQ_EINVAL;
    }
    x.threads = k.threads;
    x.smem = k.smem;
    if (x.kind == GK_PIX_MG)
      for (const GSeg &s : x.segs) x.smem = std::max(x.smem, (size_t)4 * s.N * 32 * 2);
    if (x.smem > 227 * 1024) {
      set_error("internal: grouped kernel needs %zu bytes of shared memory", x.smem);
      return OCQ_ENOTSUP;
    }
    const int64_t cap = resident(k, x.smem);
    int64_t cta = 0;
    for (GSeg &s : x.segs) {
      switch (x.kind) {
        case GK_CLS_FRAME: s.vg = std::max<int64_t>(1, std::min<int64_t>(cdiv64(s.units, 16 * 256), cap)); break;
        case GK_BLOCK_TILE: s.vg = std::max<int64_t>(1, std::min<int64_t>(cdiv64(s.units, x.threads / 32), cap)); break;
        case GK_BLOCK_FS: s.vg = std::max<int64_t>(1, std::min<int64_t>(s.units, cap)); break;
        case GK_BLOCK_R8: s.vg = std::max<int64_t>(1, std::min<int64_t>(cdiv64(s.units, 8), cap)); break;
        case GK_BLOCK_WARP:
        case GK_BLOCK_TB: s.vg = std::max<int64_t>(1, std::min<int64_t>(cdiv64(s.units, 8), cap)); break;
        case GK_PIX_WS_BUILD: s.vg = std::max<int64_t>(1, std::min<int64_t>(s.units, cap)); break;
        case GK_PIX_WS_CLS: s.vg = std::max<int64_t>(1, std::min<int64_t>(s.units * s.F, cap)); break;
        case GK_PIX_LIST: s.vg = std::max<int64_t>(1, std::min<int64_t>(cdiv64(s.units, 4), cap)); break;
        default: break;  // GK_OCC, GK_MERGE, GK_PIX_MG: set above
      }
    }
    for (GSeg &s : x.segs) {
      s.cta0 = cta;
      cta += s.vg;
    }
    x.grid = cta;
  }
  out.swap(L);
  return OCQ_OK;
}

// Sets CTA shapes, shared memory and per-segment virtual grids of planned
// launches (segments' units filled in).
static ocq_status finish_plan(std::vector<GLaunch> &L) {
  for (GLaunch &x : L) {
    KInfo k = kinfo(x.kind, x.a, x.b);
    if (!k.fn) {
      set_error("internal: no grouped kernel for kind %d (%d, %d)", x.kind, x.a, x.b);
      return OCQ_EINVAL;
    }
    x.threads = k.threads;
    x.smem = k.smem;
    const int64_t cap = resident(k, x.smem);
    int64_t cta = 0;
    for (GSeg &s : x.segs) {
      switch (x.kind) {
        case GK_CLS_FRAME:
        case GK_CODES: s.vg = std::max<int64_t>(1, std::min<int64_t>(cdiv64(s.units, 16 * 256), cap)); break;
        case GK_BLOCK_TB: s.vg = std::max<int64_t>(1, std::min<int64_t>(cdiv64(s.units, 8), cap)); break;
        case GK_PIX_WS_CLS: s.vg = std::max<int64_t>(1, std::min<int64_t>(s.units * s.F, cap)); break;
        case GK_PIX_LIST: s.vg = std::max<int64_t>(1, std::min<int64_t>(cdiv64(s.units, 4), cap)); break;
        case GK_COUNT: s.vg = std::max<int64_t>(1, std::min<int64_t>(cdiv64(s.units, 256), 64)); break;
        default: break;  // GK_OCC: set by the planner
      }
      s.cta0 = cta;
      cta += s.vg;
    }
    x.grid = cta;
  }
  return OCQ_OK;
}

ocq_status grouped_plan_tick(const std::vector<GFrameIn> &in, std::vector<GLaunch> &out, std::vector<int> &single,
                             std::vector<const void *> &ptrs) {
  out.clear();
  single.clear();
  ptrs.clear();
  std::vector<GLaunch> L;
  auto launch = [&](int kind, int a, int b) -> GLaunch & {
    for (GLaunch &x : L)
      if (x.kind == kind && x.a == a && x.b == b) return x;
    GLaunch x;
    x.kind = kind, x.a = a, x.b = b;
    L.push_back(x);
    return L.back();
  };
  // a camera's frames of the tick, in order (a camera has one model)
  std::vector<std::vector<int>> of;
  std::vector<char> coded(in.size(), 0);
  std::unordered_map<const ocq_model *, int> cam_of;
  for (int i = 0; i < (int)in.size(); ++i) {
    auto it = cam_of.emplace(in[i].model, (int)of.size()).first;
    if (it->second == (int)of.size()) of.emplace_back();
    std::vector<int> &fr = of[it->second];
    if ((int)fr.size() != in[i].j) return OCQ_EINVAL;  // frames of a camera come in order
    fr.push_back(i);
  }
  for (const std::vector<int> &fr : of) {
    const GFrameIn &f = in[fr[0]];
    const ocq_model *m = f.model;
    const int d = m->depth;
    const int64_t hw = (int64_t)m->H * m->W;
    uintptr_t al = 0;
    for (int i : fr) al |= reinterpret_cast<uintptr_t>(in[i].frame) | reinterpret_cast<uintptr_t>(in[i].mask);
    GSeg c;
    memset(&c, 0, sizeof c);
    c.in = f.frame, c.mask = f.mask, c.model = m->bits, c.kept = m->kept, c.hw = hw;
    c.N = m->N, c.F = (int)fr.size(), c.H = m->H, c.W = m->W, c.block = m->block, c.T = m->T;
    c.bw = m->block > 0 ? (m->W + m->block - 1) / m->block : 1;
    c.tab = (int64_t)ptrs.size();
    int kind = -1, a = 0, b = 0;
    if (m->kind == OCQ_REGION_BLOCK && d <= 5 && m->block % 4 == 0 && m->W % 4 == 0 && (al & 3) == 0) {
      c.aux3 = (m->W + 127) / 128;
      c.aux = (int64_t)((m->H + m->block - 1) / m->block) * c.aux3 * m->block;  // tiles
      c.aux2 = c.F, c.units = c.aux;
      kind = GK_BLOCK_TB, a = d;
    } else if (m->kind == OCQ_REGION_PIXEL && d <= 3 && m->bits && hw % 1024 == 0 && (al & 15) == 0) {
      c.units = hw / 1024;
      kind = GK_PIX_WS_CLS, a = d;
    } else if (m->kind == OCQ_REGION_PIXEL && (d == 4 || d == 5) && m->kept && m->kept_len > 0 && hw % 4 == 0 &&
               (al & 3) == 0) {
      c.units = (hw + 127) / 128;
      kind = GK_PIX_LIST, a = d, b = m->kept_len;
    }
    if (kind >= 0) {
      for (int i : fr) ptrs.push_back(in[i].frame);
      for (int i : fr) ptrs.push_back(in[i].mask);
      if (f.win == 2) {  // the classify writes the frames' codes into their window slots
        c.codes = 1;
        for (int i : fr) {
          ptrs.push_back(reinterpret_cast<uint16_t *>(in[i].ring) + in[i].slot * hw);
          coded[i] = 1;
        }
      }
      launch(kind, a, b).segs.push_back(c);
      continue;
    }
    for (int i : fr) {  // one segment per frame (whole frames: a frame's pixels are contiguous)
      const GFrameIn &g = in[i];
      if (m->kind == OCQ_REGION_FRAME && d <= 6) {
        GSeg e = c;
        e.in = g.frame, e.mask = g.mask, e.F = 1, e.tab = -1, e.units = hw;
        launch(GK_CLS_FRAME, d, 0).segs.push_back(e);
      } else {
        single.push_back(i);
      }
    }
  }
  // the window: codes (where the classify did not write them), or bitsets
  // then the counts (after every classify)
  for (size_t i = 0; i < in.size(); ++i) {
    const GFrameIn &f = in[i];
    if (coded[i]) continue;
    const ocq_model *m = f.model;
    const int64_t hw = (int64_t)m->H * m->W;
    GSeg w;
    memset(&w, 0, sizeof w);
    w.tab = -1;
    w.in = f.frame, w.hw = hw, w.N = f.N, w.F = 1;
    if (f.win == 2) {
      w.kept = reinterpret_cast<uint16_t *>(f.ring) + f.slot * hw;
      w.units = hw;
      launch(GK_CODES, m->depth, 0).segs.push_back(w);
    } else {
      const int64_t wpr = wpr32(m->depth);
      w.occ = f.fresh + (int64_t)f.j * wpr;
      w.aux = (hw + kGroupOccChunk - 1) / kGroupOccChunk, w.vg = w.aux;
      launch(GK_OCC, m->depth, 0).segs.push_back(w);
    }
  }
  for (const GFrameIn &f : in) {
    if (f.win != 1 || f.j != 0) continue;
    GSeg k;
    memset(&k, 0, sizeof k);
    k.tab = -1;
    k.model = reinterpret_cast<uint32_t *>(f.ring), k.occ = f.fresh, k.kept = f.counts;
    k.units = wpr32(f.model->depth), k.aux = f.slot, k.N = f.N, k.F = f.m;
    k.aux2 = f.model->depth == 1 ? 8 : 32;
    launch(GK_COUNT, 0, 0).segs.push_back(k);
  }
  // classify launches first, then the window's (a camera's counts after its bitsets)
  std::stable_sort(L.begin(), L.end(), [](const GLaunch &p, const GLaunch &q) {
    auto rank = [](int k) { return k == GK_COUNT ? 3 : k == GK_OCC || k == GK_CODES ? 2 : 1; };
    return rank(p.kind) < rank(q.kind);
  });
  ocq_status rc = finish_plan(L);
  if (rc == OCQ_OK) out.swap(L);
  return rc;
}

ocq_status grouped_launch(const GLaunch &L, cudaStream_t st) {
  if (L.grid <= 0 || L.segs.empty()) return OCQ_OK;
  if (L.grid > 0x7FFFFFFFLL) {
    set_error("grouped launch of %lld CTAs", (long long)L.grid);
    return OCQ_ENOTSUP;
  }
  KInfo k = kinfo(L.kind, L.a, L.b);
  const GSeg *segs = L.dev;
  int n = (int)L.segs.size();
  void *args[] = {(void *)&segs, (void *)&n};
  cudaError_t e = cudaLaunchKernel((const void *)k.fn, dim3((unsigned)L.grid), dim3((unsigned)L.threads), args, L.smem, st);
  count_launch();
  return cuda_status(e, "grouped kernel");
}

bool grouped_take_timeout() {
  unsigned int flag = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&flag, g_grouped_timeout, sizeof flag) != cudaSuccess) return false;
  if (flag) cudaMemcpyToSymbol(g_grouped_timeout, &zero, sizeof zero);
  return flag != 0;
}

}  // namespace ocq
