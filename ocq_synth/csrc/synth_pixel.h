/*
 * Seeded synthetic video for the octree background model: one pixel at a time.
 *
 * This header holds input generation only, none of the method's arithmetic
 * (no path codes, trees, counts or lookups).  It is compiled twice from this
 * one source: by gcc into the host generator library and by nvcc into the
 * device generator library, so frames made on either side are byte-identical.
 *
 * A scene is a flat int32 array (the "blob") built by ocq_synth/scene.py:
 * a 32-word header followed by small tables.  Every per-pixel random value is
 * a counter-based splitmix64 hash of (seed, stream, tag, frame, y, x), so any
 * frame can be regenerated on demand in any order.
 *
 * Frames are HWC RGB8 with no row padding; frame f starts at f*H*W*3.
 */
#ifndef OCQ_SYNTH_PIXEL_H
#define OCQ_SYNTH_PIXEL_H

#include <stdint.h>

#ifdef __CUDACC__
#define SYNTH_HD __host__ __device__ __forceinline__
#else
#define SYNTH_HD static inline
#endif

/* Header word indices of a scene blob. */
enum {
  SY_MAGIC = 0,     /* 0x4F435153 */
  SY_KIND = 1,      /* 1 clusters, 2 swaying palette, 3 bimodal per pixel */
  SY_H = 2,
  SY_W = 3,
  SY_NTRAIN = 4,    /* frames [0, NTRAIN) carry background only */
  SY_NFRAMES = 5,   /* frames covered by the tables */
  SY_SEED_LO = 6,
  SY_SEED_HI = 7,
  SY_NOISE = 8,     /* +- noise amplitude per channel */
  SY_PATCH = 9,     /* clusters: patch edge in pixels */
  SY_NCENTRES = 10,
  SY_SHAPE = 11,    /* 0 rectangle, 1 ellipse, 2 textured disc */
  SY_NOBJ = 12,
  SY_OFF_CENTRES = 13,
  SY_OFF_DRIFT = 14,
  SY_OFF_OBJS = 15, /* (NFRAMES-NTRAIN) x NOBJ x 4 geometry words */
  SY_OFF_COLOURS = 16, /* NOBJ x 3 */
  SY_STREAM = 17,
  SY_HEADER_WORDS = 32
};

#define SY_MAGIC_VALUE 0x4F435153

SYNTH_HD uint64_t synth_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* One 64-bit value per (seed, tag, f, y, x). */
SYNTH_HD uint64_t synth_hash(uint64_t seed, uint32_t tag, uint64_t f, uint32_t y, uint32_t x) {
  uint64_t z = synth_mix(seed ^ ((uint64_t)(tag + 1u) * 0x9E3779B97F4A7C15ull));
  uint64_t key = (f << 40) ^ ((uint64_t)y << 20) ^ (uint64_t)x;
  return synth_mix(z + key * 0xD1B54A32D192ED03ull);
}

SYNTH_HD int synth_clamp8(int v) { return v < 0 ? 0 : (v > 255 ? 255 : v); }

SYNTH_HD uint64_t synth_seed(const int32_t *S) {
  uint64_t s = ((uint64_t)(uint32_t)S[SY_SEED_HI] << 32) | (uint64_t)(uint32_t)S[SY_SEED_LO];
  return synth_mix(s ^ ((uint64_t)(uint32_t)S[SY_STREAM] * 0xA24BAED4963EE407ull));
}

/* Writes the RGB bytes of pixel (f, y, x) to rgb[0..2]; *gt = 1 when a
 * foreground object covers the pixel, else 0. */
SYNTH_HD void synth_pixel(const int32_t *S, uint64_t seed, int64_t f, int y, int x,
                          uint8_t *rgb, uint8_t *gt) {
  int c[3];
  const int kind = S[SY_KIND];
  const int A = S[SY_NOISE];
  if (kind == 1) {
    /* fixed patches, each showing one of NCENTRES cluster colours + uniform noise */
    const int P = S[SY_PATCH];
    uint64_t hp = synth_hash(seed, 1, 0, (uint32_t)(y / P), (uint32_t)(x / P));
    int k = (int)((uint32_t)(hp >> 32) % (uint32_t)S[SY_NCENTRES]);
    const int32_t *C = S + S[SY_OFF_CENTRES] + 3 * k;
    uint64_t hn = synth_hash(seed, 2, (uint64_t)f, (uint32_t)y, (uint32_t)x);
    for (int ch = 0; ch < 3; ++ch)
      c[ch] = C[ch] + (int)((uint32_t)(hn >> (16 * ch)) % (uint32_t)(2 * A + 1)) - A;
  } else if (kind == 2) {
    /* each location alternates between k in {2,3} palette colours; global drift */
    uint64_t hk = synth_hash(seed, 3, 0, (uint32_t)y, (uint32_t)x);
    uint32_t k = 2u + (uint32_t)(hk & 1u);
    uint64_t hc = synth_hash(seed, 4, (uint64_t)f, (uint32_t)y, (uint32_t)x);
    uint32_t pick = (uint32_t)(hc >> 32) % k;
    uint64_t hp = synth_hash(seed, 5, pick, (uint32_t)(y >> 3), (uint32_t)(x >> 3));
    uint64_t ho = synth_hash(seed, 6, pick, (uint32_t)y, (uint32_t)x);
    int drift = S[S[SY_OFF_DRIFT] + (int)f];
    for (int ch = 0; ch < 3; ++ch)
      c[ch] = (int)((hp >> (8 * ch)) & 255u) + (int)((uint32_t)(ho >> (16 * ch)) % (uint32_t)(2 * A + 1)) - A + drift;
  } else {
    /* two seeded modes per pixel, mixing weight in [0.30, 0.70], noise */
    uint64_t m0 = synth_hash(seed, 7, 0, (uint32_t)y, (uint32_t)x);
    uint64_t m1 = synth_hash(seed, 7, 1, (uint32_t)y, (uint32_t)x);
    uint32_t w = 77u + (uint32_t)(synth_hash(seed, 8, 0, (uint32_t)y, (uint32_t)x) >> 32) % 103u;
    uint64_t hc = synth_hash(seed, 9, (uint64_t)f, (uint32_t)y, (uint32_t)x);
    uint64_t m = ((uint32_t)(hc & 255u) < w) ? m0 : m1;
    for (int ch = 0; ch < 3; ++ch)
      c[ch] = (int)((m >> (8 * ch)) & 255u) + (int)((uint32_t)(hc >> (8 + 16 * ch)) % (uint32_t)(2 * A + 1)) - A;
  }
  uint8_t g = 0;
  const int ntrain = S[SY_NTRAIN];
  const int nobj = S[SY_NOBJ];
  if (f >= ntrain && nobj > 0 && f < S[SY_NFRAMES]) {
    const int32_t *G = S + S[SY_OFF_OBJS] + (int64_t)(f - ntrain) * nobj * 4;
    const int shape = S[SY_SHAPE];
    for (int o = 0; o < nobj; ++o) {
      const int32_t *q = G + 4 * o;
      int inside;
      if (shape == 0) {
        inside = x >= q[0] && x < q[0] + q[2] && y >= q[1] && y < q[1] + q[3];
      } else {
        int64_t dx = x - q[0], dy = y - q[1];
        if (shape == 1) {
          int64_t a = q[2], b = q[3];
          inside = dx * dx * b * b + dy * dy * a * a <= a * a * b * b;
        } else {
          inside = dx * dx + dy * dy <= (int64_t)q[2] * q[2];
        }
      }
      if (inside) {
        g = 1;
        if (shape == 2) {
          uint64_t ht = synth_hash(seed, 10, (uint64_t)f, (uint32_t)y, (uint32_t)x);
          for (int ch = 0; ch < 3; ++ch) c[ch] = (int)((ht >> (8 * ch)) & 255u);
        } else {
          const int32_t *col = S + S[SY_OFF_COLOURS] + 3 * o;
          for (int ch = 0; ch < 3; ++ch) c[ch] = col[ch];
        }
      }
    }
  }
  for (int ch = 0; ch < 3; ++ch) rgb[ch] = (uint8_t)synth_clamp8(c[ch]);
  *gt = g;
}

#endif
