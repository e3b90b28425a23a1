"""Scene descriptions (small tables) for the seeded synthetic video.

A scene is a flat ``int32`` numpy array: a 32-word header (layout in
``csrc/synth_pixel.h``) followed by the cluster-centre, drift, object-geometry
and object-colour tables.  Per-pixel content is produced from the scene by the
host or device generator (``ocq_synth.fill_host`` / ``fill_device``).

The tables here are drawn from a counter-based splitmix64 stream written in
plain Python integers, so a scene is identical on every machine.  Nothing in
this module computes any part of the octree method.

Workload recipes (sizes and distributions follow the paper's setting of a
static camera with a moving foreground and a swaying background, Sec. 3-5):

* ``clusters``: background of ``n_centres`` colour clusters (centres uniform in
  [6, 249]^3), each ``patch`` x ``patch`` patch showing one cluster, +-``noise``
  uniform per channel per frame.  Test frames add moving rectangles (10-40 px at
  160x120, scaled with the frame) of colours more than 24 (L-inf) from every centre,
  moving linearly and bouncing off the walls.
* ``sway``: each location alternates between 2-3 palette colours (palette per
  8x8 cell, +-``noise`` per location), the pick hashed per frame, plus a global
  drift round(8 sin(2 pi t / n_frames)).  Test frames add random-walk ellipses
  (semi-axes 8-30 px at 320x240, steps of at most 4 px per frame) of random colour.
* ``bimodal``: every pixel has two seeded modes, a mixing weight uniform in
  [0.30, 0.70] and +-``noise`` per channel.  Test frames add textured discs of
  radius 65-81 px (at 1080 rows) moving linearly with wall bounces; the 10 discs
  of a 1920x1080 frame cover about 8% of it.
"""
from __future__ import annotations

import math

import numpy as np

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
MAGIC = 0x4F435153
HEADER_WORDS = 32

KIND_CLUSTERS, KIND_SWAY, KIND_BIMODAL = 1, 2, 3
SHAPE_RECT, SHAPE_ELLIPSE, SHAPE_DISC = 0, 1, 2


def _mix(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


class TableRng:
    """Counter-based splitmix64 stream used only for the small scene tables."""

    def __init__(self, seed: int, stream: int, tag: int):
        self.base = _mix((seed ^ (stream * 0xA24BAED4963EE407) ^ ((tag + 1) * GOLDEN)) & M64)
        self.i = 0

    def u64(self) -> int:
        self.i += 1
        return _mix(self.base + self.i * GOLDEN)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + self.u64() % (hi - lo + 1)


def _bounce(pos: int, vel: int, lo: int, hi: int):
    pos += vel
    if pos < lo:
        pos, vel = 2 * lo - pos, -vel
    if pos > hi:
        pos, vel = 2 * hi - pos, -vel
    pos = min(max(pos, lo), hi)
    return pos, vel


def make_scene(kind: str, H: int, W: int, n_train: int, n_test: int, seed: int,
               stream: int = 0, n_obj: int | None = None) -> np.ndarray:
    """Build the scene blob for ``n_train`` background frames followed by
    ``n_test`` frames with foreground objects."""
    if H < 1 or W < 1 or n_train < 0 or n_test < 0:
        raise ValueError("bad scene size")
    n_frames = n_train + n_test
    hdr = np.zeros(HEADER_WORDS, dtype=np.int64)
    tables: list[np.ndarray] = []
    off = HEADER_WORDS

    def put(arr) -> int:
        nonlocal off
        a = np.asarray(arr, dtype=np.int64).ravel()
        at = off
        tables.append(a)
        off += a.size
        return at

    hdr[0] = MAGIC
    hdr[2], hdr[3], hdr[4], hdr[5] = H, W, n_train, n_frames
    hdr[6], hdr[7] = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    hdr[17] = stream
    rng = TableRng(seed, stream, 100)
    if kind == "clusters":
        hdr[1] = KIND_CLUSTERS
        hdr[8], hdr[9], hdr[10] = 6, 20, 6
        centres = [[rng.randint(6, 249) for _ in range(3)] for _ in range(6)]
        hdr[13] = put(centres)
        nobj = 2 if n_obj is None else n_obj
        scale = max(1.0, min(H / 120.0, W / 160.0))
        geo = np.zeros((n_test, nobj, 4), dtype=np.int64)
        cols = []
        for o in range(nobj):
            while True:
                col = [rng.randint(0, 255) for _ in range(3)]
                if all(max(abs(col[c] - ce[c]) for c in range(3)) > 24 for ce in centres):
                    break
            cols.append(col)
            w = min(W, int(round(rng.randint(10, 40) * scale)))
            h = min(H, int(round(rng.randint(10, 40) * scale)))
            x0, y0 = rng.randint(0, W - w), rng.randint(0, H - h)
            vs = max(1, int(round(3 * scale)))
            vx, vy = rng.randint(-vs, vs), rng.randint(-vs, vs)
            if vx == 0 and vy == 0:
                vx = 1
            for t in range(n_test):
                geo[t, o] = (x0, y0, w, h)
                x0, vx = _bounce(x0, vx, 0, W - w)
                y0, vy = _bounce(y0, vy, 0, H - h)
        hdr[11], hdr[12] = SHAPE_RECT, nobj
        hdr[15] = put(geo)
        hdr[16] = put(cols if cols else np.zeros(0))
    elif kind == "sway":
        hdr[1] = KIND_SWAY
        hdr[8] = 12
        drift = [int(round(8.0 * math.sin(2.0 * math.pi * t / max(1, n_frames)))) for t in range(n_frames)]
        hdr[14] = put(drift)
        nobj = 5 if n_obj is None else n_obj
        scale = max(1.0, min(H / 240.0, W / 320.0))
        geo = np.zeros((n_test, nobj, 4), dtype=np.int64)
        cols = []
        for o in range(nobj):
            cols.append([rng.randint(0, 255) for _ in range(3)])
            a = int(round(rng.randint(8, 30) * scale))
            b = int(round(rng.randint(8, 30) * scale))
            cx, cy = rng.randint(0, W - 1), rng.randint(0, H - 1)
            step = max(1, int(round(4 * scale)))
            for t in range(n_test):
                geo[t, o] = (cx, cy, a, b)
                cx = min(max(cx + rng.randint(-step, step), 0), W - 1)
                cy = min(max(cy + rng.randint(-step, step), 0), H - 1)
        hdr[11], hdr[12] = SHAPE_ELLIPSE, nobj
        hdr[15] = put(geo)
        hdr[16] = put(cols if cols else np.zeros(0))
    elif kind == "bimodal":
        hdr[1] = KIND_BIMODAL
        hdr[8] = 4
        nobj = 10 if n_obj is None else n_obj
        scale = max(0.05, H / 1080.0)
        geo = np.zeros((n_test, nobj, 4), dtype=np.int64)
        for o in range(nobj):
            r = max(1, int(round(rng.randint(65, 81) * scale)))
            cx, cy = rng.randint(0, W - 1), rng.randint(0, H - 1)
            vs = max(1, int(round(8 * scale)))
            vx, vy = rng.randint(-vs, vs), rng.randint(-vs, vs)
            for t in range(n_test):
                geo[t, o] = (cx, cy, r, 0)
                cx, vx = _bounce(cx, vx, 0, W - 1)
                cy, vy = _bounce(cy, vy, 0, H - 1)
        hdr[11], hdr[12] = SHAPE_DISC, nobj
        hdr[15] = put(geo)
    else:
        raise ValueError(f"unknown scene kind {kind!r}")
    blob = np.concatenate([hdr] + tables) if tables else hdr
    return blob.astype(np.int32)


def scene_hw(scene: np.ndarray):
    return int(scene[2]), int(scene[3])
