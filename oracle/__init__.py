"""CPU oracle for the octree background model (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import this package.  The product path (the CUDA library and
its binding) never imports it and shares no code with it.

* ``octree_oracle.c`` -- pointer octrees built with Store Color (Alg. 1),
  merged with Merge Trees (Alg. 2), queried with Check Color (Alg. 3); see
  its header for the readings taken where the paper is open.
* ``brute.py`` -- Python set-based restatement of the same result for tiny
  inputs: a leaf is a colour's d most significant bits per channel (Sec. 2),
  the model keeps leaves seen in at least T training frames (Sec. 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "octree_oracle.c")
_SO = os.path.join(_HERE, "liboctree_oracle.so")
_lock = threading.Lock()
_lib = None

REGION_FRAME, REGION_BLOCK, REGION_PIXEL = 0, 1, 2


def build_command():
    return ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", _SO, _SRC]


def build() -> None:
    """Compile the oracle with gcc (in-tree)."""
    if os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return
    r = subprocess.run(build_command(), capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("building the oracle failed:\n" + r.stdout + r.stderr)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i32, i64, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            lib.oracle_region_count.restype = i64
            lib.oracle_region_count.argtypes = [i32, i32, i32, i32]
            lib.oracle_words_per_region.restype = i64
            lib.oracle_words_per_region.argtypes = [i32]
            lib.oracle_run.restype = i32
            lib.oracle_run.argtypes = [vp, i32, vp, i32, i32, i32, i32, i32, i32, i32, vp, i64, vp, vp]
            lib.oracle_build.restype = i32
            lib.oracle_build.argtypes = [vp, i32, i32, i32, i32, i32, i32, i32, vp, i64, vp]
            lib.oracle_classify.restype = i32
            lib.oracle_classify.argtypes = [vp, i32, i32, i32, i32, i32, vp, i32, vp, i64, vp]
            lib.oracle_tree_stats.restype = i32
            lib.oracle_tree_stats.argtypes = [vp, i32, i32, i32, i32, i32, vp, vp, vp]
            lib.oracle_leaf_codes.restype = i32
            lib.oracle_leaf_codes.argtypes = [vp, i64, i32, vp]
            lib.oracle_run_groups.restype = i32
            lib.oracle_run_groups.argtypes = [vp, i32, i32, vp, i32, i32, i32, i32, i32, i32, i32, vp, i64, vp, vp]
            lib.oracle_redraw.restype = i32
            lib.oracle_redraw.argtypes = [vp, i64, i32, vp]
            lib.oracle_confusion.restype = i32
            lib.oracle_confusion.argtypes = [vp, vp, i64, i64, vp]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(rc, what):
    if rc == 1:
        raise ValueError(f"{what}: bad arguments")
    if rc == 2:
        raise MemoryError(f"{what}: allocation failed")
    if rc != 0:
        raise RuntimeError(f"{what}: error {rc}")


def region_count(H, W, kind, block=0) -> int:
    return int(_load().oracle_region_count(H, W, kind, block))


def words_per_region(depth) -> int:
    return int(_load().oracle_words_per_region(depth))


def _frames(a, name):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    if a.ndim != 4 or a.shape[3] != 3:
        raise ValueError(f"{name} must be uint8[n, H, W, 3]")
    return a


def _regions(regions):
    if regions is None:
        return None, 0
    r = np.ascontiguousarray(regions, dtype=np.int64)
    return r, r.size


def _gathered_size(H, W, kind, block, regs, F):
    total = 0
    for r in regs:
        if kind == REGION_FRAME:
            total += H * W
        elif kind == REGION_BLOCK:
            bw = (W + block - 1) // block
            by, bx = divmod(int(r), bw)
            total += (min(H, by * block + block) - by * block) * (min(W, bx * block + block) - bx * block)
        else:
            total += 1
    return total * F


def run(train, depth, T, kind, block=0, test=None, regions=None, group=1):
    """Build the merged model from ``train`` (uint8[N,H,W,3]) and classify
    ``test`` with Check Color on the merged trees.  ``group`` > 1 builds one
    tree per group of that many consecutive frames (Sec. 3) and T counts
    groups.

    Returns ``(model, mask)``: ``model`` is uint64[n_regions, words_per_region]
    (rows follow ``regions`` when given); ``mask`` is uint8[F,H,W] (or, with
    ``regions``, the gathered 1-D array: per region, per frame, its pixels in
    row-major order), or None without ``test``."""
    lib = _load()
    train = _frames(train, "train")
    N, H, W, _ = train.shape
    regs, nreg = _regions(regions)
    R = region_count(H, W, kind, block)
    if R < 1:
        raise ValueError("bad region")
    nrows = nreg if regs is not None else R
    model = np.zeros((nrows, words_per_region(depth)), dtype=np.uint64)
    mask = None
    F = 0
    if test is not None:
        test = _frames(test, "test")
        F = test.shape[0]
        if test.shape[1:3] != (H, W):
            raise ValueError("test frames must match training frame size")
        if regs is None:
            mask = np.zeros((F, H, W), dtype=np.uint8)
        else:
            mask = np.zeros(_gathered_size(H, W, kind, block, regs, F), dtype=np.uint8)
    rc = lib.oracle_run_groups(train.ctypes.data, N, group, _ptr(test), F, H, W, kind, block, depth, T,
                               _ptr(regs), nreg, model.ctypes.data, _ptr(mask))
    _check(rc, "oracle_run_groups")
    return model, mask


def build_model(train, depth, T, kind, block=0, regions=None):
    return run(train, depth, T, kind, block, None, regions)[0]


def classify(model, frames, depth, kind, block=0, regions=None):
    """Check Color (Alg. 3) of ``frames`` against an exported ``model``
    (rows follow ``regions`` when given)."""
    lib = _load()
    frames = _frames(frames, "frames")
    F, H, W, _ = frames.shape
    model = np.ascontiguousarray(model, dtype=np.uint64)
    regs, nreg = _regions(regions)
    if regs is None:
        mask = np.zeros((F, H, W), dtype=np.uint8)
    else:
        mask = np.zeros(_gathered_size(H, W, kind, block, regs, F), dtype=np.uint8)
    rc = lib.oracle_classify(model.ctypes.data, H, W, kind, block, depth, frames.ctypes.data, F,
                             _ptr(regs), nreg, mask.ctypes.data)
    _check(rc, "oracle_classify")
    return mask


def tree_stats(frame, depth, kind, block=0):
    """Per region of one frame: (leaves, sum of leaf pixel counters, nodes)."""
    lib = _load()
    frame = _frames(frame[None] if frame.ndim == 3 else frame, "frame")
    _, H, W, _ = frame.shape
    R = region_count(H, W, kind, block)
    leaves = np.zeros(R, dtype=np.int64)
    sums = np.zeros(R, dtype=np.int64)
    nodes = np.zeros(R, dtype=np.int64)
    rc = lib.oracle_tree_stats(frame.ctypes.data, H, W, kind, block, depth, leaves.ctypes.data,
                               sums.ctypes.data, nodes.ctypes.data)
    _check(rc, "oracle_tree_stats")
    return leaves, sums, nodes


def leaf_codes(rgb, depth):
    """Path code (child indices from the root, Alg. 1) of each colour in
    ``rgb`` (uint8[n, 3])."""
    lib = _load()
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8).reshape(-1, 3)
    out = np.zeros(rgb.shape[0], dtype=np.uint32)
    rc = lib.oracle_leaf_codes(rgb.ctypes.data, rgb.shape[0], depth, out.ctypes.data)
    _check(rc, "oracle_leaf_codes")
    return out


def redraw(rgb, depth):
    """Each colour of ``rgb`` (uint8[..., 3]) redrawn as its leaf in a tree
    pruned at ``depth`` levels (Sec. 2, Fig. 2)."""
    lib = _load()
    a = np.ascontiguousarray(rgb, dtype=np.uint8)
    out = np.empty_like(a)
    rc = lib.oracle_redraw(a.ctypes.data, a.size // 3, depth, out.ctypes.data)
    _check(rc, "oracle_redraw")
    return out


def confusion(mask, gt):
    """Per frame {Tp, Fp, Tn, Fn} of a foreground mask (uint8[F, H, W], non-zero
    = foreground) against ground truth of the same shape (Sec. 5)."""
    lib = _load()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    g = np.ascontiguousarray(gt, dtype=np.uint8)
    if m.shape != g.shape or m.ndim < 2:
        raise ValueError("mask and gt must have the same shape [F, ...]")
    F = m.shape[0]
    out = np.zeros((F, 4), dtype=np.uint64)
    rc = lib.oracle_confusion(m.ctypes.data, g.ctypes.data, F, m[0].size, out.ctypes.data)
    _check(rc, "oracle_confusion")
    return out


def f_scores(counts):
    """The paper's F0 (Sec. 5): P0 = Tn / (Tn + Fn), R0 = Tn / (Tn + Fp),
    F0 = 2 P0 R0 / (P0 + R0); also the foreground F1 = 2 Tp / (2 Tp + Fp + Fn).
    ``counts`` = {Tp, Fp, Tn, Fn} (summed over frames when 2-D).  A ratio with
    a zero denominator is taken as 1 (nothing to get wrong)."""
    c = np.asarray(counts, dtype=np.float64)
    if c.ndim == 2:
        c = c.sum(axis=0)
    tp, fp, tn, fn = c
    p0 = tn / (tn + fn) if tn + fn else 1.0
    r0 = tn / (tn + fp) if tn + fp else 1.0
    f0 = 2 * p0 * r0 / (p0 + r0) if p0 + r0 else 0.0
    f1 = 2 * tp / (2 * tp + fp + fn) if 2 * tp + fp + fn else 1.0
    return {"P0": p0, "R0": r0, "F0": f0, "F1": f1}
