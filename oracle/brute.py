"""Brute-force restatement of the model with Python sets (TEST INFRASTRUCTURE).

For tiny inputs only.  A leaf of a tree pruned at height d is identified with
the colour's d most significant bits per channel (Sec. 2: a leaf at level d
keeps d original bits, the rest are zero), a tuple (r >> (8-d), g >> (8-d),
b >> (8-d)).  The merged model of a region keeps the leaves that occur in at
least T of the N per-frame trees (Alg. 2 kept exactly these, since every tree
that holds a leaf also holds all of its ancestors); Check Color (Alg. 3)
reports a pixel as background when its leaf is in the model.

This module shares nothing with ``octree_oracle.c``: it never forms a path
code, and it enumerates regions from their definition.
"""
from __future__ import annotations

from collections import Counter


def region_of(y, x, H, W, kind, block):
    if kind == 0:
        return 0
    if kind == 1:
        return (y // block) * (-(-W // block)) + x // block
    return y * W + x


def n_regions(H, W, kind, block):
    if kind == 0:
        return 1
    if kind == 1:
        return (-(-H // block)) * (-(-W // block))
    return H * W


def leaf(px, d):
    s = 8 - d
    return (int(px[0]) >> s, int(px[1]) >> s, int(px[2]) >> s)


def frame_leaf_sets(frame, d, kind, block):
    """Per region, the set of leaves present in one frame (uint8[H, W, 3])."""
    H, W, _ = frame.shape
    sets = [set() for _ in range(n_regions(H, W, kind, block))]
    for y in range(H):
        for x in range(W):
            sets[region_of(y, x, H, W, kind, block)].add(leaf(frame[y, x], d))
    return sets


def model_sets(train, d, T, kind, block=0):
    """Per region, the set of leaves present in at least T training frames."""
    N, H, W, _ = train.shape
    counts = [Counter() for _ in range(n_regions(H, W, kind, block))]
    for f in range(N):
        for r, s in enumerate(frame_leaf_sets(train[f], d, kind, block)):
            counts[r].update(s)
    return [{c for c, k in cnt.items() if k >= T} for cnt in counts]


def model_sets_groups(train, d, T, kind, block=0, group=1):
    """Per region, the set of leaves present in at least T of the trees built
    from groups of ``group`` consecutive training frames (Sec. 3): a group's
    tree holds every leaf of any of its frames."""
    N, H, W, _ = train.shape
    counts = [Counter() for _ in range(n_regions(H, W, kind, block))]
    for g0 in range(0, N, group):
        union = [set() for _ in counts]
        for f in range(g0, min(N, g0 + group)):
            for r, s in enumerate(frame_leaf_sets(train[f], d, kind, block)):
                union[r] |= s
        for r, s in enumerate(union):
            counts[r].update(s)
    return [{c for c, k in cnt.items() if k >= T} for cnt in counts]


def classify(msets, frames, d, kind, block=0):
    """uint8 mask list-of-lists: 1 = foreground (leaf not in the region's model)."""
    F, H, W, _ = frames.shape
    out = []
    for f in range(F):
        rows = []
        for y in range(H):
            rows.append([0 if leaf(frames[f, y, x], d) in msets[region_of(y, x, H, W, kind, block)] else 1
                         for x in range(W)])
        out.append(rows)
    return out
