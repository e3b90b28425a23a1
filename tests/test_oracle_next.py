"""Pins of the oracle's redraw (Sec. 2, Fig. 2), group-of-frames trees
(Sec. 3) and F0 (Sec. 5) functions: hand-derived golden cases
(``tests/golden/next_cases.txt``), closed forms, exhaustive colour sweeps and
the set-based restatement in ``oracle/brute.py``."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "next_cases.txt")
FRAME, BLOCK, PIXEL = 0, 1, 2


def _golden(kind):
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if line.startswith(kind + " "):
            out.append(line[len(kind) + 1:])
    return out


def _rgb(t):
    return [int(v) for v in t.split(",")]


def test_redraw_golden():
    cases = _golden("redraw")
    assert len(cases) >= 5
    for c in cases:
        left, right = c.split("->")
        d, col = left.split()
        got = oracle.redraw(np.array([_rgb(col)], np.uint8), int(d))
        assert got[0].tolist() == _rgb(right.strip()), c


@pytest.fixture(scope="module")
def all_colours():
    v = np.arange(1 << 24, dtype=np.uint32)
    return np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], axis=1).astype(np.uint8)


@pytest.mark.parametrize("d", range(1, 9))
def test_redraw_exhaustive(all_colours, d):
    """Every colour: the d top bits of each channel, zeros below (Sec. 2);
    the redrawn colour lies in the same leaf and redraws to itself."""
    out = oracle.redraw(all_colours, d)
    keep = np.uint8((0xFF << (8 - d)) & 0xFF)
    assert (out == (all_colours & keep)).all()
    sample = all_colours[:: 997]
    assert (oracle.leaf_codes(oracle.redraw(sample, d), d) == oracle.leaf_codes(sample, d)).all()
    assert (oracle.redraw(out[:: 997], d) == out[:: 997]).all()


def _bits(s):
    return np.array([int(ch) for ch in s], np.uint8)


def _frac(s):
    a, b = s.split("/")
    return Fraction(int(a), int(b))


def test_confusion_and_f0_golden():
    cases = _golden("confusion")
    assert len(cases) >= 3
    for c in cases:
        lhs, rhs = c.split("->")
        m, g = (x.strip() for x in lhs.split("|"))
        counts_s, ratios_s = rhs.split(";")
        got = oracle.confusion(_bits(m)[None], _bits(g)[None])
        assert got[0].tolist() == [int(v) for v in counts_s.split()], c
        sc = oracle.f_scores(got)
        want = [_frac(v) for v in ratios_s.split()]
        for key, w in zip(("P0", "R0", "F0", "F1"), want):
            assert abs(sc[key] - float(w)) < 1e-12, (c, key)


def test_confusion_brute_force_and_nonbinary_bytes():
    g = np.random.default_rng(3)
    mask = g.integers(0, 2, size=(5, 7, 9), dtype=np.uint8) * g.integers(1, 256, size=(5, 7, 9), dtype=np.uint8)
    gt = g.integers(0, 2, size=(5, 7, 9), dtype=np.uint8)
    got = oracle.confusion(mask, gt)
    for f in range(5):
        m, t = mask[f] != 0, gt[f] != 0
        assert got[f].tolist() == [int((m & t).sum()), int((m & ~t).sum()), int((~m & ~t).sum()),
                                   int((~m & t).sum())]
    assert int(got.sum()) == mask.size


def test_f0_is_background_class_f_score():
    """F0 is the F-score of the background class: swapping the classes of
    mask and ground truth turns it into the foreground F1."""
    g = np.random.default_rng(4)
    mask = g.integers(0, 2, size=(3, 11, 13), dtype=np.uint8)
    gt = g.integers(0, 2, size=(3, 11, 13), dtype=np.uint8)
    a = oracle.f_scores(oracle.confusion(mask, gt))
    b = oracle.f_scores(oracle.confusion(1 - mask, 1 - gt))
    assert abs(a["F0"] - b["F1"]) < 1e-12 and abs(a["F1"] - b["F0"]) < 1e-12


def _leaf_codes_of_row(row):
    bits = np.unpackbits(row.view(np.uint8), bitorder="little")
    return sorted(np.nonzero(bits)[0].tolist())


def test_groups_golden():
    cases = _golden("groups")
    assert len(cases) >= 4
    for c in cases:
        head, rest = c.split(":")
        N, group, d, T = (int(v) for v in head.split())
        cols, want = rest.split("->")
        train = np.array([_rgb(t) for t in cols.split()], np.uint8).reshape(N, 1, 1, 3)
        model, _ = oracle.run(train, d, T, FRAME, 0, group=group)
        want = [] if want.strip() == "-" else [int(v) for v in want.split()]
        assert _leaf_codes_of_row(model[0]) == want, c


def _leaf_sets(model, d):
    out = []
    for row in model:
        s = set()
        for c in _leaf_codes_of_row(row):
            r = g = b = 0
            for lvl in range(d):  # path code -> per-channel top-d bits
                idx = (c >> (3 * (d - 1 - lvl))) & 7
                r, g, b = (r << 1) | (idx >> 2), (g << 1) | ((idx >> 1) & 1), (b << 1) | (idx & 1)
            s.add((r, g, b))
        out.append(s)
    return out


@pytest.mark.parametrize("kind,block", [(FRAME, 0), (BLOCK, 3), (PIXEL, 0)])
@pytest.mark.parametrize("group", [1, 2, 3, 7])
def test_groups_brute_force(kind, block, group):
    """One tree per group of frames (Sec. 3) against Python sets: a group's
    tree holds the leaves of any of its frames; keep leaves in >= T trees."""
    g = np.random.default_rng(100 + group + kind)
    palette = g.integers(0, 256, size=(6, 3), dtype=np.uint8)
    N = 7
    train = palette[g.integers(0, 6, size=(N, 5, 7))]
    d = 3
    for T in range(1, -(-N // group) + 1):
        model, _ = oracle.run(train, d, T, kind, block, group=group)
        assert _leaf_sets(model, d) == brute.model_sets_groups(train, d, T, kind, block, group), (T,)


def test_groups_reduce_to_frames_and_union():
    g = np.random.default_rng(9)
    palette = g.integers(0, 256, size=(5, 3), dtype=np.uint8)
    train = palette[g.integers(0, 5, size=(6, 4, 6))]
    for kind, block in ((FRAME, 0), (BLOCK, 2), (PIXEL, 0)):
        per_frame = [brute.frame_leaf_sets(train[f], 4, kind, block) for f in range(6)]
        union = [set().union(*[per_frame[f][r] for f in range(6)]) for r in range(len(per_frame[0]))]
        one_tree, _ = oracle.run(train, 4, 1, kind, block, group=6)
        assert _leaf_sets(one_tree, 4) == union
        for T in (1, 3, 6):
            a, _ = oracle.run(train, 4, T, kind, block, group=1)
            assert _leaf_sets(a, 4) == brute.model_sets(train, 4, T, kind, block)


def test_groups_threshold_counts_trees():
    """With groups of 2 out of 5 frames there are ceil(5 / 2) = 3 trees: T = 3
    is the largest threshold allowed."""
    train = np.zeros((5, 2, 2, 3), np.uint8)
    model, _ = oracle.run(train, 2, 3, FRAME, 0, group=2)
    assert _leaf_codes_of_row(model[0]) == [0]  # black is in all 3 trees
    with pytest.raises(ValueError):
        oracle.run(train, 2, 4, FRAME, 0, group=2)
