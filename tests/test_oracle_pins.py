"""Pins of the CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: each check comes from the
paper's statements (Sec. 2 leaf colours, Alg. 1-3), a closed form, an
invariant, a hand-derived golden case, or the independent set-based
restatement in ``oracle/brute.py``.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FRAME, BLOCK, PIXEL = 0, 1, 2


def rng(seed):
    return np.random.default_rng(seed)


def model_codes(row):
    """Set bits of one exported model row (u64 words, bit c%64 of word c/64)."""
    bits = np.unpackbits(row.view(np.uint8), bitorder="little")
    return set(np.nonzero(bits)[0].tolist())


def code_of_leaf_tuple(q, d):
    """Oracle path code of a leaf given as (r,g,b) top-d-bit tuple: the oracle
    walks a representative colour (the leaf's bits followed by zeros)."""
    s = 8 - d
    col = np.array([[q[0] << s, q[1] << s, q[2] << s]], dtype=np.uint8)
    return int(oracle.leaf_codes(col, d)[0])


# ---- S1: path codes ---------------------------------------------------------

def test_path_code_golden():
    rows = []
    for line in open(os.path.join(GOLDEN, "path_codes.txt")):
        line = line.split("#")[0].strip()
        if line:
            rows.append([int(v) for v in line.split()])
    for r, g, b, d, code in rows:
        got = oracle.leaf_codes(np.array([[r, g, b]], np.uint8), d)[0]
        assert got == code, (r, g, b, d, got, code)


@pytest.fixture(scope="module")
def all_colours():
    v = np.arange(1 << 24, dtype=np.uint32)
    return np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], axis=1).astype(np.uint8)


@pytest.fixture(scope="module")
def all_codes(all_colours):
    return {d: oracle.leaf_codes(all_colours, d) for d in range(1, 9)}


@pytest.mark.parametrize("d", range(1, 9))
def test_path_code_partition_exhaustive(all_colours, all_codes, d):
    """Sec. 2: colours share a leaf iff they share their d most significant bits
    per channel.  Over all 2^24 colours: 8^d leaves of 2^(24-3d) colours each,
    and the code is constant on each top-d-bit class."""
    codes = all_codes[d]
    assert codes.max() < 8 ** d
    counts = np.bincount(codes, minlength=8 ** d)
    assert (counts == 1 << (24 - 3 * d)).all()
    s = 8 - d
    q = ((all_colours[:, 0].astype(np.uint32) >> s) << (2 * d)) | \
        ((all_colours[:, 1].astype(np.uint32) >> s) << d) | (all_colours[:, 2].astype(np.uint32) >> s)
    # code is a function of the top-d-bit class and a bijection between classes and codes
    first = np.full(8 ** d, -1, np.int64)
    first[q] = codes
    assert (first[q] == codes).all()
    assert np.unique(first).size == 8 ** d


@pytest.mark.parametrize("d", range(1, 9))
def test_path_code_decodes_to_leaf_colour(all_colours, all_codes, d):
    """Sec. 2: the leaf colour is the path's d original bits followed by zeros.
    Reading each base-8 digit of the code as (r,g,b) bits MSB-first must give
    the colour with its low 8-d bits cleared."""
    codes = all_codes[d].astype(np.uint32)
    rec = np.zeros((codes.size, 3), np.uint32)
    for level in range(d):
        digit = (codes >> (3 * (d - 1 - level))) & 7
        bit = 7 - level
        rec[:, 0] |= ((digit >> 2) & 1) << bit
        rec[:, 1] |= ((digit >> 1) & 1) << bit
        rec[:, 2] |= (digit & 1) << bit
    keep = np.uint32((0xFF << (8 - d)) & 0xFF)
    assert (rec == (all_colours.astype(np.uint32) & keep)).all()


@pytest.mark.parametrize("d", range(1, 8))
def test_path_code_nesting(all_codes, d):
    """Pruning one more level drops the last child index: code_d = code_{d+1} >> 3."""
    assert (all_codes[d] == all_codes[d + 1] >> 3).all()


# ---- S2: per-frame trees ----------------------------------------------------

@pytest.mark.parametrize("kind,block", [(FRAME, 0), (BLOCK, 5), (PIXEL, 0)])
@pytest.mark.parametrize("d", [1, 3, 8])
def test_constant_frame_one_leaf(kind, block, d):
    frame = np.zeros((13, 17, 3), np.uint8)
    frame[...] = (201, 77, 3)
    leaves, sums, nodes = oracle.tree_stats(frame, d, kind, block)
    R = oracle.region_count(13, 17, kind, block)
    assert leaves.size == R and (leaves == 1).all()
    assert (nodes == d + 1).all()
    sizes = np.bincount([brute.region_of(y, x, 13, 17, kind, block) for y in range(13) for x in range(17)],
                        minlength=R)
    assert (sums == sizes).all()


@pytest.mark.parametrize("kind,block", [(FRAME, 0), (BLOCK, 4), (BLOCK, 7), (PIXEL, 0)])
@pytest.mark.parametrize("d", [1, 2, 4, 6])
def test_leaf_counts_sum_to_pixels(kind, block, d):
    """Leaf pixel counters sum to the region's pixel count; the number of leaves is
    the number of distinct top-d-bit colours in the region (brute force)."""
    frame = rng(7 + d).integers(0, 256, size=(11, 14, 3), dtype=np.uint8)
    leaves, sums, nodes = oracle.tree_stats(frame, d, kind, block)
    sets = brute.frame_leaf_sets(frame, d, kind, block)
    sizes = np.bincount([brute.region_of(y, x, 11, 14, kind, block) for y in range(11) for x in range(14)],
                        minlength=len(sets))
    assert (sums == sizes).all()
    assert leaves.tolist() == [len(s) for s in sets]
    # a pruned tree has at most sum over levels of min(8^l, leaves) nodes and at least d+1
    assert (nodes >= d + 1).all()


def test_complete_tree_node_count(all_colours):
    """A tree holding every colour, pruned at d, is the complete octree:
    8^d leaves and (8^(d+1)-1)/7 nodes."""
    img = all_colours.reshape(1, 4096, 4096, 3)
    for d in (1, 2, 3):
        leaves, sums, nodes = oracle.tree_stats(img[0], d, FRAME, 0)
        assert leaves[0] == 8 ** d and sums[0] == 1 << 24 and nodes[0] == (8 ** (d + 1) - 1) // 7


# ---- S3/S4: merge and check, hand-derived golden cases -------------------------

def load_merge_cases():
    cases, cur = [], None
    for raw in open(os.path.join(GOLDEN, "merge_cases.txt")):
        line = raw.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("case "):
            _, name, N, H, W, d, T = line.split()
            cur = dict(name=name, N=int(N), H=int(H), W=int(W), d=int(d), T=int(T), frames=[], probes=[])
            cases.append(cur)
        elif line.startswith("model"):
            v = line.split()[1:]
            cur["model"] = set() if v == ["-"] else {int(c) for c in v}
        elif line.startswith("probe"):
            col, exp = line[len("probe"):].split("->")
            cur["probes"].append(([int(c) for c in col.split(",")], int(exp)))
        else:
            cur["frames"].append([[int(c) for c in t.split(",")] for t in line.split()])
    return cases


@pytest.mark.parametrize("case", load_merge_cases(), ids=lambda c: c["name"])
def test_merge_golden(case):
    train = np.array(case["frames"], np.uint8).reshape(case["N"], case["H"], case["W"], 3)
    probes = np.array([p for p, _ in case["probes"]], np.uint8).reshape(1, 1, -1, 3)
    # the probes form one test frame of width len(probes), region = whole frame
    model, _ = oracle.run(train, case["d"], case["T"], FRAME)
    assert model_codes(model[0]) == case["model"]
    # classify via the exported model (Alg. 3 on the re-imported tree)
    mask = oracle.classify(model, probes, case["d"], FRAME)
    assert mask.ravel().tolist() == [e for _, e in case["probes"]]
    # and Check Color on the merged tree itself: one test frame per probe colour
    test = np.empty((len(case["probes"]), case["H"], case["W"], 3), np.uint8)
    test[...] = probes.reshape(-1, 1, 1, 3)
    _, mask2 = oracle.run(train, case["d"], case["T"], FRAME, 0, test)
    assert mask2.reshape(len(case["probes"]), -1).min(axis=1).tolist() == [e for _, e in case["probes"]]
    assert mask2.reshape(len(case["probes"]), -1).max(axis=1).tolist() == [e for _, e in case["probes"]]


# ---- invariants against the set-based restatement ------------------------------

def leaf_sets_from_model(model, d):
    """Convert exported rows into sets of top-d-bit tuples using the oracle's own
    walk for the code of each candidate leaf."""
    table = {code_of_leaf_tuple((r, g, b), d): (r, g, b)
             for r in range(1 << d) for g in range(1 << d) for b in range(1 << d)}
    return [{table[c] for c in model_codes(row)} for row in model]


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_tiny(seed):
    g = rng(100 + seed)
    H, W = int(g.integers(1, 5)), int(g.integers(1, 5))
    N = int(g.integers(1, 6))
    d = int(g.integers(1, 4))
    kind = int(g.integers(0, 3))
    block = int(g.integers(1, 4)) if kind == BLOCK else 0
    # few distinct colours so that leaves repeat across frames
    palette = g.integers(0, 256, size=(4, 3), dtype=np.uint8)
    train = palette[g.integers(0, 4, size=(N, H, W))]
    test = np.concatenate([palette[g.integers(0, 4, size=(3, H, W))],
                           g.integers(0, 256, size=(2, H, W, 3), dtype=np.uint8)])
    for T in range(1, N + 1):
        model, mask = oracle.run(train, d, T, kind, block, test)
        expect = brute.model_sets(train, d, T, kind, block)
        assert leaf_sets_from_model(model, d) == expect, (T,)
        assert mask.tolist() == brute.classify(expect, test, d, kind, block)


def _random_video(seed, N, H, W, ncol=6):
    g = rng(seed)
    palette = g.integers(0, 256, size=(ncol, 3), dtype=np.uint8)
    return palette[g.integers(0, ncol, size=(N, H, W))], g


@pytest.mark.parametrize("kind,block", [(FRAME, 0), (BLOCK, 3), (PIXEL, 0)])
def test_T1_union_and_TN_intersection(kind, block):
    train, _ = _random_video(5, 6, 7, 9)
    d = 3
    per_frame = [brute.frame_leaf_sets(train[f], d, kind, block) for f in range(6)]
    R = len(per_frame[0])
    union = [set().union(*[per_frame[f][r] for f in range(6)]) for r in range(R)]
    inter = [set.intersection(*[per_frame[f][r] for f in range(6)]) for r in range(R)]
    m1, mask = oracle.run(train, d, 1, kind, block, train)
    assert leaf_sets_from_model(m1, d) == union
    assert not mask.any(), "T=1: every training pixel must be background"
    mN, _ = oracle.run(train, d, 6, kind, block)
    assert leaf_sets_from_model(mN, d) == inter


@pytest.mark.parametrize("kind,block", [(FRAME, 0), (BLOCK, 4), (PIXEL, 0)])
def test_monotone_in_T(kind, block):
    train, _ = _random_video(11, 8, 6, 10)
    prev = None
    for T in range(1, 9):
        m = oracle.build_model(train, 4, T, kind, block)
        if prev is not None:
            assert not (m & ~prev).any(), "raising T may only remove leaves"
        prev = m


def test_pixel_location_keeps_at_most_N_over_T_leaves():
    """Per pixel location each frame's tree holds exactly one leaf, so a leaf
    in T or more trees uses up T of the N frames: at most floor(N/T) leaves
    survive the merge (the bound that makes 8-entry kept-leaf lists exact when
    floor(N/T) <= 8), and the bound is reached when the frames cycle through
    floor(N/T) colours."""
    train, _ = _random_video(23, 12, 5, 7, ncol=4)
    for d in (4, 5):
        for T in (1, 2, 3, 4, 6, 12):
            m = oracle.build_model(train, d, T, PIXEL, 0)
            per_loc = np.array([bin(int(w)).count("1") for w in m.reshape(-1)]).reshape(m.shape).sum(axis=1)
            assert per_loc.max() <= 12 // T, (d, T)
    # k = floor(12 / 3) = 4 colours, each in exactly 3 of the 12 frames
    cols = np.array([[0, 0, 0], [255, 0, 0], [0, 255, 0], [0, 0, 255]], dtype=np.uint8)
    cyc = np.broadcast_to(cols[np.arange(12) % 4][:, None, None, :], (12, 2, 3, 3)).copy()
    m = oracle.build_model(cyc, 4, 3, PIXEL, 0)
    assert all(sum(bin(int(w)).count("1") for w in row) == 4 for row in m)


@pytest.mark.parametrize("kind,block", [(FRAME, 0), (BLOCK, 4), (PIXEL, 0)])
def test_permutation_invariance(kind, block):
    train, g = _random_video(13, 7, 6, 8)
    perm = g.permutation(7)
    for T in (1, 3, 7):
        a = oracle.build_model(train, 3, T, kind, block)
        b = oracle.build_model(train[perm], 3, T, kind, block)
        assert (a == b).all()


@pytest.mark.parametrize("kind,block", [(FRAME, 0), (BLOCK, 4), (PIXEL, 0)])
def test_depth_nesting(kind, block):
    """A leaf kept at depth d has its parent kept at depth d-1 (the frames that
    hold the leaf also hold its prefix)."""
    train, _ = _random_video(17, 6, 5, 9, ncol=9)
    for d in range(2, 6):
        fine = oracle.build_model(train, d, 3, kind, block)
        coarse = oracle.build_model(train, d - 1, 3, kind, block)
        for rf, rc in zip(fine, coarse):
            assert {c >> 3 for c in model_codes(rf)} <= model_codes(rc)


def test_frame_equals_large_block():
    train, _ = _random_video(19, 5, 9, 11)
    test, _ = _random_video(20, 3, 9, 11)
    a, ma = oracle.run(train, 3, 2, FRAME, 0, test)
    b, mb = oracle.run(train, 3, 2, BLOCK, 11, test)
    assert (a == b).all() and (ma == mb).all()


def test_classify_roundtrip_matches_merged_tree():
    """Classifying with the exported model (re-imported tree) equals classifying
    with the merged tree itself."""
    train, _ = _random_video(23, 6, 8, 10, ncol=12)
    test, _ = _random_video(24, 4, 8, 10, ncol=12)
    for kind, block in [(FRAME, 0), (BLOCK, 3), (PIXEL, 0)]:
        for d in (1, 2, 5):
            m, mask = oracle.run(train, d, 2, kind, block, test)
            assert (oracle.classify(m, test, d, kind, block) == mask).all()


def test_region_subset_matches_full():
    train, _ = _random_video(29, 5, 7, 9)
    test, _ = _random_video(30, 2, 7, 9)
    full, fmask = oracle.run(train, 3, 2, PIXEL, 0, test)
    regs = np.array([0, 5, 62, 17], np.int64)
    sub, smask = oracle.run(train, 3, 2, PIXEL, 0, test, regions=regs)
    assert (sub == full[regs]).all()
    assert smask.reshape(len(regs), 2).tolist() == fmask.reshape(2, -1)[:, regs].T.tolist()


def test_fraction_threshold_reading():
    """Reading R3: the paper's test count/N >= t equals count >= ceil(t*N)."""
    train, _ = _random_video(31, 9, 4, 6)
    for t in (0.1, 1 / 3, 0.5, 0.77, 1.0):
        T = int(np.ceil(t * 9 - 1e-12))
        T = max(T, 1)
        m = oracle.build_model(train, 3, T, FRAME)
        counts = {}
        for f in range(9):
            for leaf in brute.frame_leaf_sets(train[f], 3, FRAME, 0)[0]:
                counts[leaf] = counts.get(leaf, 0) + 1
        expect = {leaf for leaf, c in counts.items() if c / 9 >= t}
        assert leaf_sets_from_model(m, 3)[0] == expect


def test_bad_arguments_raise():
    train = np.zeros((2, 3, 3, 3), np.uint8)
    with pytest.raises(ValueError):
        oracle.build_model(train, 0, 1, FRAME)
    with pytest.raises(ValueError):
        oracle.build_model(train, 9, 1, FRAME)
    with pytest.raises(ValueError):
        oracle.build_model(train, 3, 3, FRAME)
    with pytest.raises(ValueError):
        oracle.build_model(train, 3, 0, FRAME)
