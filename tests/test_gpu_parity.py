"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Everything here is integer work, so the bar is bit-exact: exported model
bitsets and foreground masks must equal the oracle's element by element.
"""
import numpy as np
import pytest

import ocq_synth
import oracle
from ocq_synth import configs

pytestmark = pytest.mark.gpu
FRAME, BLOCK, PIXEL = 0, 1, 2


@pytest.fixture(scope="module")
def ocq(cuda_ready):
    return cuda_ready


@pytest.fixture(scope="module")
def torch():
    import torch

    return torch


def to_dev(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_model_and_mask(ocq, torch, train, test, d, T, kind, block):
    tr = to_dev(train, torch)
    m = ocq.build_model(tr, d, T, kind, block)
    words = ocq.export_model(m).cpu().numpy().view(np.uint64)
    mask = None
    if test is not None:
        mask = ocq.classify(m, to_dev(test, torch)).cpu().numpy()
    ocq.device_status()
    m.free()
    return words, mask


# ---- S1 -------------------------------------------------------------------------

def test_path_code_all_colours(ocq, torch):
    v = np.arange(1 << 24, dtype=np.uint32)
    rgb = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], axis=1).astype(np.uint8)
    dev = to_dev(rgb, torch)
    for d in range(1, 9):
        got = ocq.path_code(dev, d).cpu().numpy().view(np.uint32)
        assert (got == oracle.leaf_codes(rgb, d)).all(), d


# ---- S2 -------------------------------------------------------------------------

@pytest.mark.parametrize("kind,block", [(FRAME, 0), (BLOCK, 5), (PIXEL, 0)])
@pytest.mark.parametrize("d", [1, 3, 5, 8])
def test_occupancy_matches_per_frame_trees(ocq, torch, kind, block, d):
    g = np.random.default_rng(40 + d)
    H, W = (5, 3) if (kind == PIXEL and d >= 6) else (13, 19)
    frames = g.integers(0, 256, size=(3, H, W, 3), dtype=np.uint8)
    occ = ocq.occupancy(to_dev(frames, torch), d, kind, block).cpu().numpy().view(np.uint64)
    for f in range(3):
        # a per-frame tree's leaf set is the merge of that one tree with T = 1
        expect = oracle.build_model(frames[f:f + 1], d, 1, kind, block)
        assert (occ[f] == expect).all(), f


# ---- S1-S4 on small random shapes ------------------------------------------------

CASES = []
for kind, block in [(FRAME, 0), (BLOCK, 1), (BLOCK, 4), (BLOCK, 7), (PIXEL, 0)]:
    for d in range(1, 9):
        CASES.append((kind, block, d))


@pytest.mark.parametrize("kind,block,d", CASES)
def test_build_classify_random(ocq, torch, kind, block, d):
    g = np.random.default_rng(1000 + 17 * kind + block * 3 + d)
    H, W = int(g.integers(5, 23)), int(g.integers(5, 29))
    if d >= 6 and kind != FRAME:  # rows of 8^d bits: keep the models small
        H, W = int(g.integers(2, 9)), int(g.integers(2, 9))
    N = int(g.integers(1, 9))
    palette = g.integers(0, 256, size=(7, 3), dtype=np.uint8)
    train = palette[g.integers(0, 7, size=(N, H, W))]
    train[:, ::3] = g.integers(0, 256, size=train[:, ::3].shape, dtype=np.uint8)
    test = np.concatenate([palette[g.integers(0, 7, size=(3, H, W))],
                           g.integers(0, 256, size=(2, H, W, 3), dtype=np.uint8)])
    for T in sorted({1, (N + 1) // 2, N}):
        words, mask = gpu_model_and_mask(ocq, torch, train, test, d, T, kind, block)
        ow, om = oracle.run(train, d, T, kind, block, test)
        assert (words == ow).all(), ("model", T)
        assert (mask == om).all(), ("mask", T)


@pytest.mark.parametrize("H,W", [(48, 64), (52, 80), (29, 37), (16, 1024), (1, 2049)])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_pixel_tiles_and_ragged_tail(ocq, torch, H, W, d):
    """Pixel regions, depth <= 3: the tiled kernel (full tiles) plus the
    remainder, and the generic path when H*W is not a multiple of 16."""
    sc = ocq_synth.make_scene("bimodal", H, W, 12, 9, seed=77 + d)
    frames = ocq_synth.fill_host(sc, 0, 21)
    train, test = frames[:12], frames[12:]
    words, mask = gpu_model_and_mask(ocq, torch, train, test, d, 3, PIXEL, 0)
    ow, om = oracle.run(train, d, 3, PIXEL, 0, test)
    assert (words == ow).all()
    assert (mask == om).all()


def test_pixel_wide_counters(ocq, torch):
    """N > 255 switches the per-pixel counters to 16 bits."""
    g = np.random.default_rng(5)
    palette = g.integers(0, 256, size=(3, 3), dtype=np.uint8)
    train = palette[g.integers(0, 3, size=(300, 4, 8))]
    test = palette[g.integers(0, 3, size=(2, 4, 8))]
    for T in (1, 97, 150, 300):
        words, mask = gpu_model_and_mask(ocq, torch, train, test, 3, T, PIXEL, 0)
        ow, om = oracle.run(train, 3, T, PIXEL, 0, test)
        assert (words == ow).all() and (mask == om).all(), T


def test_constant_frames_edge_cases(ocq, torch):
    train = np.zeros((4, 6, 7, 3), np.uint8)
    train[...] = (10, 200, 30)
    test = np.zeros((2, 6, 7, 3), np.uint8)
    test[0] = (10, 200, 30)
    test[1] = (200, 10, 30)
    for kind, block in [(FRAME, 0), (BLOCK, 3), (PIXEL, 0)]:
        words, mask = gpu_model_and_mask(ocq, torch, train, test, 4, 4, kind, block)
        ow, om = oracle.run(train, 4, 4, kind, block, test)
        assert (words == ow).all() and (mask == om).all()
        assert not mask[0].any() and mask[1].all()


def test_export_import_roundtrip(ocq, torch):
    g = np.random.default_rng(9)
    train = g.integers(0, 256, size=(5, 9, 11, 3), dtype=np.uint8)
    test = g.integers(0, 256, size=(3, 9, 11, 3), dtype=np.uint8)
    for kind, block in [(FRAME, 0), (BLOCK, 4), (PIXEL, 0)]:
        for d in (1, 2, 3, 5):
            m = ocq.build_model(to_dev(train, torch), d, 2, kind, block)
            words = ocq.export_model(m)
            m2 = ocq.import_model(words, 9, 11, kind, block, d)
            assert (ocq.export_model(m2).cpu() == words.cpu()).all()
            t = to_dev(test, torch)
            assert (ocq.classify(m2, t).cpu() == ocq.classify(m, t).cpu()).all()
            # classify of an oracle-made model imported into the library
            ow = oracle.build_model(train, d, 2, kind, block)
            m3 = ocq.import_model(to_dev(ow.view(np.int64), torch), 9, 11, kind, block, d)
            assert (ocq.classify(m3, t).cpu().numpy() == oracle.classify(ow, test, d, kind, block)).all()
            m.free(), m2.free(), m3.free()


def test_list_model_full_lists(ocq, torch):
    """Lists at capacity: 16 frames cycling through 8 colours, T = 2, so every
    location keeps exactly floor(N/T) = 8 leaves (all 8 entries used); a
    ninth colour and the kept ones classify as the oracle says, in every
    classify form."""
    cols = np.array([[0, 0, 0], [255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 0], [255, 0, 255],
                     [0, 255, 255], [255, 255, 255], [128, 64, 32]], dtype=np.uint8)
    H, W = 16, 36
    train = np.broadcast_to(cols[np.arange(16) % 8][:, None, None, :], (16, H, W, 3)).copy()
    test = np.broadcast_to(cols[np.arange(9)][:, None, None, :], (9, H, W, 3)).copy()
    lst = ocq.ocq.OCQ_TUNE_CLASSIFY_PIXEL_LIST
    saved = ocq.ocq.ocq_tune_selected(lst)
    try:
        for d in (4, 5):
            ow, om = oracle.run(train, d, 2, PIXEL, 0, test)
            assert om[:8].sum() == 0 and om[8].all()
            for form in range(ocq.ocq.ocq_tune_count(lst)):
                ocq.ocq.ocq_tune_select(lst, form)
                words, mask = gpu_model_and_mask(ocq, torch, train, test, d, 2, PIXEL, 0)
                assert (words == ow).all() and (mask == om).all(), (d, form)
    finally:
        ocq.ocq.ocq_tune_select(lst, saved)


def test_list_model_import(ocq, torch):
    """A header that makes a list model (per pixel, d = 4-5, floor(N/T) <= 8)
    reads the bitset into lists: export round-trips, an oracle-made model
    classifies as the oracle does, and a location with more than floor(N/T)
    leaves is refused with OCQ_EINVAL; other headers keep the rows."""
    H, W, N = 14, 22, 12
    sc = ocq_synth.make_scene("clusters", H, W, N, 5, seed=5)
    frames = ocq_synth.fill_host(sc, 0, N + 5)
    train, test = frames[:N], frames[N:]
    t = to_dev(test, torch)
    for d, T in ((4, 3), (5, 2), (5, 1)):  # k = 4, 6, 12 (the last: rows)
        ow, om = oracle.run(train, d, T, PIXEL, 0, test)
        m = ocq.import_model(to_dev(ow.view(np.int64), torch), H, W, PIXEL, 0, d, T=T, N=N)
        assert (ocq.export_model(m).cpu().numpy().view(np.uint64) == ow).all(), (d, T)
        assert (ocq.classify(m, t).cpu().numpy() == om).all(), (d, T)
        m.free()
        if N // T <= 8:
            bad = ow.copy()
            bad[7, :] = 0
            bad[7, 0] = (1 << (N // T + 1)) - 1  # floor(N/T) + 1 leaves at location 7
            with pytest.raises(ocq.ocq.OcqError) as e:
                ocq.import_model(to_dev(bad.view(np.int64), torch), H, W, PIXEL, 0, d, T=T, N=N)
            assert e.value.status == 1


# ---- the preset workloads -----------------------------------------------------------

def _workload_frames(wl, n_test=None):
    sc = ocq_synth.make_scene(wl.scene_kind, wl.H, wl.W, wl.N, wl.F, wl.seed, wl.stream)
    F = wl.F if n_test is None else n_test
    frames = ocq_synth.fill_host(sc, 0, wl.N + F)
    return frames[:wl.N], frames[wl.N:]


def test_tiny_frame_preset(ocq, torch):
    wl = configs.TINY_FRAME
    train, test = _workload_frames(wl)
    words, mask = gpu_model_and_mask(ocq, torch, train, test, wl.depth, wl.T, wl.region, wl.block)
    ow, om = oracle.run(train, wl.depth, wl.T, wl.region, wl.block, test)
    assert (words == ow).all() and (mask == om).all()


def test_block_preset(ocq, torch):
    wl = configs.BLOCKS_320x240
    train, test = _workload_frames(wl)
    words, mask = gpu_model_and_mask(ocq, torch, train, test, wl.depth, wl.T, wl.region, wl.block)
    ow, om = oracle.run(train, wl.depth, wl.T, wl.region, wl.block, test)
    assert (words == ow).all() and (mask == om).all()


def test_pixel_1080p_full_size_sampled(ocq, torch):
    """The 1920x1080 per-pixel preset at full size (50 training + 1000 test
    frames, generated on the device), in the bench's launch configuration;
    the oracle checks every frame at sampled pixel locations, including the
    first and last pixel of tiles and of the frame."""
    wl = configs.PIXEL_1080P
    H, W, N, F = wl.H, wl.W, wl.N, wl.F
    sc = ocq_synth.make_scene(wl.scene_kind, H, W, N, F, wl.seed)
    train = torch.empty((N, H, W, 3), dtype=torch.uint8, device="cuda")
    test = torch.empty((F, H, W, 3), dtype=torch.uint8, device="cuda")
    ocq_synth.fill_device(sc, 0, N, train)
    ocq_synth.fill_device(sc, N, F, test)
    m = ocq.build_model(train, wl.depth, wl.T, wl.region, wl.block)
    mask = ocq.classify(m, test)
    ocq.device_status()
    words = ocq.export_model(m)
    g = np.random.default_rng(123)
    hw = H * W
    picks = set(g.integers(0, hw, size=600).tolist())
    for t in (0, 1, 1023, 1024, 2047, 2048, hw // 2, hw - 1025, hw - 1024, hw - 1):
        picks.add(t)
    idx = np.array(sorted(picks), np.int64)
    ys, xs = idx // W, idx % W
    tr = train[:, ys, xs].cpu().numpy()[:, None]        # [N, 1, k, 3]
    te = test[:, ys, xs].cpu().numpy()[:, None]         # [F, 1, k, 3]
    ow, om = oracle.run(tr, wl.depth, wl.T, PIXEL, 0, te)
    gw = words[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint64)
    assert (gw == ow).all()
    gm = mask[:, ys, xs].cpu().numpy()
    assert (gm == om[:, 0]).all()
    # the synthetic truth: pixels the foreground discs never cover are mostly background
    assert mask.float().mean().item() < 0.5
    m.free()


def test_synth_device_matches_host(ocq, torch):
    for wl in (configs.TINY_FRAME, configs.BLOCKS_320x240):
        sc = ocq_synth.make_scene(wl.scene_kind, wl.H, wl.W, wl.N, wl.F, wl.seed)
        host, gt = ocq_synth.fill_host(sc, wl.N - 2, 5, with_gt=True)
        dev = torch.empty(host.shape, dtype=torch.uint8, device="cuda")
        dgt = torch.empty(gt.shape, dtype=torch.uint8, device="cuda")
        ocq_synth.fill_device(sc, wl.N - 2, 5, dev, dgt)
        assert (dev.cpu().numpy() == host).all() and (dgt.cpu().numpy() == gt).all()


def test_pixel_staged_counter_widths(ocq, torch):
    """Staged per-pixel build with 4-bit (T <= 15) and 8-bit (T <= 255)
    counters saturating at T, also with N > 255."""
    g = np.random.default_rng(21)
    palette = g.integers(0, 256, size=(4, 3), dtype=np.uint8)
    train = palette[g.integers(0, 4, size=(300, 16, 32))]
    train[:, :, ::5] = g.integers(0, 256, size=train[:, :, ::5].shape, dtype=np.uint8)
    test = palette[g.integers(0, 4, size=(3, 16, 32))]
    for T in (1, 14, 15, 16, 90, 255):
        words, mask = gpu_model_and_mask(ocq, torch, train, test, 3, T, PIXEL, 0)
        ow, om = oracle.run(train, 3, T, PIXEL, 0, test)
        assert (words == ow).all() and (mask == om).all(), T


@pytest.mark.parametrize("H,W", [(64, 96), (50, 80)])
def test_every_tuning_variant(ocq, torch, H, W):
    """Each selectable kernel variant of the per-pixel build and classify gives
    the oracle's result (several tiles of every tile size, plus a ragged rest)."""
    O = ocq.ocq
    sc = ocq_synth.make_scene("bimodal", H, W, 20, 11, seed=5)
    frames = ocq_synth.fill_host(sc, 0, 31)
    train, test = frames[:20], frames[20:]
    for d in (1, 2, 3):
        for T in (4, 17):
            ow, om = oracle.run(train, d, T, PIXEL, 0, test)
            for kernel in (O.OCQ_TUNE_BUILD_PIXEL, O.OCQ_TUNE_CLASSIFY_PIXEL):
                saved = O.ocq_tune_selected(kernel)
                try:
                    for v in range(O.ocq_tune_count(kernel)):
                        O.ocq_tune_select(kernel, v)
                        words, mask = gpu_model_and_mask(ocq, torch, train, test, d, T, PIXEL, 0)
                        assert (words == ow).all(), (kernel, v, d, T)
                        assert (mask == om).all(), (kernel, v, d, T)
                finally:
                    O.ocq_tune_select(kernel, saved)


@pytest.mark.parametrize("H,W", [(32, 64), (20, 52)])
def test_pixel_build_variants_many_distinct_leaves(ocq, torch, H, W):
    """Every per-pixel build variant at depth <= 3 when locations hold many
    distinct leaves: uniform noise in half the locations (as many distinct
    leaves as frames, past the candidate build's counters), scene content in
    the other half; several tiles and a ragged rest; N = 60 and N = 127."""
    O = ocq.ocq
    kern = O.OCQ_TUNE_BUILD_PIXEL
    saved = O.ocq_tune_selected(kern)
    try:
        for N in (60, 127):
            sc = ocq_synth.make_scene("bimodal", H, W, N, 3, seed=40 + N + W)
            frames = ocq_synth.fill_host(sc, 0, N + 3)
            g = np.random.default_rng(N * 7 + W)
            noise = g.integers(0, 256, size=frames.shape, dtype=np.uint8)
            sel = g.random((H, W)) < 0.5
            frames = np.where(sel[None, :, :, None], noise, frames)
            train, test = frames[:N], frames[N:]
            for d in (2, 3):
                for T in (1, 3, 10, N):
                    ow, om = oracle.run(train, d, T, PIXEL, 0, test)
                    for v in range(O.ocq_tune_count(kern)):
                        O.ocq_tune_select(kern, v)
                        words, mask = gpu_model_and_mask(ocq, torch, train, test, d, T, PIXEL, 0)
                        assert (words == ow).all(), (N, d, T, v)
                        assert (mask == om).all(), (N, d, T, v)
    finally:
        O.ocq_tune_select(kern, saved)


@pytest.mark.parametrize("b", [8, 16, 32, 64])
@pytest.mark.parametrize("d", [1, 3, 4, 5])
def test_block_tiled_classify(ocq, torch, b, d):
    """Block regions with b % 8 == 0 and W % 16 == 0 go through the strip-tiled
    classify kernel; partial blocks at the right and bottom edges included."""
    H, W = 3 * b + 5, 176 if b <= 16 else 2 * b + 48
    sc = ocq_synth.make_scene("sway", H, W, 9, 13, seed=300 + b + d)
    frames = ocq_synth.fill_host(sc, 0, 22)
    train, test = frames[:9], frames[9:]
    words, mask = gpu_model_and_mask(ocq, torch, train, test, d, 4, BLOCK, b)
    ow, om = oracle.run(train, d, 4, BLOCK, b, test)
    assert (words == ow).all()
    assert (mask == om).all()


@pytest.mark.parametrize("b", [2, 5, 8, 11, 16, 17])
@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_block_build_warp_tables(ocq, torch, b, d):
    """Block regions with b <= 16 and N <= 255 are built one warp per region
    with a leaf table in shared memory; b = 17 takes the CTA-per-region
    kernel.  Scene content, then uniform noise (far more distinct leaves per
    region than the table holds at depth 4-5, so the chunked fallback runs),
    with ragged blocks at the right and bottom edges."""
    for H, W in ((2 * b + 3, 3 * b + 7), (2 * b + 3, 4 * b + 4)):  # W % 4 == 0: word loads for full 8x8 blocks
        sc = ocq_synth.make_scene("sway", H, W, 10, 6, seed=500 + 7 * b + d + W)
        frames = ocq_synth.fill_host(sc, 0, 16)
        g = np.random.default_rng(900 + b * 11 + d + W)
        noise = g.integers(0, 256, size=(10, H, W, 3), dtype=np.uint8)
        for train in (frames[:10], noise):
            for T in (1, 3, 10):
                words, mask = gpu_model_and_mask(ocq, torch, train, frames[10:], d, T, BLOCK, b)
                ow, om = oracle.run(train, d, T, BLOCK, b, frames[10:])
                assert (words == ow).all(), (W, T)
                assert (mask == om).all(), (W, T)


@pytest.mark.parametrize("b", [8, 16])
@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_block_build_tiles(ocq, torch, b, d):
    """8 x 8 and 16 x 16 blocks with W % 8 == 0 are built by warps over 16 x 16
    pixel tiles (direct leaf tables at depth <= 3 and at depth 4 with 16 x 16
    blocks, hashed tables otherwise).  Widths with a half tile at the right
    edge, heights with ragged blocks at the bottom; scene content, then uniform
    noise (more distinct leaves per region than a hashed table takes, so the
    region is recounted by the chunked passes), and every build form (one
    warp per region, the default choice, frames split over a CTA's warps,
    warp tiles)."""
    O = ocq.ocq
    kern = O.OCQ_TUNE_BUILD_BLOCK
    saved = O.ocq_tune_selected(kern)
    try:
        for H, W in ((2 * b + 3, 40), (3 * b + 5, 64), (17, 8)):
            sc = ocq_synth.make_scene("sway", H, W, 12, 5, seed=700 + 13 * b + d + W)
            frames = ocq_synth.fill_host(sc, 0, 17)
            g = np.random.default_rng(910 + b * 7 + d + W)
            noise = g.integers(0, 256, size=(12, H, W, 3), dtype=np.uint8)
            for train in (frames[:12], noise):
                for T in (1, 4, 12):
                    ow, om = oracle.run(train, d, T, BLOCK, b, frames[12:])
                    for form in range(O.ocq_tune_count(kern)):
                        O.ocq_tune_select(kern, form)
                        words, mask = gpu_model_and_mask(ocq, torch, train, frames[12:], d, T, BLOCK, b)
                        assert (words == ow).all(), (H, W, T, form)
                        assert (mask == om).all(), (H, W, T, form)
    finally:
        O.ocq_tune_select(kern, saved)


@pytest.mark.parametrize("b,d", [(8, 3), (8, 4), (8, 5), (16, 4), (16, 5)])
def test_block_build_one_and_two_frames(ocq, torch, b, d):
    """Every block build form with N = 1 and N = 2 (T = 1 keeps every leaf of
    the frames, T = N only the leaves of both), on several regions with a
    ragged bottom row of blocks."""
    O = ocq.ocq
    kern = O.OCQ_TUNE_BUILD_BLOCK
    saved = O.ocq_tune_selected(kern)
    try:
        H, W = 3 * b + 5, 48
        sc = ocq_synth.make_scene("sway", H, W, 2, 3, seed=950 + 7 * b + d)
        frames = ocq_synth.fill_host(sc, 0, 5)
        for N in (1, 2):
            for T in sorted({1, N}):
                ow, om = oracle.run(frames[:N], d, T, BLOCK, b, frames[2:])
                for form in range(O.ocq_tune_count(kern)):
                    O.ocq_tune_select(kern, form)
                    words, mask = gpu_model_and_mask(ocq, torch, frames[:N], frames[2:], d, T, BLOCK, b)
                    assert (words == ow).all() and (mask == om).all(), (N, T, form)
    finally:
        O.ocq_tune_select(kern, saved)


@pytest.mark.parametrize("N", [254, 255, 256])
def test_block_build_frame_count_limits(ocq, torch, N):
    """The warp tables and the frame-split counters keep counts in 8 bits:
    N = 255 is their limit, N = 256 goes to the CTA-per-region kernel."""
    O = ocq.ocq
    kern = O.OCQ_TUNE_BUILD_BLOCK
    saved = O.ocq_tune_selected(kern)
    g = np.random.default_rng(N)
    palette = g.integers(0, 256, size=(5, 3), dtype=np.uint8)
    try:
        for W in (20, 24):  # one warp per region; tiles or frames split (W % 8 == 0)
            train = palette[g.integers(0, 5, size=(N, 12, W))]
            test = palette[g.integers(0, 5, size=(2, 12, W))]
            for d in (3, 4, 5):
                for T in (1, N // 5, N // 2, N):
                    ow, om = oracle.run(train, d, T, BLOCK, 8, test)
                    for form in range(O.ocq_tune_count(kern)):
                        O.ocq_tune_select(kern, form)
                        words, mask = gpu_model_and_mask(ocq, torch, train, test, d, T, BLOCK, 8)
                        assert (words == ow).all() and (mask == om).all(), (W, d, T, form)
    finally:
        O.ocq_tune_select(kern, saved)


@pytest.mark.parametrize("d", [4, 5, 6])
@pytest.mark.parametrize("H,W", [(24, 40), (13, 37), (9, 132)])
def test_pixel_deep_candidates_and_tiles(ocq, torch, d, H, W):
    """Pixel regions at depth >= 4: the build keeps 1, 2, 4 or 8 frequent-leaf
    candidates per location (or counts every distinct leaf when N / T > 8), and
    the classify walks all frames of 128-location tiles (H*W % 4 == 0) or falls
    back to per-pixel lookups; several warps' tiles plus a ragged one."""
    if d == 6:
        H, W = min(H, 6), min(W, 20)
    N = 40
    sc = ocq_synth.make_scene("bimodal", H, W, N, 9, seed=600 + d + H)
    frames = ocq_synth.fill_host(sc, 0, N + 9)
    g = np.random.default_rng(d * 100 + W)
    train = frames[:N].copy()
    train[::7] = g.integers(0, 256, size=train[::7].shape, dtype=np.uint8)  # a few noisy frames
    test = frames[N:]
    for T in (1, 4, 5, 10, 14, 21, 40):  # N // T = 40, 10, 8, 4, 2, 1, 1
        words, mask = gpu_model_and_mask(ocq, torch, train, test, d, T, PIXEL, 0)
        ow, om = oracle.run(train, d, T, PIXEL, 0, test)
        assert (words == ow).all(), T
        assert (mask == om).all(), T


def test_pixel_deep_classify_variants(ocq, torch):
    """Every form of the deep per-pixel classify (kept-leaf lists in each
    launch form, or the rows with each residency choice) gives the oracle's
    masks, with few and with many (> 8, the rows decide) kept leaves per
    location; 2880 locations leave a ragged tail after whole tiles."""
    O = ocq.ocq
    H, W = 40, 72
    sc = ocq_synth.make_scene("bimodal", H, W, 12, 10, seed=8)
    frames = ocq_synth.fill_host(sc, 0, 22)
    train, test = frames[:12].copy(), frames[12:]
    train[::2, ::3] = np.random.default_rng(8).integers(0, 256, size=train[::2, ::3].shape, dtype=np.uint8)
    deep, lst, mf = O.OCQ_TUNE_CLASSIFY_PIXEL_DEEP, O.OCQ_TUNE_CLASSIFY_PIXEL_LIST, O.OCQ_TUNE_PIXEL_MODEL_FORM
    saved = O.ocq_tune_selected(deep), O.ocq_tune_selected(lst), O.ocq_tune_selected(mf)
    try:
        for d in (4, 5):
            for T in (1, 2, 3, 6, 12):  # lists of 8, 4, 2 codes; T = 1: no list (k = 12 > 8)
                ow, om = oracle.run(train, d, T, PIXEL, 0, test)
                for model_form in (1, 0):  # list model (exported from the lists), rows + lists
                    O.ocq_tune_select(mf, model_form)
                    for form in range(O.ocq_tune_count(lst)):
                        O.ocq_tune_select(lst, form)
                        for v in range(O.ocq_tune_count(deep)) if form == 0 else (saved[0],):
                            O.ocq_tune_select(deep, v)
                            words, mask = gpu_model_and_mask(ocq, torch, train, test, d, T, PIXEL, 0)
                            assert (words == ow).all() and (mask == om).all(), (d, T, model_form, form, v)
    finally:
        O.ocq_tune_select(deep, saved[0])
        O.ocq_tune_select(lst, saved[1])
        O.ocq_tune_select(mf, saved[2])


def test_list_model_any_alignment(ocq, torch):
    """List models classify through every launch shape: H*W % 16 != 0 (tail),
    H*W % 4 != 0 (the one-pixel form), and frames at an odd offset; model
    export equals the oracle's bitsets."""
    H_W = ((33, 48), (13, 23), (40, 72))
    for H, W in H_W:
        sc = ocq_synth.make_scene("clusters", H, W, 10, 7, seed=H)
        frames = ocq_synth.fill_host(sc, 0, 17)
        train, test = frames[:10], frames[10:]
        for d, T in ((4, 3), (5, 2)):
            ow, om = oracle.run(train, d, T, PIXEL, 0, test)
            m = ocq.build_model(torch.from_numpy(train).cuda(), d, T, "pixel")
            words = ocq.export_model(m).cpu().numpy().view(np.uint64)
            assert (words == ow).all(), (H, W, d)
            buf = torch.from_numpy(np.concatenate([np.zeros(1, np.uint8), test.reshape(-1)])).cuda()
            for off in (0, 1):
                te = buf[off:off + test.size] if off else buf[1:].clone()
                mask = torch.empty(test.shape[:3], dtype=torch.uint8, device="cuda")
                mbuf = torch.empty(mask.numel() + 1, dtype=torch.uint8, device="cuda")
                out = mbuf[off:off + mask.numel()]
                ocq.ocq.ocq_classify(m, te, test.shape[0], out, torch.cuda.current_stream())
                torch.cuda.synchronize()
                assert (out.cpu().numpy().reshape(om.shape) == om).all(), (H, W, d, off)
            m.free()


@pytest.mark.parametrize("b", [4, 8, 12, 16])
@pytest.mark.parametrize("d", [3, 4, 5, 6])
def test_block_deep_classify_forms(ocq, torch, b, d):
    """Block regions at depth >= 4: both classify forms (rows staged in shared
    memory where it applies, and L1-cached lookups by warps walking all frames)
    give the oracle's masks; partial blocks at the right and bottom edges, a
    width that is not a multiple of 128, and one that is not a multiple of 4
    (generic kernel)."""
    O = ocq.ocq
    kernel = O.OCQ_TUNE_CLASSIFY_BLOCK_DEEP
    saved = O.ocq_tune_selected(kernel)
    try:
        for H, W in ((2 * b + 3, 4 * 36), (b + 1, 139)):
            if d == 6:
                H, W = min(H, 2 * b), min(W, 3 * b + (W % 4))
            sc = ocq_synth.make_scene("sway", H, W, 9, 7, seed=40 * b + d + W)
            frames = ocq_synth.fill_host(sc, 0, 16)
            train, test = frames[:9], frames[9:]
            ow, om = oracle.run(train, d, 3, BLOCK, b, test)
            for form in range(O.ocq_tune_count(kernel)):
                O.ocq_tune_select(kernel, form)
                words, mask = gpu_model_and_mask(ocq, torch, train, test, d, 3, BLOCK, b)
                assert (words == ow).all(), (H, W, form)
                assert (mask == om).all(), (H, W, form)
    finally:
        O.ocq_tune_select(kernel, saved)


@pytest.mark.parametrize("H,W,N,F", [(37, 53, 6, 5), (1080, 1920, 10, 70)])
def test_detect_from_host_memory(ocq, torch, H, W, N, F):
    """ocq_detect_host (copies in, build, chunked classify with copies in and
    out overlapped) gives the device path's masks;
    the 1080p case spans three chunks, the last one short."""
    sc = ocq_synth.make_scene("bimodal", H, W, N, F, seed=H + F)
    train = torch.empty((N, H, W, 3), dtype=torch.uint8, device="cuda")
    test = torch.empty((F, H, W, 3), dtype=torch.uint8, device="cuda")
    ocq_synth.fill_device(sc, 0, N, train)
    ocq_synth.fill_device(sc, N, F, test)
    h_train = train.cpu().pin_memory()
    h_test = test.cpu().pin_memory()
    h_mask = torch.full((F, H, W), 9, dtype=torch.uint8).pin_memory()
    ocq.ocq.ocq_detect_host(h_train, N, h_test, F, H, W, PIXEL, 0, 3, 3, h_mask)
    m = ocq.build_model(train, 3, 3, "pixel")
    dev_mask = ocq.classify(m, test).cpu()
    m.free()
    assert torch.equal(h_mask, dev_mask)
    if H * W < 10000:
        _, om = oracle.run(h_train.numpy(), 3, 3, PIXEL, 0, h_test.numpy())
        assert (h_mask.numpy() == om).all()


def test_degenerate_inputs(ocq, torch):
    """No test frames (nothing written), a single pixel, a single training
    frame with T = 1, and a batch stream with no test frames."""
    O = ocq.ocq
    one = to_dev(np.array([[[[10, 20, 30]]]], np.uint8), torch)
    m = ocq.build_model(one, 8, 1, "pixel")
    empty = torch.empty((0, 1, 1, 3), dtype=torch.uint8, device="cuda")
    mask = torch.full((0, 1, 1), 7, dtype=torch.uint8, device="cuda")
    O.ocq_classify(m, empty, 0, mask)
    got = ocq.classify(m, to_dev(np.array([[[[10, 20, 30]]], [[[10, 20, 31]]]], np.uint8), torch)).cpu().numpy()
    m.free()
    assert got.ravel().tolist() == [0, 1]
    g = np.random.default_rng(2)
    train = g.integers(0, 256, size=(1, 9, 13, 3), dtype=np.uint8)
    for kind, block in ((FRAME, 0), (BLOCK, 4), (PIXEL, 0)):
        words, mask = gpu_model_and_mask(ocq, torch, train, train, 5, 1, kind, block)
        ow, om = oracle.run(train, 5, 1, kind, block, train)
        assert (words == ow).all() and not mask.any()
    tr = to_dev(train, torch)
    desc = [dict(train=tr, test=None, mask=None, N=1, H=9, W=13, kind=BLOCK, block=4, depth=3, T=1, F=0)]
    b = O.ocq_batch_create(desc)
    try:
        O.ocq_batch_run(b)
        O.ocq_batch_status(b)
        assert (ocq.export_model(b.model(0)).cpu().numpy().view(np.uint64) ==
                oracle.build_model(train, 3, 1, BLOCK, 4)).all()
    finally:
        b.destroy()
