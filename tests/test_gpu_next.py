"""Parity of the redraw (Sec. 2), group-of-frames build (Sec. 3) and the
evaluation counts (Sec. 5) with the CPU oracle, bit-exact."""
import numpy as np
import pytest

import ocq_synth
import oracle

pytestmark = pytest.mark.gpu
FRAME, BLOCK, PIXEL = 0, 1, 2


@pytest.fixture(scope="module")
def ocq(cuda_ready):
    return cuda_ready


@pytest.fixture(scope="module")
def torch():
    import torch

    return torch


def test_redraw_all_colours(ocq, torch):
    v = np.arange(1 << 24, dtype=np.uint32)
    rgb = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], axis=1).astype(np.uint8)
    dev = torch.from_numpy(rgb).cuda()
    for d in range(1, 9):
        got = ocq.redraw(dev, d).cpu().numpy()
        assert (got == oracle.redraw(rgb, d)).all(), d


@pytest.mark.parametrize("npix,offset", [(1, 0), (5, 1), (16, 0), (1000, 3), (4097, 0), (123457, 5)])
def test_redraw_ragged_unaligned_and_in_place(ocq, torch, npix, offset):
    g = np.random.default_rng(npix)
    buf = g.integers(0, 256, size=npix * 3 + offset, dtype=np.uint8)
    rgb = buf[offset:].reshape(npix, 3)
    dev = torch.from_numpy(buf).cuda()
    view = dev[offset:]
    for d in (2, 5):
        out = torch.empty(npix * 3, dtype=torch.uint8, device="cuda")
        ocq.ocq.ocq_redraw(view, npix, d, out)
        assert (out.cpu().numpy().reshape(npix, 3) == oracle.redraw(rgb, d)).all()
    inplace = view.clone()
    ocq.ocq.ocq_redraw(inplace, npix, 4, inplace)
    assert (inplace.cpu().numpy().reshape(npix, 3) == oracle.redraw(rgb, 4)).all()
    ocq.device_status()


@pytest.mark.parametrize("F,H,W", [(1, 1, 1), (3, 7, 9), (4, 32, 64), (2, 1080, 1920), (5, 33, 31)])
def test_confusion_counts(ocq, torch, F, H, W):
    g = np.random.default_rng(F * 1000 + W)
    mask = g.integers(0, 2, size=(F, H, W), dtype=np.uint8) * g.integers(1, 256, size=(F, H, W), dtype=np.uint8)
    gt = g.integers(0, 2, size=(F, H, W), dtype=np.uint8)
    got = ocq.confusion(torch.from_numpy(mask).cuda(), torch.from_numpy(gt).cuda()).cpu().numpy()
    want = oracle.confusion(mask, gt)
    assert (got.astype(np.uint64) == want).all()
    a, b = ocq.f_scores(got.sum(axis=0)), oracle.f_scores(want)
    for k in ("P0", "R0", "F0", "F1"):
        assert a[k] == pytest.approx(b[k], rel=0, abs=1e-12), k


def test_confusion_of_classified_scene(ocq, torch):
    """F0 of the classify masks of a synthetic scene against the generator's
    ground truth: counts equal the oracle's on the same masks, and the oracle's
    own masks give the same counts (mask parity)."""
    sc = ocq_synth.make_scene("clusters", 60, 80, 8, 10, seed=21)
    frames, gt = ocq_synth.fill_host(sc, 0, 18, with_gt=True)
    train, test, gt = frames[:8], frames[8:], gt[8:]
    m = ocq.build_model(torch.from_numpy(train).cuda(), 4, 4, "frame")
    mask = ocq.classify(m, torch.from_numpy(test).cuda())
    counts = ocq.confusion(mask, torch.from_numpy(gt).cuda()).cpu().numpy().astype(np.uint64)
    m.free()
    _, omask = oracle.run(train, 4, 4, FRAME, 0, test)
    assert (counts == oracle.confusion(omask, gt)).all()
    assert ocq.f_scores(counts.sum(axis=0))["F0"] > 0.9


CASES = [(FRAME, 0, d) for d in (1, 3, 5, 7)] + [(BLOCK, b, d) for b, d in ((4, 2), (5, 4), (8, 5))] + \
        [(PIXEL, 0, d) for d in (2, 3, 5, 7)]


@pytest.mark.parametrize("kind,block,d", CASES)
@pytest.mark.parametrize("group", [2, 3, 5])
def test_group_of_frames_build(ocq, torch, kind, block, d, group):
    g = np.random.default_rng(kind * 100 + block * 10 + d + group)
    H, W = (6, 7) if kind == PIXEL and d >= 5 else (13, 17)
    N = 11
    palette = g.integers(0, 256, size=(6, 3), dtype=np.uint8)
    train = palette[g.integers(0, 6, size=(N, H, W))]
    train[::4] = g.integers(0, 256, size=train[::4].shape, dtype=np.uint8)
    test = palette[g.integers(0, 6, size=(3, H, W))]
    G = -(-N // group)
    for T in sorted({1, (G + 1) // 2, G}):
        m = ocq.build_model_groups(torch.from_numpy(train).cuda(), d, T, group, kind, block)
        words = ocq.export_model(m).cpu().numpy().view(np.uint64)
        mask = ocq.classify(m, torch.from_numpy(test).cuda()).cpu().numpy()
        m.free()
        ow, om = oracle.run(train, d, T, kind, block, test, group=group)
        assert (words == ow).all(), T
        assert (mask == om).all(), T
    ocq.device_status()


def test_group_of_frames_bad_threshold(ocq, torch):
    train = torch.zeros((5, 4, 4, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(ocq.OcqError):
        ocq.build_model_groups(train, 3, 4, 2, "frame")  # ceil(5 / 2) = 3 trees < T = 4
    m = ocq.build_model_groups(train, 3, 3, 2, "frame")
    m.free()
