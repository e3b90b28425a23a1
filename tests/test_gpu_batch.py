"""Batched form: every stream's model and masks from the one persistent,
graph-replayed launch equal the plain per-stream path and the oracle
(bit-exact): every stream of the small mix in full, every stream of the
64-stream preset at sampled regions."""
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


def _streams_host(specs, torch):
    out = []
    for i, (kind, scene, H, W, N, F, region, block, d, T) in enumerate(specs):
        sc = ocq_synth.make_scene(scene, H, W, N, F, 1000 + i)
        frames = ocq_synth.fill_host(sc, 0, N + F)
        out.append(dict(train=torch.from_numpy(frames[:N].copy()).cuda(),
                        test=torch.from_numpy(frames[N:].copy()).cuda(),
                        mask=torch.full((F, H, W), 7, dtype=torch.uint8, device="cuda"),
                        N=N, H=H, W=W, kind=region, block=block, depth=d, T=T, F=F,
                        host_train=frames[:N], host_test=frames[N:]))
    return out


SMALL_MIX = [
    (0, "clusters", 120, 160, 8, 8, FRAME, 0, 4, 4),
    (0, "sway", 37, 53, 12, 9, FRAME, 0, 6, 5),
    (0, "sway", 20, 30, 5, 4, FRAME, 0, 8, 2),
    (0, "clusters", 64, 96, 9, 6, BLOCK, 8, 5, 3),
    (0, "sway", 50, 70, 10, 7, BLOCK, 16, 3, 4),
    (0, "sway", 33, 47, 7, 5, BLOCK, 5, 4, 7),
    (0, "bimodal", 48, 64, 20, 11, PIXEL, 0, 3, 7),
    (0, "bimodal", 29, 37, 15, 6, PIXEL, 0, 2, 5),
    (0, "clusters", 40, 56, 12, 5, PIXEL, 0, 4, 4),
    (0, "sway", 24, 40, 9, 5, PIXEL, 0, 5, 3),
    (0, "clusters", 13, 23, 10, 4, PIXEL, 0, 4, 5),  # H*W % 4 != 0: rows kept beside the index
    (0, "bimodal", 12, 20, 30, 3, PIXEL, 0, 5, 2),  # floor(N/T) = 15 > 8: rows, no index
    (0, "bimodal", 16, 1024, 6, 4, PIXEL, 0, 1, 2),
    (0, "clusters", 31, 33, 11, 3, FRAME, 0, 1, 11),
    (0, "sway", 40, 64, 9, 6, BLOCK, 8, 3, 4),      # W % 8 == 0: warp tiles (the persistent kernel's too)
    (0, "clusters", 48, 80, 8, 5, BLOCK, 16, 4, 3),  # 16 x 16 at depth 4: direct-table tiles
]


def _plain(ocq, s):
    m = ocq.build_model(s["train"], s["depth"], s["T"], s["kind"], s["block"])
    words = ocq.export_model(m).cpu().numpy()
    mask = ocq.classify(m, s["test"]).cpu().numpy()
    m.free()
    return words, mask


@pytest.mark.parametrize("mode,staging", [(0, 0), (0, 1), (1, 0), (2, 0)])
def test_batch_small_mix_matches_plain_and_oracle(ocq, mode, staging):
    """Every form: the persistent work-list kernel (0; per-pixel depth <= 3
    rows through L1 or staged in shared memory), the graph of per-stream
    branches (1) and the grouped launches per kernel body (2; the mix holds
    streams those bodies cover and streams left to their plain kernels)."""
    import torch

    S = _streams_host(SMALL_MIX, torch)
    b = ocq.ocq.ocq_batch_create(S)
    try:
        ocq.ocq.ocq_batch_set_mode(b, mode)
        ocq.ocq.ocq_batch_set_staging(b, staging)
        assert ocq.ocq.ocq_batch_get_mode(b) == mode and ocq.ocq.ocq_batch_get_staging(b) == staging
        for rep in range(2):  # first run captures the graph, second replays it
            for s in S:
                s["mask"].fill_(7)
            ocq.ocq.ocq_batch_run(b)
            ocq.ocq.ocq_batch_status(b)
            for i, s in enumerate(S):
                words = ocq.export_model(b.model(i)).cpu().numpy()
                pw, pm = _plain(ocq, s)
                assert (words == pw).all(), (rep, i)
                assert (s["mask"].cpu().numpy() == pm).all(), (rep, i)
        for i in range(len(S)):
            s = S[i]
            ow, om = oracle.run(s["host_train"], s["depth"], s["T"], s["kind"], s["block"], s["host_test"])
            assert (ocq.export_model(b.model(i)).cpu().numpy().view(np.uint64) == ow).all(), i
            assert (s["mask"].cpu().numpy() == om).all(), i
    finally:
        b.destroy()


def test_batch_tiles_and_autotune_keep_results(ocq):
    import torch

    S = _streams_host(SMALL_MIX[:8], torch)
    b = ocq.ocq.ocq_batch_create(S)
    try:
        ocq.ocq.ocq_batch_run(b)
        ref = [s["mask"].clone() for s in S]
        for kind, units in ((FRAME, 3), (BLOCK, 1), (PIXEL, 500)):
            ocq.ocq.ocq_batch_set_work(b, kind, units)
        for s in S:
            s["mask"].fill_(9)
        ocq.ocq.ocq_batch_run(b)
        ocq.ocq.ocq_batch_status(b)
        assert all((s["mask"] == r).all().item() for s, r in zip(S, ref))
        ocq.ocq.ocq_batch_autotune(b, 1)
        assert ocq.ocq.ocq_batch_get_mode(b) in (0, 1)
        for mode in (ocq.ocq.ocq_batch_get_mode(b), 1 - ocq.ocq.ocq_batch_get_mode(b)):
            ocq.ocq.ocq_batch_set_mode(b, mode)
            for s in S:
                s["mask"].fill_(9)
            ocq.ocq.ocq_batch_run(b)
            ocq.ocq.ocq_batch_status(b)
            assert all((s["mask"] == r).all().item() for s, r in zip(S, ref)), mode
    finally:
        b.destroy()


def _sampled_oracle_check(ocq, s, model, mask, rng):
    """Stream ``s`` against the oracle at sampled regions: regions are
    independent (Sec. 3), so a block (or a set of pixel locations) cropped out
    of every frame is its own video.  Whole-frame streams: the model in full
    and the masks of three test frames."""
    import torch

    H, W, F, d, T, kind, b = s["H"], s["W"], s["F"], s["depth"], s["T"], s["kind"], s["block"]
    words = ocq.export_model(model)
    if kind == FRAME:
        ow, om = oracle.run(s["train"].cpu().numpy(), d, T, FRAME, 0, s["test"][[0, F // 2, F - 1]].cpu().numpy())
        assert (words.cpu().numpy().view(np.uint64) == ow).all()
        assert (mask[[0, F // 2, F - 1]].cpu().numpy() == om).all()
    elif kind == BLOCK:
        bh, bw = (H + b - 1) // b, (W + b - 1) // b
        picks = {0, bh * bw - 1, bw - 1, (bh - 1) * bw} | set(rng.integers(0, bh * bw, size=12).tolist())
        for r in sorted(picks):
            y0, x0 = (r // bw) * b, (r % bw) * b
            tr = s["train"][:, y0:y0 + b, x0:x0 + b].contiguous().cpu().numpy()
            te = s["test"][:, y0:y0 + b, x0:x0 + b].contiguous().cpu().numpy()
            ow, om = oracle.run(tr, d, T, BLOCK, b, te)
            assert (words[r].cpu().numpy().view(np.uint64) == ow[0]).all(), r
            assert (mask[:, y0:y0 + b, x0:x0 + b].cpu().numpy() == om).all(), r
    else:
        hw = H * W
        picks = {0, 1, 127, 128, hw // 2, hw - 1} | set(rng.integers(0, hw, size=200).tolist())
        idx = np.array(sorted(picks), np.int64)
        ys, xs = torch.from_numpy(idx // W).cuda(), torch.from_numpy(idx % W).cuda()
        ow, om = oracle.run(s["train"][:, ys, xs].cpu().numpy()[:, None], d, T, PIXEL, 0,
                            s["test"][:, ys, xs].cpu().numpy()[:, None])
        assert (words[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint64) == ow).all()
        assert (mask[:, ys, xs].cpu().numpy() == om[:, 0]).all()


def test_batch_64_stream_preset_matches_plain(ocq):
    """The 64-stream preset (resolutions up to 1920x1080, depth 3-5, 1x1 /
    8x8 / whole-frame regions), frames generated on the device: both forms
    equal the plain path, and every stream equals the oracle at sampled
    regions."""
    import torch

    descs = []
    for wl in configs.batched_streams():
        sc = ocq_synth.make_scene(wl.scene_kind, wl.H, wl.W, wl.N, wl.F, wl.seed, wl.stream)
        tr = torch.empty((wl.N, wl.H, wl.W, 3), dtype=torch.uint8, device="cuda")
        te = torch.empty((wl.F, wl.H, wl.W, 3), dtype=torch.uint8, device="cuda")
        ocq_synth.fill_device(sc, 0, wl.N, tr)
        ocq_synth.fill_device(sc, wl.N, wl.F, te)
        descs.append(dict(train=tr, test=te, mask=torch.empty((wl.F, wl.H, wl.W), dtype=torch.uint8, device="cuda"),
                          N=wl.N, H=wl.H, W=wl.W, kind=wl.region, block=wl.block, depth=wl.depth, T=wl.T, F=wl.F))
    b = ocq.ocq.ocq_batch_create(descs)
    try:
        ocq.ocq.ocq_batch_run(b)
        ocq.ocq.ocq_batch_status(b)
        persistent = [s["mask"].clone() for s in descs]
        for mode in (2, 1):  # grouped launches, then the graph of per-stream branches
            ocq.ocq.ocq_batch_set_mode(b, mode)
            for s in descs:
                s["mask"].fill_(5)
            ocq.ocq.ocq_batch_run(b)
            ocq.ocq.ocq_batch_status(b)
            assert all((s["mask"] == p).all().item() for s, p in zip(descs, persistent)), mode
        for i, s in enumerate(descs):
            m = ocq.build_model(s["train"], s["depth"], s["T"], s["kind"], s["block"])
            pmask = ocq.classify(m, s["test"])
            same_model = (ocq.export_model(b.model(i)) == ocq.export_model(m)).all().item()
            same_mask = (s["mask"] == pmask).all().item()
            m.free()
            assert same_model and same_mask, i
        rng = np.random.default_rng(64)
        for i, s in enumerate(descs):
            _sampled_oracle_check(ocq, s, b.model(i), s["mask"], rng)
    finally:
        b.destroy()
