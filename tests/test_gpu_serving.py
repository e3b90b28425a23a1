"""Served form (window re-merge, the reading of the paper's "octree
updation"): each frame's mask equals the oracle's under the window semantics,
is the same whether the camera runs alone or in a mix, and admission respects
the HBM budget."""
import numpy as np
import pytest

import ocq_synth
import oracle

pytestmark = pytest.mark.gpu
FRAME, BLOCK, PIXEL = 0, 1, 2

# (scene, H, W, region, block, depth, T, N, K, test frames)
CAMERAS = [
    ("clusters", 40, 48, FRAME, 0, 4, 3, 6, 4, 14),
    ("sway", 32, 48, BLOCK, 8, 3, 2, 5, 3, 11),
    ("bimodal", 32, 64, PIXEL, 0, 3, 2, 6, 5, 13),
    ("sway", 24, 40, PIXEL, 0, 4, 3, 7, 7, 15),
    ("clusters", 30, 38, BLOCK, 5, 2, 4, 8, 2, 9),
]


def _frames(i, cam):
    scene, H, W, region, block, d, T, N, K, F = cam
    sc = ocq_synth.make_scene(scene, H, W, N, F, 4000 + i)
    return ocq_synth.fill_host(sc, 0, N + F)


def _window_oracle(frames, cam):
    """Masks under the window semantics, from the oracle alone: test frame t
    uses M_floor(t/K), M_k = merge of frames [kK, kK + N - 1]."""
    scene, H, W, region, block, d, T, N, K, F = cam
    out = []
    models = {}
    for t in range(F):
        k = t // K
        if k not in models:
            models[k] = oracle.build_model(frames[k * K:k * K + N], d, T, region, block)
        out.append(oracle.classify(models[k], frames[N + t:N + t + 1], d, region, block)[0])
    return out


def _run(ocq, torch, cams, frames, order):
    """Submits (camera, t) pairs in `order` to one server; returns masks."""
    O = ocq.ocq
    srv = O.ocq_server_create(1 << 34, 16)
    ids, dev, masks = {}, {}, {}
    try:
        for i in sorted({c for c, _ in order}):
            scene, H, W, region, block, d, T, N, K, F = cams[i]
            dev[i] = torch.from_numpy(frames[i]).cuda()
            torch.cuda.synchronize()
            ids[i] = O.ocq_server_admit(srv, H, W, region, block, d, T, N, K, dev[i][:N].contiguous())
            assert ids[i] is not None
            masks[i] = torch.full((F, H, W), 9, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()  # the cameras' streams do not wait on torch's
        for i, t in order:
            N = cams[i][7]
            O.ocq_server_submit(srv, ids[i], dev[i][N + t], masks[i][t], tag=i * 1000 + t)
        O.ocq_server_sync(srv)
        done = O.ocq_server_poll(srv, 10000)
        assert len(done) == len(order)
        assert all(d_ >= a for _, _, _, a, d_ in done)
        for i in ids:
            O.ocq_server_release(srv, ids[i])
        ocq.device_status()
        return {i: masks[i].cpu().numpy() for i in masks}
    finally:
        srv.destroy()


def test_serving_window_semantics_alone_and_mixed(cuda_ready):
    import torch

    ocq = cuda_ready
    frames = [_frames(i, c) for i, c in enumerate(CAMERAS)]
    alone = {}
    for i, c in enumerate(CAMERAS):
        alone.update(_run(ocq, torch, CAMERAS, frames, [(i, t) for t in range(c[9])]))
    # the mix: all cameras at once, their frames interleaved in a seeded order
    rng = np.random.default_rng(3)
    queues = {i: list(range(c[9])) for i, c in enumerate(CAMERAS)}
    order = []
    while any(queues.values()):
        i = int(rng.choice([k for k, q in queues.items() if q]))
        order.append((i, queues[i].pop(0)))
    mixed = _run(ocq, torch, CAMERAS, frames, order)
    for i, c in enumerate(CAMERAS):
        assert (alone[i] == mixed[i]).all(), i
        expect = _window_oracle(frames[i], c)
        for t in range(c[9]):
            assert (mixed[i][t] == expect[t]).all(), (i, t)


def test_serving_admission_by_footprint(cuda_ready):
    import torch

    ocq = cuda_ready
    O = ocq.ocq
    cam = CAMERAS[2]
    scene, H, W, region, block, d, T, N, K, F = cam
    fp = O.ocq_server_camera_footprint(H, W, region, block, d, T, N, K)
    assert fp > 0
    frames = torch.from_numpy(_frames(2, cam)).cuda()
    torch.cuda.synchronize()
    srv = O.ocq_server_create(fp + fp // 2, 8)  # room for one camera, not two
    try:
        a = O.ocq_server_admit(srv, H, W, region, block, d, T, N, K, frames[:N].contiguous())
        assert a is not None
        assert O.ocq_server_admit(srv, H, W, region, block, d, T, N, K, frames[:N].contiguous()) is None
        used, budget, _ = O.ocq_server_usage(srv)
        assert used == fp and budget == fp + fp // 2
        O.ocq_server_release(srv, a)
        b = O.ocq_server_admit(srv, H, W, region, block, d, T, N, K, frames[:N].contiguous())
        assert b is not None
        O.ocq_server_release(srv, b)
        assert O.ocq_server_usage(srv)[0] == 0
    finally:
        srv.destroy()
