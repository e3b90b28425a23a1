"""Served form (window re-merge, the reading of the octree update the
paper's Sec. 4 title names): each frame's mask equals the oracle's under the window semantics,
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


def _first(streams, W, region, depth=None):
    for i, s in enumerate(streams):
        if s.wl.W == W and s.wl.region == region and (depth is None or s.wl.depth == depth):
            return i
    raise LookupError((W, region, depth))


def test_serving_preset_cameras_full_size_sampled(cuda_ready):
    """Cameras of the 256-camera preset at full size (3840x2160 per-pixel
    d = 5, 1920x1080 8x8 blocks d = 5, 320x240 whole frame), two windows each
    (N = K = 30, T = 10), frames rendered on the device; the masks at sampled
    pixel locations / blocks (whole frame: every pixel) equal the oracle's
    under the window semantics, on the same frames rendered by the host
    generator."""
    import torch

    from ocq_synth import configs

    ocq = cuda_ready
    O = ocq.ocq
    streams = configs.serving_streams()
    picks = [_first(streams, 3840, PIXEL, 5), _first(streams, 1920, BLOCK, 5), _first(streams, 320, FRAME)]
    srv = O.ocq_server_create(72 << 30, 8)
    rng = np.random.default_rng(77)
    try:
        for i in picks:
            wl = streams[i].wl
            H, W, N, K, T, d = wl.H, wl.W, wl.N, wl.N, wl.T, wl.depth
            F = 2 * K
            sc = ocq_synth.make_scene(wl.scene_kind, H, W, N, F, wl.seed, wl.stream)
            dev = torch.empty((N + F, H, W, 3), dtype=torch.uint8, device="cuda")
            ocq_synth.fill_device(sc, 0, N + F, dev)
            masks = torch.full((F, H, W), 7, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            cam = O.ocq_server_admit(srv, H, W, wl.region, wl.block, d, T, N, K, dev[:N])
            assert cam is not None
            for t in range(F):
                O.ocq_server_submit(srv, cam, dev[N + t], masks[t], tag=t)
            O.ocq_server_sync(srv)
            assert len(O.ocq_server_poll(srv, 1000)) == F
            O.ocq_server_release(srv, cam)
            if wl.region == PIXEL:
                idx = np.sort(rng.choice(H * W, size=300, replace=False))
                frames = ocq_synth.fill_pixels_host(sc, 0, N + F, idx).reshape(N + F, len(idx), 1, 3)
                got = masks.reshape(F, H * W)[:, torch.from_numpy(idx).cuda()].cpu().numpy().reshape(F, len(idx), 1)
            elif wl.region == BLOCK:
                b = wl.block
                bw = -(-W // b)
                blocks = np.sort(rng.choice(bw * (-(-H // b)), size=40, replace=False))
                cols = []
                for r in blocks:
                    y0, x0 = (r // bw) * b, (r % bw) * b
                    cols.append(np.array([(y0 + yy) * W + x0 + xx for yy in range(b) for xx in range(b)]))
                idx = np.concatenate(cols)
                # the sampled blocks side by side: one b-row frame of len(blocks) blocks
                frames = ocq_synth.fill_pixels_host(sc, 0, N + F, idx).reshape(N + F, len(blocks), b, b, 3)
                frames = frames.transpose(0, 2, 1, 3, 4).reshape(N + F, b, len(blocks) * b, 3)
                flat = masks.reshape(F, H * W)[:, torch.from_numpy(idx).cuda()].cpu().numpy()
                got = flat.reshape(F, len(blocks), b, b).transpose(0, 2, 1, 3).reshape(F, b, len(blocks) * b)
            else:
                frames = ocq_synth.fill_host(sc, 0, N + F)
                got = masks.cpu().numpy()
            kind, block = wl.region, wl.block
            for k in range(2):  # window k: M_k from frames [kK, kK + N), then test frames kK .. kK + K - 1
                model = oracle.build_model(frames[k * K:k * K + N], d, T, kind, block)
                expect = oracle.classify(model, frames[N + k * K:N + k * K + K], d, kind, block)
                assert (got[k * K:k * K + K] == expect).all(), (i, k)
            del dev, masks
            torch.cuda.empty_cache()
    finally:
        srv.destroy()


@pytest.mark.parametrize("kind,block,d", [(BLOCK, 5, 4), (PIXEL, 0, 5)])
def test_serving_snapshot_and_resume(cuda_ready, kind, block, d):
    """A camera checkpointed after 13 test frames (mid-window; re-merges after
    frames 3, 7, 11) and resumed in a fresh server gives, for frames 13-21,
    the masks of the window semantics, as if it had never stopped.  The
    per-pixel d = 5 camera (N = 6, T = 3) keeps list models: the snapshot
    expands one, the resume reads it back into lists."""
    import torch

    ocq = cuda_ready
    O = ocq.ocq
    H, W, T, N, K, F, cut = 30, 44, 3, 6, 4, 22, 13
    sc = ocq_synth.make_scene("sway", H, W, N, F, 123)
    host = ocq_synth.fill_host(sc, 0, N + F)
    dev = torch.from_numpy(host).cuda()
    masks = torch.full((F, H, W), 9, dtype=torch.uint8, device="cuda")
    wpr = max(1, 8 ** d // 64)
    regions = -(-H // block) * -(-W // block) if kind == BLOCK else H * W
    words = torch.zeros((regions, wpr), dtype=torch.int64, device="cuda")
    ring = torch.zeros((N, H, W, 3), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    srv = O.ocq_server_create(1 << 28, 2)
    try:
        cam = O.ocq_server_admit(srv, H, W, kind, block, d, T, N, K, dev[:N])
        for t in range(cut):
            O.ocq_server_submit(srv, cam, dev[N + t], masks[t], tag=t)
        assert O.ocq_server_snapshot(srv, cam, words, ring) == cut
        torch.cuda.synchronize()
        O.ocq_server_release(srv, cam)
    finally:
        srv.destroy()
    srv = O.ocq_server_create(1 << 28, 2)
    try:
        cam = O.ocq_server_resume(srv, H, W, kind, block, d, T, N, K, words, ring, cut)
        assert cam is not None
        for t in range(cut, F):
            O.ocq_server_submit(srv, cam, dev[N + t], masks[t], tag=t)
        O.ocq_server_sync(srv)
        O.ocq_server_release(srv, cam)
    finally:
        srv.destroy()
    expect = _window_oracle(host, ("sway", H, W, kind, block, d, T, N, K, F))
    got = masks.cpu().numpy()
    for t in range(F):
        assert (got[t] == expect[t]).all(), t
