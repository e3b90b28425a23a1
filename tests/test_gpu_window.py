"""Serving windows: the three forms a camera's window takes (leaf bitsets with
resident counts, per-pixel leaf codes, or the frames themselves) each give the
masks of the window semantics (test frame t against the merge of global frames
[kK, kK + N - 1], k = floor(t / K); Alg. 2 and 3 on the oracle), and each
reserves what its form needs."""
import numpy as np
import pytest

import ocq_synth
import oracle

pytestmark = pytest.mark.gpu
FRAME, BLOCK, PIXEL = 0, 1, 2

# (scene, H, W, region, block, depth, T, N, K, test frames, form)
#   form 1: leaf bitsets + counts, 2: per-pixel codes, 0: frames
CAMERAS = [
    ("clusters", 36, 52, FRAME, 0, 5, 3, 7, 3, 12, 1),
    ("sway", 96, 128, FRAME, 0, 6, 2, 5, 4, 9, 1),
    ("clusters", 6, 10, FRAME, 0, 6, 2, 4, 3, 7, 0),     # a bitset (32 KB) larger than a frame
    ("sway", 33, 40, BLOCK, 8, 5, 3, 9, 4, 10, 2),
    ("sway", 40, 40, BLOCK, 16, 3, 4, 6, 5, 11, 2),
    ("sway", 34, 38, BLOCK, 17, 3, 2, 5, 2, 7, 0),       # blocks wider than 16
    ("bimodal", 22, 30, PIXEL, 0, 3, 2, 6, 4, 10, 2),
    ("clusters", 17, 23, PIXEL, 0, 4, 3, 9, 2, 8, 2),
    ("bimodal", 16, 20, PIXEL, 0, 5, 1, 12, 5, 11, 2),   # floor(N/T) > 8: rows, every distinct leaf counted
    ("sway", 12, 16, PIXEL, 0, 6, 2, 5, 3, 7, 0),        # depth 6: frames
]


def _window_oracle(frames, cam):
    scene, H, W, region, block, d, T, N, K, F, form = cam
    out, models = [], {}
    for t in range(F):
        k = t // K
        if k not in models:
            models[k] = oracle.build_model(frames[k * K:k * K + N], d, T, region, block)
        out.append(oracle.classify(models[k], frames[N + t:N + t + 1], d, region, block)[0])
    return np.stack(out)


@pytest.mark.parametrize("i", range(len(CAMERAS)))
def test_window_forms_follow_the_window_semantics(cuda_ready, i):
    import torch

    O = cuda_ready.ocq
    cam = CAMERAS[i]
    scene, H, W, region, block, d, T, N, K, F, form = cam
    hw = H * W
    slot = {1: max(1, 8 ** d // 32) * 4, 2: 2 * hw, 0: 3 * hw}[form]
    assert O.ocq_server_window_bytes(H, W, region, block, d, T, N, K) == N * slot
    sc = ocq_synth.make_scene(scene, H, W, N, F, 7100 + i)
    host = ocq_synth.fill_host(sc, 0, N + F)
    dev = torch.from_numpy(host).cuda()
    masks = torch.full((F, H, W), 9, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    srv = O.ocq_server_create(1 << 28, 2)
    try:
        c = O.ocq_server_admit(srv, H, W, region, block, d, T, N, K, dev[:N].contiguous())
        assert c is not None
        for t in range(F):
            O.ocq_server_submit(srv, c, dev[N + t], masks[t], tag=t)
        O.ocq_server_sync(srv)
        model = cuda_ready.export_model(O.ocq_server_camera_model(srv, c)).cpu().numpy().view(np.uint64)
        O.ocq_server_release(srv, c)
    finally:
        srv.destroy()
    assert (masks.cpu().numpy() == _window_oracle(host, cam)).all()
    # after F test frames the model is M_floor(F/K), merged from frames [kK, kK + N)
    k = F // K
    assert (model == oracle.build_model(host[k * K:k * K + N], d, T, region, block)).all()


def test_window_footprints_shrink(cuda_ready):
    """A 4K whole-frame camera keeps kilobytes instead of its frames; 4K
    per-pixel cameras keep 2 bytes per pixel and frame instead of 3, and one
    model instead of two."""
    O = cuda_ready.ocq
    H, W, N, K, T = 2160, 3840, 30, 30, 10
    frame = O.ocq_server_camera_footprint(H, W, FRAME, 0, 4, T, N, K)
    assert frame < 1 << 20
    for d in (3, 5):
        model = O.ocq_model_footprint(H, W, PIXEL, 0, d)
        fp = O.ocq_server_camera_footprint(H, W, PIXEL, 0, d, T, N, K)
        if d == 5:
            model = H * W * 16  # a list model (floor(N/T) = 3 <= 8)
        assert fp == model + N * H * W * 2


@pytest.mark.parametrize("chunks", [1, 3, 7])
def test_batched_submits_follow_the_window_semantics(cuda_ready, chunks):
    """Every camera of the set in one server, their frames interleaved and
    handed over in `chunks` batched submits (continuous batching: a tick holds
    several frames of several cameras and splits at each camera's re-merge);
    each camera's masks and final model follow the window semantics."""
    import torch

    O = cuda_ready.ocq
    srv = O.ocq_server_create(1 << 30, len(CAMERAS))
    hosts, devs, masks, ids = [], [], [], []
    try:
        for i, cam in enumerate(CAMERAS):
            scene, H, W, region, block, d, T, N, K, F, form = cam
            host = ocq_synth.fill_host(ocq_synth.make_scene(scene, H, W, N, F, 7300 + i), 0, N + F)
            hosts.append(host)
            devs.append(torch.from_numpy(host).cuda())
            masks.append(torch.full((F, H, W), 9, dtype=torch.uint8, device="cuda"))
        torch.cuda.synchronize()
        for i, cam in enumerate(CAMERAS):
            scene, H, W, region, block, d, T, N, K, F, form = cam
            ids.append(O.ocq_server_admit(srv, H, W, region, block, d, T, N, K, devs[i][:N].contiguous()))
            assert ids[-1] is not None
        order = [(i, t) for t in range(max(c[9] for c in CAMERAS)) for i, c in enumerate(CAMERAS) if t < c[9]]
        rng = np.random.default_rng(chunks)
        cuts = sorted(rng.choice(np.arange(1, len(order)), size=chunks - 1, replace=False).tolist()) if chunks > 1 else []
        for a, b in zip([0] + cuts, cuts + [len(order)]):
            part = order[a:b]
            O.ocq_server_submit_many(srv, [ids[i] for i, _ in part],
                                     [devs[i][CAMERAS[i][7] + t] for i, t in part],
                                     [masks[i][t] for i, t in part], [1000 * i + t for i, t in part])
        O.ocq_server_sync(srv)
        done = O.ocq_server_poll(srv, 100000)
        assert len(done) == len(order)
        for i, cam in enumerate(CAMERAS):
            scene, H, W, region, block, d, T, N, K, F, form = cam
            assert (masks[i].cpu().numpy() == _window_oracle(hosts[i], cam)).all(), i
            model = cuda_ready.export_model(O.ocq_server_camera_model(srv, ids[i])).cpu().numpy().view(np.uint64)
            k = F // K
            assert (model == oracle.build_model(hosts[i][k * K:k * K + N], d, T, region, block)).all(), i
    finally:
        srv.destroy()


def test_batching_window_holds_frames_and_keeps_the_semantics(cuda_ready):
    """With a batching window the frames of tick cameras wait on the host
    (nothing completes before the window ends), then run in ticks that hold
    several frames per camera; masks and final models still follow the window
    semantics."""
    import time

    import torch

    O = cuda_ready.ocq
    cams = [c for c in CAMERAS if c[10] in (1, 2)]
    srv = O.ocq_server_create(1 << 30, len(cams))
    hosts, devs, masks, ids = [], [], [], []
    try:
        for i, cam in enumerate(cams):
            scene, H, W, region, block, d, T, N, K, F, form = cam
            host = ocq_synth.fill_host(ocq_synth.make_scene(scene, H, W, N, F, 7500 + i), 0, N + F)
            hosts.append(host)
            devs.append(torch.from_numpy(host).cuda())
            masks.append(torch.full((F, H, W), 9, dtype=torch.uint8, device="cuda"))
        torch.cuda.synchronize()
        for i, cam in enumerate(cams):
            scene, H, W, region, block, d, T, N, K, F, form = cam
            ids.append(O.ocq_server_admit(srv, H, W, region, block, d, T, N, K, devs[i][:N].contiguous()))
            assert ids[-1] is not None
        O.ocq_server_sync(srv)  # every M_0 built: frames are held only by the window
        O.ocq_server_set_batching(srv, 1.0, 2)
        order = [(i, t) for t in range(max(c[9] for c in cams)) for i, c in enumerate(cams) if t < c[9]]
        t0 = time.monotonic()
        for i, t in order:
            O.ocq_server_submit(srv, ids[i], devs[i][cams[i][7] + t], masks[i][t], tag=1000 * i + t)
        early = O.ocq_server_poll(srv, 100000)
        if time.monotonic() - t0 < 0.5:
            assert early == []
        O.ocq_server_set_batching(srv, 0.002, 2)
        done = list(early)
        deadline = time.monotonic() + 20.0
        while len(done) < len(order) and time.monotonic() < deadline:
            time.sleep(0.003)
            done += O.ocq_server_poll(srv, 100000)
        O.ocq_server_sync(srv)
        done += O.ocq_server_poll(srv, 100000)
        assert len(done) == len(order)
        for i, cam in enumerate(cams):
            scene, H, W, region, block, d, T, N, K, F, form = cam
            assert (masks[i].cpu().numpy() == _window_oracle(hosts[i], cam)).all(), i
            model = cuda_ready.export_model(O.ocq_server_camera_model(srv, ids[i])).cpu().numpy().view(np.uint64)
            k = F // K
            assert (model == oracle.build_model(hosts[i][k * K:k * K + N], d, T, region, block)).all(), i
    finally:
        srv.destroy()


def test_array_submits_and_polls(cuda_ready):
    """The numpy-array bindings (device addresses in uint64 arrays, completions
    as a structured array) submit and report the same frames as the list
    forms: every frame once, its tag back, masks under the window semantics."""
    import time

    import torch

    O = cuda_ready.ocq
    cams = [CAMERAS[3], CAMERAS[6], CAMERAS[0]]  # block codes, pixel codes, whole-frame bitsets
    srv = O.ocq_server_create(1 << 30, len(cams))
    hosts, devs, masks, ids = [], [], [], []
    try:
        for i, cam in enumerate(cams):
            scene, H, W, region, block, d, T, N, K, F, form = cam
            host = ocq_synth.fill_host(ocq_synth.make_scene(scene, H, W, N, F, 7700 + i), 0, N + F)
            hosts.append(host)
            devs.append(torch.from_numpy(host).cuda())
            masks.append(torch.full((F, H, W), 9, dtype=torch.uint8, device="cuda"))
        torch.cuda.synchronize()
        for i, cam in enumerate(cams):
            scene, H, W, region, block, d, T, N, K, F, form = cam
            ids.append(O.ocq_server_admit(srv, H, W, region, block, d, T, N, K, devs[i][:N].contiguous()))
        order = [(i, t) for t in range(max(c[9] for c in cams)) for i, c in enumerate(cams) if t < c[9]]
        O.ocq_server_submit_arrays(srv, np.array([ids[i] for i, _ in order], dtype=np.int32),
                                   np.array([devs[i][cams[i][7] + t].data_ptr() for i, t in order], dtype=np.uint64),
                                   np.array([masks[i][t].data_ptr() for i, t in order], dtype=np.uint64),
                                   np.array([1000 * i + t for i, t in order], dtype=np.uint64))
        got = []
        deadline = time.monotonic() + 20.0
        while sum(len(g) for g in got) < len(order) and time.monotonic() < deadline:
            got.append(O.ocq_server_poll_array(srv))
            time.sleep(0.002)
        done = np.concatenate(got)
        assert sorted(done["tag"].tolist()) == sorted(1000 * i + t for i, t in order)
        assert (done["done_s"] >= done["arrival_s"]).all()
        for i, cam in enumerate(cams):
            assert (masks[i].cpu().numpy() == _window_oracle(hosts[i], cam)).all(), i
    finally:
        srv.destroy()


def test_block_code_window_many_leaves(cuda_ready):
    """8 x 8 blocks at depth 5 re-merged from their code window when regions
    hold more depth-3 prefixes than the region tables' pool (uniform noise in
    half the frames' pixels, so those regions are recounted by the chunked
    passes), with a ragged bottom row of blocks; masks and the final model
    under the window semantics."""
    import torch

    O = cuda_ready.ocq
    H, W, N, K, T, F = 21, 32, 9, 3, 2, 10
    cam = ("sway", H, W, BLOCK, 8, 5, T, N, K, F, 2)
    g = np.random.default_rng(77)
    host = ocq_synth.fill_host(ocq_synth.make_scene("sway", H, W, N, F, 7900), 0, N + F)
    noise = g.integers(0, 256, size=host.shape, dtype=np.uint8)
    host = np.where((g.random((N + F, H, W)) < 0.5)[..., None], noise, host)
    dev = torch.from_numpy(host).cuda()
    masks = torch.full((F, H, W), 9, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    srv = O.ocq_server_create(1 << 28, 1)
    try:
        c = O.ocq_server_admit(srv, H, W, BLOCK, 8, 5, T, N, K, dev[:N].contiguous())
        assert c is not None
        for t in range(F):
            O.ocq_server_submit(srv, c, dev[N + t], masks[t], tag=t)
        O.ocq_server_sync(srv)
        model = cuda_ready.export_model(O.ocq_server_camera_model(srv, c)).cpu().numpy().view(np.uint64)
        O.ocq_server_release(srv, c)
    finally:
        srv.destroy()
    assert (masks.cpu().numpy() == _window_oracle(host, cam)).all()
    k = F // K
    assert (model == oracle.build_model(host[k * K:k * K + N], 5, T, BLOCK, 8)).all()
