"""The serving harness of bench.py on a fake server (CPU only): every frame of
every admitted camera is submitted exactly once, in arrival order per camera,
with its own frame and mask buffers; tags come back to the right camera and
frame, a camera is released after its last frame, and no latency (completion
minus scheduled arrival) is negative."""
import time

import numpy as np
import torch

import bench
from ocq_synth.configs import ServeStream, Workload


class _FakeServer:
    def __init__(self):
        self.cams, self.pending, self.log, self.released = {}, [], [], []

    def destroy(self):
        pass


class _FakeO:
    """The ocq_server_* calls _serve_run makes; a submitted frame completes
    at its next poll."""

    def ocq_server_create(self, budget, n):
        self.srv = _FakeServer()
        return self.srv

    def ocq_server_set_batching(self, srv, delay, tif):
        assert delay >= 0 and tif >= 0

    def ocq_server_usage(self, srv):
        return (0, 1 << 40, 0)

    def ocq_server_admit(self, srv, H, W, region, block, depth, T, N, K, train):
        cam = len(srv.cams)
        srv.cams[cam] = (H, W)
        return cam

    def ocq_server_submit_arrays(self, srv, cams, frames, masks, tags):
        now = time.monotonic()
        for c, f, m, t in zip(cams.tolist(), frames.tolist(), masks.tolist(), tags.tolist()):
            srv.log.append((c, int(t), now, f, m))
            srv.pending.append((c, int(t), now))

    def ocq_server_poll_array(self, srv, max_n=65536):
        dt = np.dtype([("camera", np.int32), ("reserved", np.int32), ("frame", np.int64), ("tag", np.uint64),
                       ("arrival_s", np.float64), ("done_s", np.float64)])
        out = np.zeros(len(srv.pending), dtype=dt)
        now = time.monotonic()
        for k, (c, t, a) in enumerate(srv.pending):
            out[k]["camera"], out[k]["tag"], out[k]["arrival_s"], out[k]["done_s"] = c, t, a, now
        srv.pending = []
        return out

    def ocq_server_release(self, srv, cam):
        srv.released.append(cam)

    def ocq_server_sync(self, srv):
        pass


def test_serve_run_submits_every_frame_once_in_order():
    rng = np.random.default_rng(3)
    streams, bufs, fps = [], [], []
    n_cam, fpc, pool, slots = 5, 7, 4, 8
    for i in range(n_cam):
        wl = Workload(f"cam{i}", "sway", 4, 8, 3, fpc, 2, 0, 3, 1, 0, i)
        join = 0.002 * i
        arr = list(join + np.cumsum(rng.exponential(0.001, fpc)))
        streams.append(ServeStream(wl, join, 30.0, fpc, arr))
        bufs.append((torch.zeros((wl.N + pool, 4, 8, 3), dtype=torch.uint8),
                     torch.zeros((slots, 4, 8), dtype=torch.uint8)))
        fps.append(1000)
    O = _FakeO()
    r = bench._serve_run(O, streams, bufs, fps, 1 << 30, n_cam, fpc, pool, slots, 1.0, 10.0)
    srv = O.srv
    assert r["frames_done"] == n_cam * fpc and r["done_cams"] == n_cam
    assert sorted(srv.released) == list(range(n_cam))
    per_cam = {}
    for c, tag, _, f, m in srv.log:
        i, t = divmod(tag, 100000)
        assert c == i  # cameras are admitted in join order here, so ids match stream indices
        per_cam.setdefault(i, []).append(t)
        assert f == bufs[i][0][streams[i].wl.N + t % pool].data_ptr()
        assert m == bufs[i][1][t % slots].data_ptr()
    for i in range(n_cam):
        assert per_cam[i] == list(range(fpc)), i
    assert r["lat_ms"].size == n_cam * fpc and (r["lat_ms"] >= 0).all()
    assert r["px_done"] == n_cam * fpc * 4 * 8
