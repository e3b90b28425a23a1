"""Error paths, exercised without faulting a GPU: allocation failures injected
on the host (OCQ_ENOMEM, nothing leaked), a bounded device wait made to run out
(OCQ_ETIMEOUT, the context stays usable), a camera released mid-window."""
import numpy as np
import pytest

import ocq_synth
import oracle

pytestmark = pytest.mark.gpu
FRAME, BLOCK, PIXEL = 0, 1, 2
ENOMEM, ETIMEOUT = 2, 4


@pytest.fixture(scope="module")
def ocq(cuda_ready):
    return cuda_ready


@pytest.fixture(scope="module")
def torch():
    import torch

    return torch


def _frames(torch, scene, H, W, N, F, seed):
    sc = ocq_synth.make_scene(scene, H, W, N, F, seed=seed)
    host = ocq_synth.fill_host(sc, 0, N + F)
    return host, torch.from_numpy(host).cuda()


@pytest.mark.parametrize("kind,block,d", [(FRAME, 0, 4), (FRAME, 0, 7), (BLOCK, 4, 6), (PIXEL, 0, 4)])
def test_injected_allocation_failures_leave_nothing_behind(ocq, torch, kind, block, d):
    O = ocq.ocq
    host, dev = _frames(torch, "clusters", 24, 32, 6, 0, 5 + d)
    torch.cuda.synchronize()
    before = O.ocq_debug_async_bytes_in_use()
    try:
        for k in (1, 2):
            O.ocq_debug_fail_allocations(k)
            try:
                m = ocq.build_model(dev, d, 3, kind, block)
            except ocq.OcqError as e:
                assert e.status == ENOMEM
            else:  # fewer than k allocations on this path: it must have succeeded
                m.free()
            O.ocq_debug_fail_allocations(0)
            torch.cuda.synchronize()
            assert O.ocq_debug_async_bytes_in_use() == before, k
    finally:
        O.ocq_debug_fail_allocations(0)
    m = ocq.build_model(dev, d, 3, kind, block)
    words = ocq.export_model(m).cpu().numpy().view(np.uint64)
    m.free()
    assert (words == oracle.build_model(host, d, 3, kind, block)).all()


def test_server_admission_allocation_failure(ocq, torch):
    O = ocq.ocq
    host, dev = _frames(torch, "sway", 16, 24, 5, 4, 9)
    torch.cuda.synchronize()
    srv = O.ocq_server_create(1 << 30, 4)
    try:
        O.ocq_debug_fail_allocations(1)
        with pytest.raises(ocq.OcqError) as err:
            O.ocq_server_admit(srv, 16, 24, PIXEL, 0, 3, 2, 5, 5, dev[:5])
        assert err.value.status == ENOMEM
        O.ocq_debug_fail_allocations(0)
        assert O.ocq_server_usage(srv)[0] == 0
        cam = O.ocq_server_admit(srv, 16, 24, PIXEL, 0, 3, 2, 5, 5, dev[:5])
        assert cam is not None
        O.ocq_server_release(srv, cam)
    finally:
        O.ocq_debug_fail_allocations(0)
        srv.destroy()


def test_batch_wait_times_out_and_context_survives(ocq, torch):
    """Stream 0's build items are left out of the persistent work list: its
    classify items give up after the bounded wait, the status is
    OCQ_ETIMEOUT, and the next run (builds restored) is correct."""
    O = ocq.ocq
    descs = []
    for i, (H, W, kind, block, d) in enumerate([(40, 64, PIXEL, 0, 3), (48, 48, BLOCK, 8, 4)]):
        host, dev = _frames(torch, "clusters", H, W, 8, 5, 30 + i)
        descs.append(dict(train=dev[:8].contiguous(), test=dev[8:].contiguous(),
                          mask=torch.full((5, H, W), 7, dtype=torch.uint8, device="cuda"),
                          N=8, H=H, W=W, kind=kind, block=block, depth=d, T=3, F=5,
                          host_train=host[:8], host_test=host[8:]))
    torch.cuda.synchronize()
    b = O.ocq_batch_create(descs)
    try:
        O.ocq_batch_set_mode(b, 0)
        O.ocq_batch_debug_hold_builds(b, 0)
        O.ocq_batch_run(b)
        with pytest.raises(ocq.OcqError) as err:
            O.ocq_batch_status(b)
        assert err.value.status == ETIMEOUT
        O.ocq_batch_debug_hold_builds(b, -1)
        for s in descs:
            s["mask"].fill_(7)
        O.ocq_batch_run(b)
        O.ocq_batch_status(b)
        for s in descs:
            _, om = oracle.run(s["host_train"], s["depth"], s["T"], s["kind"], s["block"], s["host_test"])
            assert (s["mask"].cpu().numpy() == om).all()
    finally:
        b.destroy()


def test_server_release_mid_window(ocq, torch):
    """Camera A is released with frames (and a re-merge) still in flight;
    camera B, served alongside, is unaffected."""
    O = ocq.ocq
    N, K, F, T, d = 6, 3, 9, 2, 3
    host_a, dev_a = _frames(torch, "sway", 24, 32, N, F, 50)
    host_b, dev_b = _frames(torch, "clusters", 20, 36, N, F, 51)
    masks_b = torch.full((F, 20, 36), 7, dtype=torch.uint8, device="cuda")
    masks_a = torch.full((F, 24, 32), 7, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    srv = O.ocq_server_create(1 << 30, 4)
    try:
        a = O.ocq_server_admit(srv, 24, 32, PIXEL, 0, d, T, N, K, dev_a[:N])
        b = O.ocq_server_admit(srv, 20, 36, BLOCK, 4, d, T, N, K, dev_b[:N])
        for t in range(F):
            if t < 5:
                O.ocq_server_submit(srv, a, dev_a[N + t], masks_a[t], tag=t)
            O.ocq_server_submit(srv, b, dev_b[N + t], masks_b[t], tag=100 + t)
            if t == 4:
                O.ocq_server_release(srv, a)  # frames 3-4 and the re-merge after frame 5's window
        O.ocq_server_sync(srv)
        assert O.ocq_server_usage(srv)[0] == O.ocq_server_camera_footprint(20, 36, BLOCK, 4, d, T, N, K)
        O.ocq_server_release(srv, b)
        assert O.ocq_server_usage(srv)[0] == 0
    finally:
        srv.destroy()
    for t in range(F):
        k = t // K
        model = oracle.build_model(host_b[k * K:k * K + N], d, T, BLOCK, 4)
        expect = oracle.classify(model, host_b[N + t:N + t + 1], d, BLOCK, 4)[0]
        assert (masks_b[t].cpu().numpy() == expect).all(), t
