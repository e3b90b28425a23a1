"""ocq_build_frame_noalloc: the whole-frame build for callers that cannot
allocate device memory at call time (pipelines that reserve every buffer up
front and must not block on the allocator).  It must give exactly the model
the allocating entry point gives (the library's tolerance for this integer
method is zero), call after call, with its shared static scratch, and that
model must be the oracle's (Alg. 1 and 2 on pointer octrees).

This file is named to be collected last."""
import numpy as np
import pytest

import ocq_synth
import oracle
from ocq_synth import configs

pytestmark = pytest.mark.gpu


def _expected(ocq, frames, depth, T):
    m = ocq.build_model(frames, depth, T, "frame")
    words = ocq.export_model(m).cpu().numpy().view(np.uint64).ravel()
    m.free()
    return words


@pytest.mark.parametrize("depth,T,N,H,W,seed", [(4, 4, 8, 120, 160, 0), (6, 7, 20, 37, 53, 1), (8, 2, 5, 19, 23, 2)])
def test_noalloc_matches_allocating_build(cuda_ready, depth, T, N, H, W, seed):
    import torch

    ocq = cuda_ready
    if seed == 0:
        wl = configs.TINY_FRAME
        sc = ocq_synth.make_scene(wl.scene_kind, wl.H, wl.W, wl.N, wl.F, wl.seed)
    else:
        sc = ocq_synth.make_scene("sway", H, W, N, 0, seed)
    host = ocq_synth.fill_host(sc, 0, N)
    frames = torch.from_numpy(host).cuda()
    expect = _expected(ocq, frames, depth, T)
    assert (expect == oracle.build_model(host, depth, T, oracle.REGION_FRAME).ravel()).all()
    wpr = 1 if depth <= 2 else 1 << (3 * depth - 6)
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        out = torch.full((wpr,), -1, dtype=torch.int64, device="cuda")
        ocq.ocq.ocq_build_frame_noalloc(frames, N, H, W, depth, T, out)
        ocq.device_status()
        got = out.cpu().numpy().view(np.uint64)
        assert (got == expect).all()


def test_noalloc_rejects_oversized_requests(cuda_ready):
    import torch

    ocq = cuda_ready
    frames = torch.zeros((1, 2, 2, 3), dtype=torch.uint8, device="cuda")
    out = torch.zeros(1 << 18, dtype=torch.int64, device="cuda")
    # depth 8 needs 2 MiB per scratch row; N = 65535 needs 16 planes + 2 rows.
    # The library refuses the size before it reads any frame, so the raw
    # address goes past the binding's buffer checks to the C entry point.
    with pytest.raises(ocq.OcqError) as e:
        ocq.ocq.ocq_build_frame_noalloc(frames.data_ptr(), 65535, 2, 2, 8, 1, out)
    assert e.value.status == ocq.ocq.OCQ_EINVAL and "maximum" in str(e.value)


def test_noalloc_wrapper_checks_buffer_sizes(cuda_ready):
    import torch

    ocq = cuda_ready
    frames = torch.zeros((2, 4, 4, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):  # model shorter than 8^4/64 words
        ocq.ocq.ocq_build_frame_noalloc(frames, 2, 4, 4, 4, 1, torch.zeros(63, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):  # frames shorter than N*H*W*3 bytes
        ocq.ocq.ocq_build_frame_noalloc(frames, 3, 4, 4, 4, 1, torch.zeros(64, dtype=torch.int64, device="cuda"))
