"""Whole-frame regions split by pixels across ranks: the row bands, the
exchange of the bands' per-frame leaf sets between gloo ranks on CPU, and (on
a GPU) the union-and-count merge of those leaf sets in the CUDA library, all
against the oracle's model of the unsplit frames (Alg. 1 and 2)."""
import os
import socket

import numpy as np
import pytest

import ocq_synth
import oracle

FRAME = 0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_frame_bands_partition_the_rows():
    from paper_1412_1945_gb300 import shard

    for H in (1, 2, 7, 120, 1080):
        for world in (1, 2, 3, 4, 8):
            bands = [shard.frame_band(H, r, world) for r in range(world)]
            assert bands[0][0] == 0 and bands[-1][1] == H
            assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
            sizes = [y1 - y0 for y0, y1 in bands]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0
    with pytest.raises(ValueError):
        shard.frame_band(10, 2, 2)


def _band_leaf_sets(frames, depth):
    """Test-only restatement of S2 for one band: per frame, the bitset of the
    path codes (oracle) its pixels reach, exported layout [N, 1, words]."""
    N = frames.shape[0]
    words = max(1, 8 ** depth // 64)
    out = np.zeros((N, 1, words), dtype=np.uint64)
    for f in range(N):
        if frames[f].size == 0:
            continue
        for c in np.unique(oracle.leaf_codes(frames[f].reshape(-1, 3), depth)):
            out[f, 0, c // 64] |= np.uint64(1) << np.uint64(c % 64)
    return out.view(np.int64)


def _rank_main(rank, world, port, out, cfg):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    from paper_1412_1945_gb300 import shard

    scene, H, W, N, depth, seed = cfg
    dist.init_process_group("gloo", rank=rank, world_size=world)
    frames = ocq_synth.fill_host(ocq_synth.make_scene(scene, H, W, N, 0, seed), 0, N)
    y0, y1 = shard.frame_band(H, rank, world)
    local = torch.from_numpy(_band_leaf_sets(np.ascontiguousarray(frames[:, y0:y1]), depth))
    parts = shard.gather_parts(local)
    out.put((rank, parts.numpy().copy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_band_leaf_sets(world):
    """Each rank gathers every rank's band leaf sets, rank-major; their union
    per frame counted over frames and thresholded is the oracle's model of
    the whole frames, at every T."""
    import torch.multiprocessing as mp

    cfg = ("clusters", 37, 48, 9, 4, 77 + world)
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out, cfg)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((out.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    scene, H, W, N, depth, seed = cfg
    frames = ocq_synth.fill_host(ocq_synth.make_scene(scene, H, W, N, 0, seed), 0, N)
    for rank, parts in res:
        assert parts.shape == (world, N, 1, max(1, 8 ** depth // 64))
        assert (parts == res[0][1]).all()  # every rank holds the same parts
    from paper_1412_1945_gb300 import shard

    for r in range(world):  # part r is rank r's band
        y0, y1 = shard.frame_band(H, r, world)
        assert (res[0][1][r] == _band_leaf_sets(np.ascontiguousarray(frames[:, y0:y1]), depth)).all()
    union = np.bitwise_or.reduce(res[0][1].view(np.uint64), axis=0)  # [N, 1, words]
    bits = np.unpackbits(union.view(np.uint8), bitorder="little").reshape(N, -1)
    counts = bits.sum(axis=0)
    for T in range(1, N + 1):
        model = np.packbits(counts >= T, bitorder="little").view(np.uint64).reshape(1, -1)
        assert (model == oracle.build_model(frames, depth, T, FRAME)).all(), T


@pytest.mark.gpu
@pytest.mark.parametrize("parts", [1, 2, 3, 5])
@pytest.mark.parametrize("depth", [2, 4, 5])
def test_merge_of_band_leaf_sets_on_the_gpu(cuda_ready, parts, depth):
    """The CUDA calls a rank makes: its band's leaf sets (ocq_occupancy), then
    the union-and-count merge of every band's (ocq_merge_occupancy); the model
    equals the oracle's on the whole frames, and so do the test frames'
    masks classified with it."""
    import torch

    from paper_1412_1945_gb300 import shard

    O = cuda_ready.ocq
    H, W, N, F, T = 41, 56, 11, 3, 3
    sc = ocq_synth.make_scene("sway", H, W, N, F, 900 + 10 * parts + depth)
    host = ocq_synth.fill_host(sc, 0, N + F)
    dev = torch.from_numpy(host).cuda()
    words = max(1, 8 ** depth // 64)
    occ = torch.empty((parts, N, 1, words), dtype=torch.int64, device="cuda")
    for r in range(parts):
        y0, y1 = shard.frame_band(H, r, parts)
        O.ocq_occupancy(dev[:N, y0:y1].contiguous(), N, y1 - y0, W, FRAME, 0, depth, occ[r])
    m = O.ocq_merge_occupancy(occ, parts, N, H, W, FRAME, 0, depth, T)
    got = cuda_ready.export_model(m).cpu().numpy().view(np.uint64)
    ow, om = oracle.run(host[:N], depth, T, FRAME, 0, host[N:])
    assert (got == ow).all()
    mask = torch.empty((F, H, W), dtype=torch.uint8, device="cuda")
    O.ocq_classify(m, dev[N:], F, mask)
    cuda_ready.device_status()
    assert (mask.cpu().numpy() == om).all()
    m.free()
