"""Host logic of the N>1 bench path on CPU: world_size-2 gloo ranks.

Each rank runs its own camera stream (weak scaling, no data-path collective);
the job's throughput is all ranks' units over the slowest rank's time, taken
with one max-reduction after a barrier."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    r, w, local = bench.dist_env()
    d = bench.Dist(w, "gloo")
    d.barrier()
    # rank r "took" 10 + 5r ms for its step; each processed 1000 units
    t_max = d.max(10.0 + 5.0 * r, "cpu")
    units = d.gather_sum(1000.0, "cpu")
    value, slowest = bench.aggregate([10.0 + 5.0 * k for k in range(w)], [1000.0] * w)
    out.put((r, bench.shard_stream_id(r, w), t_max, units, value, slowest))
    d.close()


def test_two_rank_gloo_aggregation():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [0, 1]            # distinct camera streams per rank
    assert all(r[2] == pytest.approx(15.0) for r in res)   # max over ranks
    assert all(r[3] == pytest.approx(2000.0) for r in res)
    assert res[0][4] == pytest.approx(2000.0 / 0.015)      # units of all ranks / slowest time
