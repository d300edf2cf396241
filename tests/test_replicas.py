"""The N > 1 benchmark path on CPU: world_size-2 gloo ranks run the host
logic bench.py uses for replicas (seed per rank, max-over-ranks timing,
whole-job throughput).  No GPU is involved."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # a different step time on every rank; every rank must see the slowest
    t = bench.max_over_ranks(0.1 * (rank + 1), dist, "cpu")
    import graphgen as gg

    g = gg.rmat(8, 8, seed=bench.replica_seed(rank))
    out[rank] = (t, bench.replica_seed(rank), g.m, bench.replica_throughput(world, g.m, t))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_host_logic(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict(out)
    assert sorted(res) == list(range(world))
    slow = 0.1 * world
    for r, (t, seed, m, thr) in res.items():
        assert abs(t - slow) < 1e-12            # max over ranks
        assert seed == 1 + r                     # independent replicas
        assert abs(thr - world * m / slow) < 1e-6
    # the replicas are different graphs
    assert res[0][2] != res[1][2] or res[0][1] != res[1][1]
