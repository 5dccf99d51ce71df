"""The N > 1 benchmark path on CPU: two gloo ranks run independent replicas and the
job time is the slowest rank's (the only collective is that max reduction)."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 1000.0 * (rank + 1)        # rank 1 is the slower replica
    ms, value = bench.aggregate(local_ms, world, 18, dist, "cpu")
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, value in out:
        assert ms == 2000.0                       # max over ranks
        assert value == pytest.approx(2 * 18 / 2.0)   # N x solves / slowest time


def test_single_rank_needs_no_collective():
    import bench
    ms, value = bench.aggregate(500.0, 1, 18)
    assert ms == 500.0 and value == pytest.approx(36.0)
