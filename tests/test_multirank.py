"""The benchmark's multi-rank host logic on CPU with gloo, world size 2:
barrier, max over ranks of the per-rank time, and the whole-job aggregate of
independent replicas (weak scaling)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, _, w = bench.dist_env()
    assert (r, w) == (rank, world)
    bench.barrier(world)
    mx = bench.max_over_ranks(100.0 + 50.0 * rank, world)
    val = bench.aggregate_value(17.18e9, mx, world)
    out[rank] = (mx, val)
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 150.0  # the slowest rank's time
    # two replicas of 17.18 GB each in 150 ms
    assert out[0][1] == pytest.approx(2 * 17.18e9 / 0.150 / 1e9)
