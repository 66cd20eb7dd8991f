"""bench.py's multi-rank plumbing on CPU: two gloo ranks, whole-job rate = units summed over ranks / slowest rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    d = bench.Dist()
    d.init("gloo")
    units, secs = bench.aggregate(1000.0 * (rank + 1), 2.0 + rank, d)
    d.barrier()
    d.close()
    out[rank] = (units, secs)


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (3000.0, 3.0)


def test_reference_arm_defers_to_rank_zero(monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    d = bench.Dist()

    class Args:
        workload = "rmat20"
        steps = 1
        warmup = 0
    assert bench.run_reference(Args, d) is None  # only rank 0 runs and prints the oracle arm
