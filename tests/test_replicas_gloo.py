"""The multi-process path of bench.py on CPU (gloo, world size 2).

A single matrix's factorization does not shard as one step, so bench.py runs
replicas: every rank factors its own copy and the job's rate is world x flops
x steps over the slowest rank's time. These tests check that aggregation with
two real gloo ranks on 127.0.0.1 (no GPU).
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) x the base time for the factor, solve and step
        mine = [10.0 * (rank + 1), 2.0 * (rank + 1), 12.0 * (rank + 1)]
        got = bench.reduce_max_over_ranks(dist, mine, "cpu")
        dist.barrier()
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == [20.0, 4.0, 24.0]


def test_whole_job_rate_counts_every_replica():
    # 2 replicas x 7.06e10 flops x 5 steps in 400 ms (the slowest rank) -> GFLOP/s
    assert bench.whole_job_rate(2, 7.06e10, 5, 400.0) == pytest.approx(2 * 7.06e10 * 5 / 0.4 / 1e9)
    assert bench.reduce_max_over_ranks(None, [1.0, 2.0], "cpu") == [1.0, 2.0]
