"""The multi-rank path of bench.py on CPU: two gloo ranks, each a replica solving
its own independent queries (weak scaling, no data-path collective). The job's
time is the slowest rank's (a max over ranks) and its rate counts every rank's
units. The GPU runs use the same helpers with NCCL."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, seconds, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(seconds[rank], "cpu")
        dist.barrier()
        out[rank] = (t, bench.whole_job_rate(10, world, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    seconds = [0.5, 0.8]  # rank 1 is slower
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), seconds, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, rate = res[r]
        assert t == pytest.approx(0.8)
        assert rate == pytest.approx(2 * 10 / 0.8)


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.25, "cpu") == 1.25
    assert bench.whole_job_rate(7, 1, 0.5) == pytest.approx(14.0)


def _replica_rank(rank, world, port, out):
    import time

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        calls = {"step": 0, "before": 0}
        delay = 0.01 * (rank + 1)  # rank 1 solves twice as slowly

        def step():  # stub solve: each rank works on its own queries, no collective
            calls["step"] += 1
            time.sleep(delay)

        def before():
            calls["before"] += 1

        def timer(fn):
            t0 = time.perf_counter()
            fn()
            return 1e3 * (time.perf_counter() - t0)

        ms, total_s, rate = bench.replica_steps(step, 5, world, "cpu", timer, before_step=before)
        out[rank] = (ms, total_s, rate, dict(calls))
    finally:
        dist.destroy_process_group()


def test_replica_steps_under_two_gloo_ranks():
    # the per-rank timed loop of the benchmark, driven with a stub solve: each rank
    # times its own steps, the job takes the slowest rank's total, and the rate
    # counts the steps of both ranks
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_replica_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    slow = sum(res[1][0]) / 1e3
    for r in range(world):
        ms, total_s, rate, calls = res[r]
        assert len(ms) == 5 and calls == {"step": 5, "before": 5}
        assert total_s == pytest.approx(slow)
        assert rate == pytest.approx(2 * 5 / slow)
    assert sum(res[0][0]) < sum(res[1][0])
    assert slow >= 5 * 0.02
