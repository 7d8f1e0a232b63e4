"""The N > 1 path of bench.py on CPU: two gloo ranks, max-over-ranks timing and the whole-job
rate (each rank runs an independent replica of the workload; no data-path collective)."""
import os
import sys

import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    m = bench.max_over_ranks(ms)
    rate = bench.whole_job_rate(1000.0, world, m / 1e3)
    tdist.barrier()
    out[rank] = (m, rate)
    tdist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = 29500 + (os.getpid() % 2000)
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        m, rate = out[r]
        assert m == 15.0
        assert rate == pytest.approx(world * 1000.0 / 0.015)


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert not (tdist.is_available() and tdist.is_initialized())
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
