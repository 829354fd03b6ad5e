"""The benchmark's whole-job rate over ranks, on CPU with two gloo ranks:
units processed by all ranks over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms_local = [10.0, 25.0][rank]          # rank 1 is the slow one
        rate, ms = bench.job_rate(1000.0, ms_local, world, dist, "cpu")
        dist.barrier()
        results[rank] = (rate, ms)
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_and_sums_units():
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), results), nprocs=world, join=True)
        got = dict(results)
    for r in range(world):
        rate, ms = got[r]
        assert ms == 25.0
        assert rate == pytest.approx(2 * 1000.0 / 0.025)


def test_job_rate_single_rank():
    import bench
    rate, ms = bench.job_rate(500.0, 20.0, 1)
    assert (rate, ms) == (pytest.approx(25000.0), 20.0)
