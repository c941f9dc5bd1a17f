"""Host logic of the multi-rank bench (replicas, weak scaling) on two gloo
ranks on the CPU: the job's time is the maximum over ranks and the rate
counts every rank's units."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        total = bench.job_ms(ms, dist, "cpu")
        out[rank] = (total, bench.job_throughput(1000, world, total))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_job_time_and_rate():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    total, rate = res[0]
    assert total == 15.0
    assert rate == pytest.approx(1000 * 2 / 15e-3)


def test_single_rank_is_local():
    import bench
    assert bench.job_ms(12.5) == 12.5
    assert bench.job_throughput(500, 1, 2.0) == pytest.approx(250000.0)
