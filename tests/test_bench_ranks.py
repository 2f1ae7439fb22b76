"""Host logic of the replicated multi-GPU bench: two gloo ranks on the CPU.

Each rank solves its own seeded problem (the path has no exchange step), so
the job rate is the units of all ranks over the slowest rank's time.
"""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_local = [400.0, 1000.0][rank]            # rank 1 is the slowest
        rate, ms = bench.job_rate(ms_local, 50 * 3, dist, "cpu")
        out[rank] = (rate, ms)
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        rate, ms = out[r]
        assert ms == 1000.0
        assert rate == pytest.approx(2 * 150 / 1.0)


def test_job_rate_single_process():
    import bench
    rate, ms = bench.job_rate(250.0, 10)
    assert ms == 250.0 and rate == pytest.approx(40.0)
