"""The benchmark's multi-rank bookkeeping with the gloo backend on the CPU:
two ranks, the slowest rank's time decides, the rate counts every rank's work."""
import os
import socket

import pytest

import bench

torch = pytest.importorskip("torch")


def free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    dist.barrier()
    total = bench.max_over_ranks(times[rank])
    out.put((rank, total, bench.whole_job_rate(16, 10, world, total)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_and_rate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    times = [123.0, 456.0]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, rate in got:
        assert total == 456.0
        assert rate == pytest.approx(2 * 16 * 10 / 0.456)


def test_single_process_is_identity():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(16, 10, 1, 1000.0) == pytest.approx(160.0)
