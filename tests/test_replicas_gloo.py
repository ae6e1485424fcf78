"""The multi-process path of bench.py on CPU: two gloo ranks reduce their timings with
the same helpers the GPU run uses (max over ranks, whole-job rate of replicas)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(10.0 + rank, dist, device="cpu")   # rank r took 10 + r ms
    out[rank] = (t, bench.job_rate(32, world, t / 1e3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = torch.multiprocessing.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        for r in range(world):
            t, rate = out[r]
            assert t == 11.0                         # the slowest rank's time on every rank
            assert rate == pytest.approx(2 * 32 / 0.011)   # units of both ranks / that time


def test_one_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(10, 1, 2.0) == 5.0
