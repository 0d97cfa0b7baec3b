"""The replica path of bench.py (one process per GPU, no data-path
collective) on two CPU ranks over gloo: the timing barrier, the
max-over-ranks duration and the whole-job rate."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        local = 100.0 + 50.0 * rank  # rank 1 is the slow replica
        ms = bench.max_over_ranks(local, world, device="cpu")
        out[rank] = (ms, bench.job_rate(world, 10, ms))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_duration():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    port, world = _free_port(), 2
    with mp.Manager() as man:
        out = man.dict()
        procs = [mp.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        ms, rate = res[r]
        assert ms == 150.0  # every rank reports the slowest replica
        assert rate == pytest.approx(2 * 10 / 0.150)  # steps of all replicas over the job's duration


def test_one_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    bench.barrier(1)
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.job_rate(1, 5, 500.0) == pytest.approx(10.0)
