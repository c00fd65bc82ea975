"""The replica path of bench.py (N ranks, one graph each, no data-path
collective): every rank learns the slowest rank's time, and the whole-job
rate counts the units of all ranks.  Two gloo ranks on the CPU."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], "cpu")
        out.put((rank, t, bench.whole_job_rate(1000.0, world, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [1.5, 2.25]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [2.25, 2.25]
    assert all(g[2] == pytest.approx(2 * 1000.0 / 2.25) for g in got)


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, "cpu") == 3.0
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
