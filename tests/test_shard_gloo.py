"""Sharding the count by root ranges (roots are independent subproblems,
Sec. 4 "Parallel version"; the (h, p) path histogram is the whole state of a
count, proof of Thm. main): two gloo ranks on the CPU each take half of the
roots, the oracle gives each rank the histogram of its roots, one sum
all-reduce joins them, and C_k = sum over (h, p) of hist[h][p] * C(p, k - h)
equals the one-process count.  This is the host side of sharding the device
histograms (pvt_count_hist on one GPU per rank, then pvt_combine_hist)."""
from __future__ import annotations

import math
import os
import socket

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _graph():
    from paper_2001_06784_gb300 import graphgen
    return graphgen.generate(600, er_avg_deg=10.0, planted=[(3, 12, 30, 0.9)], seed=17)


def _rank(rank, world, port, H, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    rp, col = _graph()
    n = len(rp) - 1
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = np.arange(rank * n // world, (rank + 1) * n // world, dtype=np.uint32)
        hist = oracle.count(rp, col, roots=mine, hist_dim=H)["hist"].astype(np.int64)
        t = torch.from_numpy(hist)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        out.put((rank, t.numpy().copy()))
    finally:
        dist.destroy_process_group()


def test_root_range_shards_add_up_two_ranks():
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    rp, col = _graph()
    whole = oracle.count(rp, col)
    H = whole["alpha"] + 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, H, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, a), (_, b) = got
    assert (a == b).all()  # every rank holds the sum
    hist = a
    assert hist[1].sum() == len(rp) - 1  # one all-pivot path per root
    C = [0] + [sum(int(hist[h][p]) * math.comb(p, k - h) for h in range(1, k + 1) for p in range(H) if k - h <= p)
               for k in range(1, whole["kmax"] + 1)]
    assert C == whole["C"]
