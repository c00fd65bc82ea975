"""The query server (continuous batching): every result equals the same
query run alone and the single-graph entry points, word for word
(integer results: tolerance 0), for global, per-vertex and per-edge
queries on graphs of mixed sizes submitted together."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2001_06784_gb300 import graphgen
from tests import graphs

pytestmark = pytest.mark.gpu


def mixed_graphs():
    out = []
    rng = np.random.default_rng(5)
    for i in range(24):
        n = int(np.exp(rng.uniform(np.log(100), np.log(5000))))
        deg = float(rng.uniform(5, 40))
        if i % 2:
            rp, col = graphgen.generate(n, er_avg_deg=deg, planted=[(2, 6, 18, 0.9)], seed=100 + i)
        else:
            m = max(int(n * deg / 2), 1)
            rp, col = graphgen.generate(n, chung_lu=(min(m, n * (n - 1) // 4), float(rng.uniform(2.0, 2.5))),
                                        planted=[(1, 8, 20, 1.0)], seed=100 + i)
        out.append((rp, col, ("global", "edge", "vertex")[i % 3]))
    out.append((graphs.complete(40)[0], graphs.complete(40)[1], "global"))
    out.append(graphgen.from_edges(7, np.zeros((0, 2), dtype=np.int64)) + ("edge",))
    return out


@pytest.mark.parametrize("direct_edges", [-1, 3000, 0])
def test_server_mix_equals_alone_and_oracle(direct_edges):
    """direct_edges: -1 batches every query; 3000 sends most of them down the
    whole-GPU direct path beside the batches; 0 is the default threshold."""
    import paper_2001_06784_gb300 as pvt
    qs = mixed_graphs()
    with pvt.Server(mem_budget=4 << 30, max_batch=16, streams=3, direct_edges=direct_edges) as sv:
        # all at once (they batch and overlap)
        tickets = [sv.submit(rp, col, kind) for rp, col, kind in qs]
        mixed = [sv.result(t)[0] for t in tickets if sv.wait(t, 60000)]
        assert len(mixed) == len(qs)
        # one at a time
        alone = []
        for rp, col, kind in qs:
            t = sv.submit(rp, col, kind)
            assert sv.wait(t, 60000)
            alone.append(sv.result(t)[0])
    for (rp, col, kind), a, b in zip(qs, mixed, alone):
        assert a.shape == b.shape and (a == b).all(), "result differs alone and in the mix"
        K = a.shape[1] - 1
        ref = oracle.count(rp, col, kmax=K, vertex=kind == "vertex", edge=kind == "edge")
        if kind == "global":
            assert pvt.to_ints(a[0]) == ref["C"]
        elif kind == "vertex":
            assert pvt.to_ints(a) == oracle.to_int(ref["cv"])
        else:
            assert pvt.to_ints(a) == oracle.to_int(ref["ce"])


def test_server_kmax_and_errors():
    import paper_2001_06784_gb300 as pvt
    rp, col = graphgen.generate(800, er_avg_deg=10.0, planted=[(2, 10, 16, 1.0)], seed=3)
    ref = oracle.count(rp, col, kmax=4, edge=True)
    with pvt.Server(mem_budget=1 << 30) as sv:
        t1 = sv.submit(rp, col, "global", kmax=4)
        t2 = sv.submit(rp, col, "edge", kmax=4)
        assert sv.wait(t1, 60000) and sv.wait(t2, 60000)
        assert pvt.to_ints(sv.result(t1)[0][0]) == ref["C"]
        assert pvt.to_ints(sv.result(t2)[0]) == oracle.to_int(ref["ce"])
        with pytest.raises(pvt.PivoterError):
            sv.submit(rp[:-1], col, "global")
    with pvt.Server(mem_budget=1 << 20) as small:
        with pytest.raises(pvt.PivoterError) as ei:
            small.submit(rp, col, "edge")
        assert ei.value.status == 3
