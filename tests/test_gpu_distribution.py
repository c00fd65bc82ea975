"""Frequency distributions f_k(b) of local count tables on the GPU
(pvt_local_distribution) against the oracle's, exactly (integer results)."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
from paper_2001_06784_gb300 import graphgen
from tests import graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pvt():
    import torch  # noqa: F401

    import paper_2001_06784_gb300 as p
    return p


def gpu_dag(pvt, rp, col):
    import torch
    dev = torch.device("cuda:0")
    return pvt.orient(torch.from_numpy(np.ascontiguousarray(rp)).to(dev),
                      torch.from_numpy(np.ascontiguousarray(col, dtype=np.uint32).view(np.int32)).to(dev))


def as_dict(pvt, values, counts):
    vals = pvt.to_ints(values) if len(values) else []
    cnts = counts.cpu().numpy().tolist()
    out = {}
    for v, c in zip(vals, cnts):
        assert v not in out, "a value appears twice"
        out[v] = c
    return out


@pytest.mark.parametrize("make", [lambda: graphgen.workload("er2k_d20_clique30"),
                                  lambda: graphs.disjoint_cliques([1, 2, 5, 33, 70, 130]),
                                  lambda: graphs.gnp(200, 0.2, 5)])
def test_distribution_matches_oracle(pvt, make):
    rp, col = make()
    ref = oracle.count(rp, col, vertex=True, edge=True)
    K = ref["kmax"]
    dag = gpu_dag(pvt, rp, col)
    tv = dag.count_local_vertex(kmax=K)
    te = dag.count_local_edge(kmax=K)
    for k in range(K + 1):
        assert as_dict(pvt, *pvt.local_distribution(tv, k)) == oracle.frequency(ref["cv"], k), k
        assert as_dict(pvt, *pvt.local_distribution(te, k)) == oracle.frequency(ref["ce"], k), k
    dag.free()


def test_distribution_full_size_moments(pvt):
    """Per-vertex table of the 500k-vertex graph at the paper's k = 5, 10,
    15, 20, 25: f_k sums to n and its first moment is k * C_k (C_k from the
    root-parallel oracle)."""
    rp, col = graphgen.workload("cl500k_m8m_b2.3_clq200")
    n = len(rp) - 1
    ref = oracle.count(rp, col, threads=os.cpu_count() or 1)
    dag = gpu_dag(pvt, rp, col)
    K = max(k for k, c in enumerate(ref["C"]) if c)
    tv = dag.count_local_vertex(kmax=K)
    for k in (5, 10, 15, 20, 25):
        f = as_dict(pvt, *pvt.local_distribution(tv, k))
        assert sum(f.values()) == n
        assert sum(b * c for b, c in f.items()) == k * ref["C"][k]
    dag.free()


def test_distribution_edge_cases(pvt):
    import torch
    dev = torch.device("cuda:0")
    empty = torch.zeros((0, 3, 1), dtype=torch.int64, device=dev)
    v, c = pvt.local_distribution(empty, 1)
    assert len(v) == 0 and len(c) == 0
    t = torch.zeros((1000, 4, 2), dtype=torch.int64, device=dev)
    t[::3, 2, 1] = 7  # value 7 * 2^64 on every third row
    f = as_dict(pvt, *pvt.local_distribution(t, 2))
    assert f == {0: 1000 - 334, 7 << 64: 334}
    with pytest.raises(pvt.PivoterError):
        pvt.local_distribution(t, 4)
    with pytest.raises(pvt.PivoterError):
        pvt.local_distribution(t, -1)
