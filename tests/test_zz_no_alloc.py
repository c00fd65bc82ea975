"""The allocation-free global count (pvt_count_global_noalloc) against the
regular one (pvt_count_global) and the CPU oracle, word for word, on two
calls in a row.

Some callers cannot allocate device memory while they count (pre-sized
arenas, allocators they cannot reach from C, allocation-free latency
paths); this entry point keeps all its scratch in a fixed device array.
The second call checks that the shared array is cleared between calls.
Three graphs cover the three bitset widths the entry point instantiates:
out-degrees <= 32 (one word), 33..64 (two) and 97..126 (four words, the
top of its range).  This file is collected last so that a failure here comes
after every other test has run."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from paper_2001_06784_gb300 import graphgen

pytestmark = pytest.mark.gpu


def id_oriented_dag(row_ptr, col):
    """Out-lists "neighbours with a larger id" (an acyclic orientation)."""
    n = len(row_ptr) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    keep = col.astype(np.int64) > src
    odeg = np.bincount(src[keep], minlength=n)
    orow = np.zeros(n + 1, dtype=np.int64)
    orow[1:] = np.cumsum(odeg)
    return orow, col[keep].astype(np.uint32), int(odeg.max()) if n else 0


def clique_on_last(n, avg_deg, size, seed):
    """ER G(n, avg_deg) plus a clique on the `size` highest ids: with the
    larger-id orientation the first clique vertex has out-degree size - 1."""
    rp, col = graphgen.generate(n, er_avg_deg=avg_deg, seed=seed)
    e = graphgen.edge_list(rp, col)
    ids = np.arange(n - size, n)
    iu = np.triu_indices(size, 1)
    both = np.concatenate([e, np.stack([ids[iu[0]], ids[iu[1]]], axis=1)])
    return graphgen.from_edges(n, np.unique(both, axis=0))


CASES = {
    "one-word": lambda: graphgen.generate(3000, er_avg_deg=6.0, planted=[(5, 8, 14, 1.0)], seed=23),
    "two-word": lambda: graphgen.generate(4000, er_avg_deg=12.0, planted=[(8, 10, 40, 0.95), (3, 20, 30, 1.0)],
                                          seed=17),
    "four-word": lambda: clique_on_last(1500, 8.0, 111, 29),
}


def call_noalloc(n, orow_d, ocol_d, alpha, kmax, W, out, stream):
    from paper_2001_06784_gb300 import _lib
    return _lib.lib().pvt_count_global_noalloc(n, ctypes.c_void_p(orow_d.data_ptr()), ctypes.c_void_p(ocol_d.data_ptr()),
                                               alpha, kmax, W, ctypes.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_matches_regular_count_and_oracle_twice(name):
    import torch

    import paper_2001_06784_gb300 as pvt
    from paper_2001_06784_gb300 import _lib

    rp, col = CASES[name]()
    n = len(rp) - 1
    dev = torch.device("cuda:0")
    dag = pvt.orient(torch.from_numpy(rp).to(dev), torch.from_numpy(col.view(np.int32)).to(dev))
    orow, ocol, alpha = id_oriented_dag(rp, col)
    assert alpha <= 126
    assert {"one-word": alpha <= 32, "two-word": 32 < alpha <= 64, "four-word": 96 < alpha}[name], alpha
    kmax = alpha + 1
    W = (int(n).bit_length() + alpha + 1 + 63) // 64  # every count <= n * 2^alpha
    want = dag.count_global(kmax=kmax, W=W).cpu().numpy()
    ref = oracle.count(rp, col, kmax=kmax)["C"]
    assert pvt.to_ints(want) == ref
    orow_d = torch.from_numpy(orow).to(dev)
    ocol_d = torch.from_numpy(ocol.view(np.int32)).to(dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for call in range(2):
        out = torch.full((kmax + 1, W), -1, dtype=torch.int64, device=dev)
        _lib.check(call_noalloc(n, orow_d, ocol_d, alpha, kmax, W, out, stream))
        got = out.cpu().numpy()
        assert (got == want).all(), f"call {call}: counts differ from pvt_count_global"
        assert pvt.to_ints(got) == ref, f"call {call}: counts differ from the oracle"
    # sizes beyond the fixed scratch are refused before any launch
    assert call_noalloc(n, orow_d, ocol_d, 127, kmax, W, out, stream) == 1
    # an alpha below a real out-degree is refused (the walk checks every list)
    assert call_noalloc(n, orow_d, ocol_d, alpha - 1, kmax, W, out, stream) == 1
    # a NULL out-list array with n > 0 is refused
    st = _lib.lib().pvt_count_global_noalloc(n, ctypes.c_void_p(orow_d.data_ptr()), None, alpha, kmax, W,
                                             ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 1
    # and the entry point still counts correctly afterwards
    _lib.check(call_noalloc(n, orow_d, ocol_d, alpha, kmax, W, out, stream))
    assert (out.cpu().numpy() == want).all()
    dag.free()
