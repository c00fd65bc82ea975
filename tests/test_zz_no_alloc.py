"""The allocation-free global count (pvt_count_global_noalloc) against the
regular one (pvt_count_global), word for word, on two calls in a row.

Some callers cannot allocate device memory while they count (pre-sized
arenas, allocators they cannot reach from C, allocation-free latency
paths); this entry point keeps all its scratch in a fixed device array.
The second call checks that the shared array is cleared between calls.
This file is collected last so that a failure here comes after every other
test has run."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

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


def test_noalloc_matches_regular_count_twice():
    import torch

    import paper_2001_06784_gb300 as pvt
    from paper_2001_06784_gb300 import _lib

    rp, col = graphgen.generate(4000, er_avg_deg=12.0, planted=[(8, 10, 40, 0.95), (3, 20, 30, 1.0)], seed=17)
    n = len(rp) - 1
    dev = torch.device("cuda:0")
    dag = pvt.orient(torch.from_numpy(rp).to(dev), torch.from_numpy(col.view(np.int32)).to(dev))
    orow, ocol, alpha = id_oriented_dag(rp, col)
    assert alpha <= 126
    kmax = alpha + 1
    W = (int(n).bit_length() + alpha + 1 + 63) // 64  # every count <= n * 2^alpha
    want = dag.count_global(kmax=kmax, W=W).cpu().numpy()
    orow_d = torch.from_numpy(orow).to(dev)
    ocol_d = torch.from_numpy(ocol.view(np.int32)).to(dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for call in range(2):
        out = torch.full((kmax + 1, W), -1, dtype=torch.int64, device=dev)
        st = _lib.lib().pvt_count_global_noalloc(n, ctypes.c_void_p(orow_d.data_ptr()),
                                                 ctypes.c_void_p(ocol_d.data_ptr()), alpha, kmax, W,
                                                 ctypes.c_void_p(out.data_ptr()), stream)
        _lib.check(st)
        got = out.cpu().numpy()
        assert (got == want).all(), f"call {call}: counts differ from pvt_count_global"
    # sizes beyond the fixed scratch are refused before any launch
    st = _lib.lib().pvt_count_global_noalloc(n, ctypes.c_void_p(orow_d.data_ptr()), ctypes.c_void_p(ocol_d.data_ptr()),
                                             127, kmax, W, ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 1
    dag.free()
