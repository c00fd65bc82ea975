"""Seeded synthetic input graphs (CSR), shared by the library's tests and
benchmarks and by the CPU oracle.

This module only produces inputs: simple undirected graphs in the CSR layout
the library takes (``row_ptr`` int64[n+1], ``col`` uint32[2m], rows sorted,
symmetric, no self-loops), per the paper's problem statement (Sec. 3.1).  It
contains none of the clique-counting arithmetic.  The generators themselves
are C (``graphgen.c``), compiled on first use.

The named workloads stand in for the SNAP social/web networks of the paper's
Tab. main, which are not available here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``graphgen.c`` into ``libgraphgen.so`` next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i64, u32, u64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
            lib.gg_begin.restype = vp
            lib.gg_begin.argtypes = [i64]
            lib.gg_free.argtypes = [vp]
            lib.gg_add_edge.argtypes = [vp, u32, u32]
            lib.gg_add_er.argtypes = [vp, dbl, u64]
            lib.gg_add_chung_lu.argtypes = [vp, i64, dbl, u64]
            lib.gg_add_planted.argtypes = [vp, i64, ctypes.c_int, ctypes.c_int, dbl, u64]
            lib.gg_finish.restype = i64
            lib.gg_finish.argtypes = [vp]
            lib.gg_copy_csr.argtypes = [vp, vp, vp]
            lib.gg_last_chung_lu_edges.restype = i64
            lib.gg_last_chung_lu_edges.argtypes = [vp]
            _lib = lib
    return _lib


def generate(n, *, er_avg_deg=None, chung_lu=None, planted=(), seed=0):
    """Build one graph.

    ``er_avg_deg``: add G(n, p) with p = avg/(n-1).
    ``chung_lu``: ``(m, beta)`` power-law Chung-Lu with about m edges.
    ``planted``: iterable of ``(count, smin, smax, rho)`` community groups.
    Returns ``(row_ptr int64[n+1], col uint32[2m])``.
    """
    lib = _load()
    h = lib.gg_begin(int(n))
    if not h:
        raise ValueError("bad vertex count")
    try:
        if er_avg_deg is not None and lib.gg_add_er(h, float(er_avg_deg), seed) != 0:
            raise MemoryError("graphgen: ER failed")
        if chung_lu is not None:
            rc = lib.gg_add_chung_lu(h, int(chung_lu[0]), float(chung_lu[1]), seed)
            if rc != 0:
                raise ValueError(f"graphgen: Chung-Lu failed ({rc})")
        for gi, (count, smin, smax, rho) in enumerate(planted):
            rc = lib.gg_add_planted(h, int(count), int(smin), int(smax), float(rho), seed * 1000 + gi)
            if rc != 0:
                raise ValueError(f"graphgen: planted communities failed ({rc})")
        m = lib.gg_finish(h)
        if m < 0:
            raise MemoryError("graphgen: finish failed")
        row_ptr = np.empty(int(n) + 1, dtype=np.int64)
        col = np.empty(max(2 * m, 1), dtype=np.uint32)
        lib.gg_copy_csr(h, row_ptr.ctypes.data, col.ctypes.data)
        return row_ptr, col[: 2 * m]
    finally:
        lib.gg_free(h)


def from_edges(n, edges):
    """CSR of the simple undirected graph on ``n`` vertices with the given
    edge list (pairs); self-loops and repeats are dropped."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    a = np.minimum(e[:, 0], e[:, 1])
    b = np.maximum(e[:, 0], e[:, 1])
    key = np.unique(a * np.int64(n) + b)
    a, b = key // n, key % n
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int64)
    return row_ptr, dst.astype(np.uint32)


def edge_list(row_ptr, col):
    """Undirected edges (u < v) in the library's canonical edge-id order:
    lexicographic in (u, v), i.e. the upper triangle of the CSR row by row."""
    n = len(row_ptr) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    dst = col.astype(np.int64)
    keep = src < dst
    return np.stack([src[keep], dst[keep]], axis=1)


def induced_subgraph(row_ptr, col, verts):
    """CSR of the subgraph induced on ``verts`` (relabelled 0..len-1 in the
    given order)."""
    verts = np.asarray(verts, dtype=np.int64)
    n = len(row_ptr) - 1
    loc = np.full(n, -1, dtype=np.int64)
    loc[verts] = np.arange(len(verts))
    pairs = []
    for i, v in enumerate(verts):
        nb = col[row_ptr[v]:row_ptr[v + 1]].astype(np.int64)
        j = loc[nb]
        j = j[j > i]
        if len(j):
            pairs.append(np.stack([np.full(len(j), i), j], axis=1))
    e = np.concatenate(pairs) if pairs else np.zeros((0, 2), dtype=np.int64)
    return from_edges(len(verts), e)


# Workloads shaped like the paper's graphs (Tab. main): name -> generator args.
WORKLOADS = {
    # ER G(2000, avg degree 20) plus one planted 30-clique.
    "er2k_d20_clique30": dict(n=2000, er_avg_deg=20.0, planted=[(1, 30, 30, 1.0)], seed=1),
    # Chung-Lu n=1M, m~10M, exponent 2.1, 500 communities of 20-60 at density 0.9.
    "cl1m_m10m_b2.1_comm500": dict(n=1_000_000, chung_lu=(10_000_000, 2.1),
                                   planted=[(500, 20, 60, 0.9)], seed=2),
    # Chung-Lu n=500k, m~8M, exponent 2.3, 200 planted cliques of 15-40.
    "cl500k_m8m_b2.3_clq200": dict(n=500_000, chung_lu=(8_000_000, 2.3),
                                   planted=[(200, 15, 40, 1.0)], seed=3),
    # Chung-Lu n=3M, m~117M, exponent 2.0, 2000 communities of 50-120 at 0.8
    # (shaped like com-orkut: n 3.07M, m 117M).
    "cl3m_m117m_b2.0_comm2000": dict(n=3_000_000, chung_lu=(117_000_000, 2.0),
                                     planted=[(2000, 50, 120, 0.8)], seed=4),
}


def workload(name):
    """Generate a named workload graph: ``(row_ptr, col)``."""
    return generate(**WORKLOADS[name])
