"""CPU oracle for exact all-k clique counts via the Succinct Clique Tree.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline leg may import this package; the library
itself never does.  It shares no code with the CUDA path.

The arithmetic lives in ``pivoter_oracle.c`` (plain sequential C with its
own multi-limb integers); this module compiles it, marshals arrays and turns
limb arrays into Python integers.  Each result is exact or an error.

Parity: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, brute-force enumeration, matrix identities and the
unique-encoding theorem (Thm. scr).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pivoter_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {1: "invalid argument", 3: "out of memory", 4: "limb overflow", 7: "path buffer too small"}


def build(force: bool = False) -> str:
    """Compile the oracle into ``liboracle.so`` beside its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def declare(lib):
    """Set the ctypes signatures of an oracle library."""
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.orc_orient.restype = i32
    lib.orc_orient.argtypes = [i64, vp, vp, vp, vp, vp]
    lib.orc_count.restype = i32
    lib.orc_count.argtypes = [i64, vp, vp, i32, i32, vp, vp, vp, vp, i64, i32, vp, vp, i32, vp, vp]
    lib.orc_paths.restype = i64
    lib.orc_paths.argtypes = [i64, vp, vp, vp, i64]
    lib.orc_triangles.restype = i64
    lib.orc_triangles.argtypes = [i64, vp, vp, i32]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = declare(ctypes.CDLL(build()))
    return _lib


def _csr(row_ptr, col):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.uint32)
    if len(col) == 0:
        col = np.zeros(1, dtype=np.uint32)
    return row_ptr, col


def orient(row_ptr, col):
    """Degeneracy order.  Returns ``(rank uint32[n], core uint32[n], alpha)``:
    removal index of each vertex, its core number, and the largest
    out-degree of the orientation (Lemma degen)."""
    row_ptr, col = _csr(row_ptr, col)
    n = len(row_ptr) - 1
    rank = np.zeros(max(n, 1), dtype=np.uint32)
    core = np.zeros(max(n, 1), dtype=np.uint32)
    alpha = ctypes.c_int32(0)
    rc = _load().orc_orient(n, row_ptr.ctypes.data, col.ctypes.data, rank.ctypes.data,
                            core.ctypes.data, ctypes.addressof(alpha))
    if rc:
        raise RuntimeError(f"oracle: {ERRORS.get(rc, rc)}")
    return rank[:n], core[:n], int(alpha.value)


def limbs_needed(n: int, alpha: int) -> int:
    """32-bit limbs that hold every count: each clique lies in {r} + N+(r)
    for its first vertex r, so C_k <= n * 2^alpha."""
    bits = int(n).bit_length() + alpha + 2
    return bits // 32 + 1


def to_int(limbs):
    """Limb array [..., nl] (uint32, least significant first) -> nested
    lists of Python ints over the leading axes."""
    a = np.asarray(limbs, dtype=np.uint64)
    if a.ndim == 1:
        v = 0
        for x in a[::-1]:
            v = (v << 32) | int(x)
        return v
    return [to_int(x) for x in a]


def count(row_ptr, col, *, kmax: int = -1, vertex: bool = False, edge: bool = False,
          roots=None, threads: int = 1, nl: int | None = None, hist_dim: int = 0, dag=None):
    """Exact clique counts, k = 0..kmax (kmax < 0: every k up to alpha+1).

    Returns a dict: ``C`` (list of ints), ``cv`` / ``ce`` (limb arrays
    [n][K][nl] / [m][K][nl], only if asked), ``nl``, ``alpha``, ``kmax`` and
    SCT statistics ``nodes``, ``leaves``, ``sum_s`` and ``chain`` (the nodes
    below the topmost clique label of each path, which a walk that closes
    clique labels at once never visits); ``hist`` ((h, p) leaf histogram) if
    ``hist_dim`` > 0.  ``dag = (orow, ocol)`` walks that acyclic orientation
    (out-lists sorted ascending) instead of the degeneracy order; ``alpha``
    is then its largest out-degree.
    """
    row_ptr, col = _csr(row_ptr, col)
    n = len(row_ptr) - 1
    m = int(row_ptr[-1]) // 2
    if dag is not None:
        orow = np.ascontiguousarray(dag[0], dtype=np.int64)
        ocol = np.ascontiguousarray(dag[1], dtype=np.uint32)
        if len(orow) != n + 1:
            raise ValueError("dag row pointers need n + 1 entries")
        alpha = int(np.diff(orow).max()) if n else 0
        ocol_buf = ocol if len(ocol) else np.zeros(1, dtype=np.uint32)
        dag_ptrs = (orow.ctypes.data, ocol_buf.ctypes.data)
    else:
        _, _, alpha = orient(row_ptr, col)
        dag_ptrs = (None, None)
    if kmax < 0:
        kmax = alpha + 1
    if nl is None:
        nl = limbs_needed(n, alpha)
    K = kmax + 1
    C = np.zeros((K, nl), dtype=np.uint32)
    cv = np.zeros((max(n, 1), K, nl), dtype=np.uint32) if vertex else None
    ce = np.zeros((max(m, 1), K, nl), dtype=np.uint32) if edge else None
    if roots is not None:
        roots = np.ascontiguousarray(roots, dtype=np.uint32)
        rptr, nroots = roots.ctypes.data, len(roots)
        if nroots == 0:
            rptr, nroots = np.zeros(1, dtype=np.uint32).ctypes.data, 0
    else:
        rptr, nroots = None, n
    stats = np.zeros(8, dtype=np.uint64)
    hist = np.zeros((hist_dim, hist_dim), dtype=np.uint64) if hist_dim else None
    rc = _load().orc_count(n, row_ptr.ctypes.data, col.ctypes.data, kmax, nl, C.ctypes.data,
                           cv.ctypes.data if vertex else None, ce.ctypes.data if edge else None,
                           rptr, nroots, threads, stats.ctypes.data,
                           hist.ctypes.data if hist_dim else None, hist_dim, *dag_ptrs)
    if rc:
        raise RuntimeError(f"oracle: {ERRORS.get(rc, rc)}")
    out = dict(C=to_int(C), nl=nl, alpha=alpha, kmax=kmax,
               nodes=int(stats[0]), leaves=int(stats[1]), sum_s=int(stats[2]), chain=int(stats[5]))
    if vertex:
        out["cv"] = cv[:n]
    if edge:
        out["ce"] = ce[:m]
    if hist_dim:
        out["hist"] = hist
    return out


def triangles(row_ptr, col, threads: int = 1) -> int:
    """Number of triangles (C_3, Sec. 2), by plain enumeration over the
    (degree, id) order, independent of the SCT walk (orc_triangles)."""
    row_ptr, col = _csr(row_ptr, col)
    t = _load().orc_triangles(len(row_ptr) - 1, row_ptr.ctypes.data, col.ctypes.data, int(threads))
    if t < 0:
        raise RuntimeError("oracle: triangles: invalid argument or out of memory")
    return int(t)


def frequency(table, k: int) -> dict:
    """f_k(b): how many rows of a local count table (limb array
    [rows][K][nl] from ``count``) take each value b in column k -- the
    per-vertex clique distributions of the paper's experiments
    ("Demonstrations of Pivoter"), or the same over edges.  Returns
    {b: f_k(b)} with exact integer keys."""
    col = np.asarray(table)[:, k, :]
    if len(col) == 0:
        return {}
    vals, cnt = np.unique(col, axis=0, return_counts=True)
    return {to_int(v): int(c) for v, c in zip(vals, cnt)}


def paths(row_ptr, col, cap: int = 1 << 22):
    """Every root-to-leaf path T of the SCT as ``(H(T), P(T))`` vertex lists,
    in walk order (tiny graphs only)."""
    row_ptr, col = _csr(row_ptr, col)
    n = len(row_ptr) - 1
    out = np.zeros(cap, dtype=np.int32)
    ln = _load().orc_paths(n, row_ptr.ctypes.data, col.ctypes.data, out.ctypes.data, cap)
    if ln < 0:
        raise RuntimeError(f"oracle: {ERRORS.get(-ln, -ln)}")
    res, i = [], 0
    while i < ln:
        h, p = int(out[i]), int(out[i + 1])
        H = [int(x) for x in out[i + 2:i + 2 + h]]
        P = [int(x) for x in out[i + 2 + h:i + 2 + h + p]]
        res.append((H, P))
        i += 2 + h + p
    return res
