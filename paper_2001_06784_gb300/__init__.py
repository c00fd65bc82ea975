"""Exact k-clique counts for every k on one GPU, with the Succinct Clique Tree
of Jain & Seshadhri, "The Power of Pivoting for Exact Clique Counting"
(WSDM 2020).

Thin binding over the C ABI of ``libpivoter.so`` (``include/pivoter.h``):
PyTorch supplies device memory and streams; every step of the computation
runs in the library's CUDA kernels.  There is no CPU fallback: without the
built library every entry point raises ImportError.

    import torch, paper_2001_06784_gb300 as pvt
    dag = pvt.orient(row_ptr.cuda(), col.cuda())      # degeneracy DAG
    C = pvt.to_ints(dag.count_global())               # C[k], k = 0..alpha+1
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import PVT_PROFILE, PVT_VALIDATE, PivoterError

__all__ = ["orient", "Dag", "Server", "local_distribution", "to_ints", "count_global_host", "PivoterError"]


def _stream_handle(stream, device):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


class Dag:
    """A graph oriented along its degeneracy order, resident on the GPU.

    The CSR tensors it was built from are borrowed (kept alive here) and
    must not be modified while the Dag exists."""

    def __init__(self, handle, row_ptr, col):
        self._h = handle
        self._keep = (row_ptr, col)
        self.device = row_ptr.device
        n, m = ctypes.c_int64(), ctypes.c_int64()
        a, w = ctypes.c_int32(), ctypes.c_int32()
        _lib.check(_lib.lib().pvt_dag_info(self._h, ctypes.byref(n), ctypes.byref(m),
                                           ctypes.byref(a), ctypes.byref(w)))
        self.n, self.m, self.alpha, self.min_words = n.value, m.value, a.value, w.value

    def _args(self, kmax, W):
        kmax = self.alpha + 1 if kmax is None else int(kmax)
        W = self.min_words if W is None else int(W)
        return kmax, W

    def _out(self, rows, kmax, W, out):
        shape = (rows, kmax + 1, W) if rows is not None else (kmax + 1, W)
        if out is None:
            return torch.empty(shape, dtype=torch.int64, device=self.device)
        if out.dtype != torch.int64 or tuple(out.shape) != shape or not out.is_contiguous():
            raise ValueError(f"out must be a contiguous int64 tensor of shape {shape}")
        return out

    def cores(self, stream=None):
        """Core number of every vertex (uint32 values in an int32 tensor [n])."""
        out = torch.empty(self.n, dtype=torch.int32, device=self.device)
        _lib.check(_lib.lib().pvt_dag_cores(self._h, ctypes.c_void_p(out.data_ptr() if self.n else 0),
                                            _stream_handle(stream, self.device)))
        return out

    def out_lists(self, stream=None):
        """The orientation: (orow int64 [n+1], ocol int32 [m]) device tensors,
        N+(v) = ocol[orow[v]:orow[v+1]] sorted by id (pvt_dag_out_lists)."""
        orow = torch.empty(self.n + 1, dtype=torch.int64, device=self.device)
        ocol = torch.empty(max(self.m, 1), dtype=torch.int32, device=self.device)
        _lib.check(_lib.lib().pvt_dag_out_lists(self._h, ctypes.c_void_p(orow.data_ptr()),
                                                ctypes.c_void_p(ocol.data_ptr()), _stream_handle(stream, self.device)))
        return orow, ocol[:self.m]

    def leaf_depths(self, stream=None):
        """Leaves of the last global count by depth h + p, numpy uint64
        [alpha+2] (pvt_dag_leaf_depths)."""
        out = np.zeros(self.alpha + 2, dtype=np.uint64)
        _lib.check(_lib.lib().pvt_dag_leaf_depths(self._h, out.ctypes.data, _stream_handle(stream, self.device)))
        return out

    def count_global(self, kmax=None, W=None, out=None, stream=None):
        """C_k for k = 0..kmax as an int64 tensor [kmax+1, W] of 64-bit words
        (little-endian, reinterpret as unsigned)."""
        kmax, W = self._args(kmax, W)
        out = self._out(None, kmax, W, out)
        _lib.check(_lib.lib().pvt_count_global(self._h, kmax, W, ctypes.c_void_p(out.data_ptr()),
                                               _stream_handle(stream, self.device)))
        return out

    def count_hist(self, begin=0, end=None, hist=None, kmax=None, stream=None):
        """Add the (h, p) path counts of the roots begin <= r < end to hist
        (int64 tensor [alpha+2, alpha+2], zeros if None) and return it: the
        checkpointable state of a global count (pvt_count_hist)."""
        kmax = self.alpha + 1 if kmax is None else int(kmax)
        end = self.n if end is None else int(end)
        H = self.alpha + 2
        if hist is None:
            hist = torch.zeros((H, H), dtype=torch.int64, device=self.device)
        if hist.dtype != torch.int64 or tuple(hist.shape) != (H, H) or not hist.is_contiguous():
            raise ValueError(f"hist must be a contiguous int64 tensor of shape {(H, H)}")
        _lib.check(_lib.lib().pvt_count_hist(self._h, int(begin), end, kmax, ctypes.c_void_p(hist.data_ptr()),
                                             _stream_handle(stream, self.device)))
        return hist

    def combine_hist(self, hist, kmax=None, W=None, out=None, stream=None):
        """C_k words [kmax+1, W] from a path-count histogram (pvt_combine_hist)."""
        kmax, W = self._args(kmax, W)
        out = self._out(None, kmax, W, out)
        _lib.check(_lib.lib().pvt_combine_hist(self._h, ctypes.c_void_p(hist.data_ptr()), kmax, W,
                                               ctypes.c_void_p(out.data_ptr()), _stream_handle(stream, self.device)))
        return out

    def count_local_vertex(self, kmax=None, W=None, out=None, stream=None):
        """c_k(v) as an int64 tensor [n, kmax+1, W]."""
        kmax, W = self._args(kmax, W)
        out = self._out(self.n, kmax, W, out)
        _lib.check(_lib.lib().pvt_count_local_vertex(self._h, kmax, W, ctypes.c_void_p(out.data_ptr()),
                                                     _stream_handle(stream, self.device)))
        return out

    def count_local_edge(self, kmax=None, W=None, out=None, stream=None):
        """c_k(e) as an int64 tensor [m, kmax+1, W], rows in edge-id order
        (lexicographic (min, max))."""
        kmax, W = self._args(kmax, W)
        out = self._out(self.m, kmax, W, out)
        _lib.check(_lib.lib().pvt_count_local_edge(self._h, kmax, W, ctypes.c_void_p(out.data_ptr()),
                                                   _stream_handle(stream, self.device)))
        return out

    PHASES = ("peel", "orient", "walk_d32", "walk_d64", "walk_d128", "walk_d256", "walk_d512", "walk_d1024",
              "finish", "walk_frames")

    def stats(self):
        """Statistics of the last call on this dag (see pvt_stats): SCT walk
        sizes, kernel launches, roots per out-degree class and, when
        profiling is on, device milliseconds per phase."""
        st = _lib.Stats()
        _lib.check(_lib.lib().pvt_dag_stats(self._h, ctypes.byref(st)))
        return dict(sct_nodes=st.sct_nodes, sct_leaves=st.sct_leaves, pivot_words=st.pivot_words,
                    launches=st.launches, roots=list(st.roots), class_words=list(st.class_words),
                    frame_words=st.frame_words, frames=st.frames,
                    ms=dict(zip(self.PHASES, list(st.ms))), peel_rounds=st.peel_rounds,
                    peel_levels=st.peel_levels)

    def policy(self):
        """The dag's launch policy (pvt_policy) as a dict."""
        pol = _lib.Policy()
        _lib.check(_lib.lib().pvt_dag_get_policy(self._h, ctypes.byref(pol)))
        return dict(persistent=bool(pol.persistent), chunk=pol.chunk, split=list(pol.split), graph=bool(pol.graph),
                    frames=bool(pol.frames), wait_limit_us=pol.wait_limit_us, lanes=bool(pol.lanes),
                    cta=list(pol.cta), serial=bool(pol.serial))

    def set_policy(self, persistent: bool = True, chunk: int = 4, split=None, graph: bool = False,
                   frames: bool = True, wait_limit_us: int = 0, lanes: bool = True, cta=None, serial: bool = False):
        """Launch policy of the walk kernels: persistent warps with a device
        work queue (default) or the plain one-warp-per-root form; per
        out-degree class whether heavy roots split across warps (7 flags,
        default: every class above out-degree 32); whether global counts
        replay a recorded CUDA graph; whether global counts walk the small
        labels of the classes above 32 in a second, lighter kernel;
        wait_limit_us > 0 shortens the bounded device waits (a test of the
        PVT_ETIMEOUT path); whether one-word labels of global counts are
        walked one subtree per lane (lanes) or one per warp; per out-degree
        class whether a thread block walks each root (cta, classes 4..6);
        serial runs the classes one after another (isolated phase times)."""
        split = [0, 0, 1, 1, 1, 1, 1] if split is None else [int(x) for x in split]
        cta = [0, 0, 0, 0, 0, 1, 1] if cta is None else [int(x) for x in cta]
        if len(split) != 7 or len(cta) != 7:
            raise ValueError("split and cta need one flag per out-degree class (7)")
        pol = _lib.Policy(1 if persistent else 0, int(chunk), (ctypes.c_int32 * 7)(*split), 1 if graph else 0,
                          1 if frames else 0, int(wait_limit_us), 1 if lanes else 0, (ctypes.c_int32 * 7)(*cta),
                          1 if serial else 0)
        _lib.check(_lib.lib().pvt_dag_set_policy(self._h, ctypes.byref(pol)))

    def autotune(self, kmax=None, W=None, out=None, stream=None):
        """Pick the launch policy per out-degree class by timing three
        candidates (pvt_dag_autotune); sets it on the dag and returns
        (policy dict, ms [3][7] numpy array, counts tensor)."""
        kmax, W = self._args(kmax, W)
        out = self._out(None, kmax, W, out)
        pol = _lib.Policy()
        ms = np.zeros((3, 7), dtype=np.float32)
        _lib.check(_lib.lib().pvt_dag_autotune(self._h, kmax, W, ctypes.c_void_p(out.data_ptr()),
                                               _stream_handle(stream, self.device), ctypes.byref(pol),
                                               ms.ctypes.data))
        return (dict(persistent=bool(pol.persistent), chunk=pol.chunk, split=list(pol.split),
                     graph=bool(pol.graph), frames=bool(pol.frames), wait_limit_us=pol.wait_limit_us,
                     lanes=bool(pol.lanes), cta=list(pol.cta), serial=bool(pol.serial)), ms, out)

    def set_profiling(self, on: bool):
        _lib.check(_lib.lib().pvt_dag_set_profiling(self._h, 1 if on else 0))

    def free(self):
        if self._h:
            _lib.lib().pvt_dag_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def orient(row_ptr: torch.Tensor, col: torch.Tensor, *, validate: bool = False, profile: bool = False,
           stream=None) -> Dag:
    """Orient a CSR graph (device tensors: row_ptr int64[n+1], col int32 or
    uint32 [2m]) along a degeneracy order on the GPU."""
    if not (row_ptr.is_cuda and col.is_cuda):
        raise ValueError("row_ptr and col must be CUDA tensors")
    if row_ptr.dtype != torch.int64 or col.dtype not in (torch.int32, torch.uint32):
        raise ValueError("row_ptr must be int64 and col int32/uint32")
    row_ptr = row_ptr.contiguous()
    col = col.contiguous()
    n = row_ptr.numel() - 1
    nnz = col.numel()
    h = ctypes.c_void_p()
    alpha = ctypes.c_int32()
    with torch.cuda.device(row_ptr.device):
        _lib.check(_lib.lib().pvt_orient(n, nnz, ctypes.c_void_p(row_ptr.data_ptr()),
                                         ctypes.c_void_p(col.data_ptr() if nnz else 0),
                                         (PVT_VALIDATE if validate else 0) | (PVT_PROFILE if profile else 0),
                                         _stream_handle(stream, row_ptr.device), ctypes.byref(h),
                                         ctypes.byref(alpha)))
    return Dag(h, row_ptr, col)


class Server:
    """Clique-count query server with continuous batching (pvt_server_*).

    submit() takes a host CSR (numpy) and a query kind ("global", "vertex"
    or "edge"); queries are admitted by device memory and slots, oriented and
    walked in shared batched launches; result() returns the words as a numpy
    uint64 array [rows, K, W] (rows = 1 for global) and the latency."""

    KINDS = {"global": _lib.QUERY_GLOBAL, "vertex": _lib.QUERY_VERTEX, "edge": _lib.QUERY_EDGE}

    def __init__(self, mem_budget: int = 8 << 30, max_inflight: int = 1024, max_batch: int = 256,
                 streams: int = 4, direct_edges: int = 0):
        cfg = _lib.ServerConfig(int(mem_budget), int(max_inflight), int(max_batch), int(streams), int(direct_edges))
        h = ctypes.c_void_p()
        _lib.check(_lib.lib().pvt_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, row_ptr, col, kind: str = "global", kmax=None) -> int:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        cl = np.ascontiguousarray(col, dtype=np.uint32)
        t = ctypes.c_uint64()
        _lib.check(_lib.lib().pvt_server_submit(self._h, len(rp) - 1, len(cl), rp.ctypes.data,
                                                cl.ctypes.data if len(cl) else None, self.KINDS[kind],
                                                -1 if kmax is None else int(kmax), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> bool:
        done = ctypes.c_int32()
        _lib.check(_lib.lib().pvt_server_wait(self._h, ticket, int(timeout_ms), ctypes.byref(done)))
        return bool(done.value)

    def result(self, ticket: int):
        """(words uint64[rows, K, W], latency seconds); releases the query."""
        rows, K, W = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _lib.check(_lib.lib().pvt_server_result(self._h, ticket, ctypes.byref(rows), ctypes.byref(K),
                                                ctypes.byref(W), None, 0, None))
        out = np.empty((max(rows.value, 0), K.value, W.value), dtype=np.uint64)
        lat = ctypes.c_double()
        _lib.check(_lib.lib().pvt_server_result(self._h, ticket, None, None, None,
                                                out.ctypes.data if out.size else None, out.size,
                                                ctypes.byref(lat)))
        return out, lat.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().pvt_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def local_distribution(table: torch.Tensor, k: int, stream=None):
    """f_k(b) over the rows of a local count table (int64 tensor
    [rows, K, W] from count_local_vertex / count_local_edge): returns
    (values int64 [D, W], counts int64 [D]), the D distinct values b of
    column k and how many rows take each, in no particular order."""
    if table.dim() != 3 or table.dtype != torch.int64 or not table.is_cuda or not table.is_contiguous():
        raise ValueError("table must be a contiguous CUDA int64 tensor [rows, K, W]")
    rows, K, W = table.shape
    values = torch.empty((max(rows, 1), W), dtype=torch.int64, device=table.device)
    counts = torch.empty(max(rows, 1), dtype=torch.int64, device=table.device)
    nd = ctypes.c_int64()
    _lib.check(_lib.lib().pvt_local_distribution(ctypes.c_void_p(table.data_ptr() if rows else 0), rows, K, W,
                                                 int(k), ctypes.c_void_p(values.data_ptr()),
                                                 ctypes.c_void_p(counts.data_ptr()), ctypes.byref(nd),
                                                 _stream_handle(stream, table.device)))
    return values[:nd.value], counts[:nd.value]


def measure_popc_rate(device="cuda:0", stream=None):
    """AND + population count + add triples per second that the device
    sustains (pvt_measure_popc_rate): the walk kernels' roofline peak."""
    rate = ctypes.c_double()
    dev = torch.device(device)
    with torch.cuda.device(dev):
        _lib.check(_lib.lib().pvt_measure_popc_rate(ctypes.byref(rate), _stream_handle(stream, dev)))
    return rate.value


def to_ints(t):
    """Word tensor [..., W] (64-bit little-endian words) -> nested lists of
    Python ints."""
    a = t.detach().cpu().numpy().view(np.uint64) if isinstance(t, torch.Tensor) else np.asarray(t, np.uint64)
    if a.ndim == 1:
        v = 0
        for x in a[::-1]:
            v = (v << 64) | int(x)
        return v
    return [to_ints(x) for x in a]


def count_global_host(row_ptr, col, kmax=None, device="cuda"):
    """End-to-end convenience: host CSR (numpy) in, C_k as Python ints out."""
    rp = torch.as_tensor(np.asarray(row_ptr, dtype=np.int64)).to(device)
    cl = torch.as_tensor(np.asarray(col, dtype=np.uint32).view(np.int32)).to(device)
    dag = orient(rp, cl)
    try:
        return to_ints(dag.count_global(kmax))
    finally:
        dag.free()
