"""ctypes declarations of libpivoter's C ABI (include/pivoter.h).

Argument marshalling only.  The library is the in-tree ``libpivoter.so``;
there is no fallback: importing this module without it raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpivoter.so")

STATUS = {
    0: "PVT_OK", 1: "PVT_EINVAL", 2: "PVT_ENOTSIMPLE", 3: "PVT_ENOMEM", 4: "PVT_EOVERFLOW",
    5: "PVT_ECUDA", 6: "PVT_ETIMEOUT", 7: "PVT_EINTERNAL",
}
PVT_VALIDATE = 0x1
PVT_PROFILE = 0x2


class Stats(ctypes.Structure):
    """pvt_stats (include/pivoter.h)."""
    _fields_ = [("sct_nodes", ctypes.c_uint64), ("sct_leaves", ctypes.c_uint64),
                ("pivot_words", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("roots", ctypes.c_uint64 * 7), ("class_words", ctypes.c_uint64 * 7),
                ("frame_words", ctypes.c_uint64), ("frames", ctypes.c_uint64),
                ("ms", ctypes.c_float * 10), ("peel_rounds", ctypes.c_uint32), ("peel_levels", ctypes.c_uint32)]

class Policy(ctypes.Structure):
    """pvt_policy (include/pivoter.h)."""
    _fields_ = [("persistent", ctypes.c_int32), ("chunk", ctypes.c_int32), ("split", ctypes.c_int32 * 7),
                ("graph", ctypes.c_int32), ("frames", ctypes.c_int32), ("wait_limit_us", ctypes.c_int32),
                ("lanes", ctypes.c_int32), ("cta", ctypes.c_int32 * 7), ("serial", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    """pvt_server_config (include/pivoter.h)."""
    _fields_ = [("mem_budget", ctypes.c_size_t), ("max_inflight", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("streams", ctypes.c_int32), ("direct_edges", ctypes.c_int64)]


QUERY_GLOBAL, QUERY_VERTEX, QUERY_EDGE = 0, 1, 2

# every symbol include/pivoter.h declares
EXPORTS = ("pvt_orient", "pvt_dag_info", "pvt_dag_cores", "pvt_local_distribution", "pvt_count_hist", "pvt_combine_hist", "pvt_count_global", "pvt_count_local_vertex",
           "pvt_count_local_edge", "pvt_dag_stats", "pvt_dag_set_profiling", "pvt_dag_set_policy",
           "pvt_dag_get_policy", "pvt_dag_autotune",
           "pvt_count_global_noalloc", "pvt_server_create", "pvt_server_submit", "pvt_server_wait",
           "pvt_server_result", "pvt_server_destroy", "pvt_dag_free",
           "pvt_last_error", "pvt_measure_popc_rate", "pvt_dag_leaf_depths", "pvt_dag_out_lists")


class PivoterError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def load(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libpivoter.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
    lib.pvt_orient.restype = i32
    lib.pvt_orient.argtypes = [i64, i64, vp, vp, u32, vp, ctypes.POINTER(vp), ctypes.POINTER(i32)]
    lib.pvt_dag_info.restype = i32
    lib.pvt_dag_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                 ctypes.POINTER(i32)]
    lib.pvt_measure_popc_rate.restype = i32
    lib.pvt_measure_popc_rate.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
    lib.pvt_count_hist.restype = i32
    lib.pvt_count_hist.argtypes = [vp, i64, i64, i32, vp, vp]
    lib.pvt_combine_hist.restype = i32
    lib.pvt_combine_hist.argtypes = [vp, vp, i32, i32, vp, vp]
    lib.pvt_local_distribution.restype = i32
    lib.pvt_local_distribution.argtypes = [vp, i64, i32, i32, i32, vp, vp, ctypes.POINTER(i64), vp]
    lib.pvt_dag_cores.restype = i32
    lib.pvt_dag_cores.argtypes = [vp, vp, vp]
    lib.pvt_dag_leaf_depths.restype = i32
    lib.pvt_dag_leaf_depths.argtypes = [vp, vp, vp]
    lib.pvt_dag_out_lists.restype = i32
    lib.pvt_dag_out_lists.argtypes = [vp, vp, vp, vp]
    for fn in ("pvt_count_global", "pvt_count_local_vertex", "pvt_count_local_edge"):
        f = getattr(lib, fn)
        f.restype = i32
        f.argtypes = [vp, i32, i32, vp, vp]
    lib.pvt_dag_stats.restype = i32
    lib.pvt_dag_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.pvt_dag_set_profiling.restype = i32
    lib.pvt_dag_set_profiling.argtypes = [vp, i32]
    lib.pvt_dag_set_policy.restype = i32
    lib.pvt_dag_set_policy.argtypes = [vp, ctypes.POINTER(Policy)]
    lib.pvt_dag_get_policy.restype = i32
    lib.pvt_dag_get_policy.argtypes = [vp, ctypes.POINTER(Policy)]
    lib.pvt_dag_autotune.restype = i32
    lib.pvt_dag_autotune.argtypes = [vp, i32, i32, vp, vp, ctypes.POINTER(Policy), vp]
    lib.pvt_count_global_noalloc.restype = i32
    lib.pvt_count_global_noalloc.argtypes = [i64, vp, vp, i32, i32, i32, vp, vp]
    lib.pvt_server_create.restype = i32
    lib.pvt_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    lib.pvt_server_submit.restype = i32
    lib.pvt_server_submit.argtypes = [vp, i64, i64, vp, vp, i32, i32, ctypes.POINTER(ctypes.c_uint64)]
    lib.pvt_server_wait.restype = i32
    lib.pvt_server_wait.argtypes = [vp, ctypes.c_uint64, i32, ctypes.POINTER(i32)]
    lib.pvt_server_result.restype = i32
    lib.pvt_server_result.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                      ctypes.POINTER(i32), vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)]
    lib.pvt_server_destroy.restype = None
    lib.pvt_server_destroy.argtypes = [vp]
    lib.pvt_dag_free.restype = None
    lib.pvt_dag_free.argtypes = [vp]
    lib.pvt_last_error.restype = ctypes.c_char_p
    lib.pvt_last_error.argtypes = []
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def check(status: int):
    if status != 0:
        msg = lib().pvt_last_error().decode(errors="replace")
        raise PivoterError(status, msg)
