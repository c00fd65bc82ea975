"""The C ABI library builds, loads without a GPU, and exports every function
include/pivoter.h declares; the binding declares the same set."""
from __future__ import annotations

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pivoter.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pvt_[a-z_]+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for fn in ("pvt_orient", "pvt_count_global", "pvt_count_local_vertex", "pvt_count_local_edge"):
        assert fn in names


def test_library_exports_every_declared_symbol():
    from paper_2001_06784_gb300 import _build, _lib
    path = _build.build()
    lib = ctypes.CDLL(path)
    for fn in declared_functions():
        assert hasattr(lib, fn), fn
    assert sorted(_lib.EXPORTS) == declared_functions()


def test_no_cuda_needed_for_error_paths():
    """Argument checks run on the host before any CUDA call."""
    from paper_2001_06784_gb300 import _lib
    lib = _lib.load()
    h = ctypes.c_void_p()
    st = lib.pvt_orient(-1, 0, None, None, 0, None, ctypes.byref(h), None)
    assert st == 1
    assert b"invalid" in lib.pvt_last_error()
    assert lib.pvt_dag_info(None, None, None, None, None) == 1
    lib.pvt_dag_free(None)
