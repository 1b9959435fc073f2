"""The C ABI: liblg.so builds for sm_103a, loads without a GPU and exports every
symbol that include/lg.h declares (no compute call is made here)."""
import ctypes
import os
import re

import paper_2010_15879_gb300 as lg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lg_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("lg_encode", "lg_neighbors", "lg_bfs", "lg_pagerank", "lg_free", "lg_stats_get",
                     "lg_arrays_get", "lg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lg.build()
    lib = ctypes.CDLL(lg.LIB)
    for name in declared_symbols():
        assert hasattr(lib, name), f"liblg.so does not export {name}"


def test_argument_errors_need_no_gpu():
    lib = lg.load(auto_build=True)
    out = ctypes.c_void_p(123)
    # NULL inputs are rejected before any CUDA call
    assert lib.lg_encode(None, None, None, 4, 0, None, None, ctypes.byref(out)) == 1
    assert out.value is None
    assert "NULL" in lg.lg_last_error()
    assert lib.lg_stats_get(None, None) == 1
    lib.lg_free(None)  # NULL-safe
