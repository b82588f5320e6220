"""C ABI checks that need no GPU: the library loads, exports every entry point
that include/graphmat_gb300.h declares, and rejects bad arguments on the host."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if fn.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, fn)).read()
            names |= set(re.findall(r"^GM_API\s+[\w\s\*]+?\b(gm_\w+)\s*\(", text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as ge
    ge.build_cuda_library()
    import paper_1503_07241_gb300 as pkg
    return pkg.lib()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("gm_graph_create", "gm_program_set", "gm_set_active", "gm_run", "gm_get_vertex_state"):
        assert n in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_python_binding_covers_every_entry_point():
    import paper_1503_07241_gb300 as pkg
    assert _declared() <= set(pkg.SIGNATURES)


def test_status_strings(L):
    assert L.gm_status_string(0) == b"GM_OK"
    assert L.gm_status_string(4) == b"GM_ERR_STATE"


def test_null_arguments_rejected_without_gpu(L):
    import paper_1503_07241_gb300 as pkg
    out = ctypes.c_void_p(123)
    assert L.gm_graph_create(None, 0, None, ctypes.byref(out)) == pkg.GM_ERR_INVALID_ARG
    assert out.value is None
    assert b"NULL" in L.gm_last_error()
    assert L.gm_run(None, -1, None) == pkg.GM_ERR_INVALID_ARG
    assert L.gm_program_set(None, 0, None) == pkg.GM_ERR_INVALID_ARG
    assert L.gm_graph_destroy(None) == pkg.GM_OK
    el = pkg.gm_edge_list(-1, 0, None, None, None, 0, 0, 0)
    assert L.gm_graph_create(ctypes.byref(el), 0, None, ctypes.byref(out)) == pkg.GM_ERR_INVALID_ARG
    el = pkg.gm_edge_list(10, 5, None, None, None, 0, 0, 0)  # NULL src with edges
    assert L.gm_graph_create(ctypes.byref(el), 0, None, ctypes.byref(out)) == pkg.GM_ERR_INVALID_ARG
    el = pkg.gm_edge_list(10, 0, None, None, None, 0, 0, 0)
    assert L.gm_graph_create(ctypes.byref(el), 1 << 10, None, ctypes.byref(out)) == pkg.GM_ERR_INVALID_ARG
