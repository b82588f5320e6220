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


# C field names of every struct the binding mirrors, in declaration order
_C_FIELDS = {
    "gm_edge_list": ["n_vertices", "n_edges", "src", "dst", "weight", "weight_type", "on_device", "n_left"],
    "gm_program_params": ["r", "pr_apply_all", "K", "lambda", "gamma", "init_sigma", "seed", "cf_strata"],
    "gm_tuning": ["alpha", "beta", "sssp_pull_frac", "bin_small", "bin_large", "best_ms", "pull_stage"],
    "gm_query": ["graph", "kind", "source", "reserved"],
}


def test_binding_structs_match_the_header_layout(tmp_path):
    """sizeof and every field offset of the header's structs, as the host C
    compiler lays them out, equal those of the ctypes mirrors."""
    import shutil
    import subprocess
    import paper_1503_07241_gb300 as pkg
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "graphmat_gb300.h"', "int main(void) {"]
    for st, fields in _C_FIELDS.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for f in fields:
            lines.append(f'printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True)
    c = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        st, f, v = line.split()
        c[(st, f)] = int(v)
    for st, fields in _C_FIELDS.items():
        cls = getattr(pkg, st)
        assert ctypes.sizeof(cls) == c[(st, "size")], st
        py_fields = [name for name, _ in cls._fields_]
        assert len(py_fields) == len(fields), st
        for cf, pf in zip(fields, py_fields):
            assert getattr(cls, pf).offset == c[(st, cf)], (st, cf)
