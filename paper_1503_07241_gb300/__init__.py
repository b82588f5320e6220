"""Python binding of the GraphMat GB300 C ABI (``include/graphmat_gb300.h``).

Argument marshalling only: every superstep runs in the CUDA kernels of
``libgraphmat_gb300.so``.  Host arrays are numpy arrays; device arrays are CUDA
torch tensors (PyTorch supplies device memory and streams).  Importing this
package raises if the library has not been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgraphmat_gb300.so")

GM_OK, GM_ERR_INVALID_ARG, GM_ERR_OUT_OF_MEMORY, GM_ERR_CUDA, GM_ERR_STATE, GM_ERR_TIMEOUT, \
    GM_ERR_UNSUPPORTED = range(7)
GM_W_NONE, GM_W_U32, GM_W_F32 = 0, 1, 2
GM_DROP_SELF_LOOPS, GM_DEDUP, GM_SYMMETRIZE, GM_ORIENT_BY_DEGREE = 1, 2, 4, 8
GM_PAGERANK, GM_BFS, GM_SSSP, GM_TRIANGLE_COUNT, GM_CF, GM_CONNECTED_COMPONENTS, GM_CF_SGD = range(7)
(GM_SCALAR_TC_TOTAL, GM_SCALAR_CF_LOSS, GM_SCALAR_REACHED_EDGES, GM_SCALAR_SUPERSTEPS,
 GM_SCALAR_PUSH_STEPS, GM_SCALAR_PULL_STEPS, GM_SCALAR_SCANNED_EDGES, GM_SCALAR_RELAX_MS,
 GM_SCALAR_RELAX_LAUNCHES, GM_SCALAR_PROCESSED_VERTICES, GM_SCALAR_PULL_WEIGHT_BYTES,
 GM_SCALAR_CF_STRATA, GM_SCALAR_PULL_STREAM_BYTES) = range(1, 14)
(GM_OPT_DIRECTION, GM_OPT_LOOP_MODE, GM_OPT_PROFILE, GM_OPT_BIN_SMALL, GM_OPT_BIN_LARGE,
 GM_OPT_ALPHA_X1000, GM_OPT_BETA_X1000, GM_OPT_SSSP_PULL_PPM, GM_OPT_PULL_STAGE,
 GM_OPT_TEST_STALL_STAGE, GM_OPT_TEST_STALL_SGD, GM_OPT_PULL_PACKED, GM_OPT_SPARSE_LIST) = range(1, 14)
INF_U32 = 0xFFFFFFFF
TRACE_COLS = 10  # doubles per row of gm_get_trace

_SCALAR_TYPES = {
    GM_SCALAR_TC_TOTAL: ctypes.c_uint64, GM_SCALAR_CF_LOSS: ctypes.c_double,
    GM_SCALAR_REACHED_EDGES: ctypes.c_int64, GM_SCALAR_SUPERSTEPS: ctypes.c_int32,
    GM_SCALAR_PUSH_STEPS: ctypes.c_int32, GM_SCALAR_PULL_STEPS: ctypes.c_int32,
    GM_SCALAR_SCANNED_EDGES: ctypes.c_int64, GM_SCALAR_RELAX_MS: ctypes.c_double,
    GM_SCALAR_RELAX_LAUNCHES: ctypes.c_int32, GM_SCALAR_PROCESSED_VERTICES: ctypes.c_int64,
    GM_SCALAR_PULL_WEIGHT_BYTES: ctypes.c_int32, GM_SCALAR_CF_STRATA: ctypes.c_int32,
    GM_SCALAR_PULL_STREAM_BYTES: ctypes.c_int64,
}


class GMError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({_status_name(status)}): {detail}")
        self.status = status


class gm_edge_list(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("weight", ctypes.c_void_p),
                ("weight_type", ctypes.c_int32), ("on_device", ctypes.c_int32),
                ("n_left", ctypes.c_int64)]


class gm_program_params(ctypes.Structure):
    _fields_ = [("r", ctypes.c_double), ("pr_apply_all", ctypes.c_int32), ("K", ctypes.c_int32),
                ("lam", ctypes.c_double), ("gamma", ctypes.c_double), ("init_sigma", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("cf_strata", ctypes.c_int32)]


_lib = None
# name: (argtypes, restype)
_P, _I32, _I64, _U32, _U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
SIGNATURES = {
    "gm_graph_create": ([ctypes.POINTER(gm_edge_list), _U32, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "gm_graph_destroy": ([_P], ctypes.c_int),
    "gm_graph_info": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], ctypes.c_int),
    "gm_graph_get_edges": ([_P, _P, _P, _P, ctypes.c_int], ctypes.c_int),
    "gm_graph_get_degrees": ([_P, _P, _P, ctypes.c_int], ctypes.c_int),
    "gm_graph_device_view": ([_P, _P], ctypes.c_int),
    "gm_program_set": ([_P, _I32, ctypes.POINTER(gm_program_params)], ctypes.c_int),
    "gm_set_active": ([_P, _P, _I64, ctypes.c_int], ctypes.c_int),
    "gm_run": ([_P, _I32, ctypes.POINTER(_I32)], ctypes.c_int),
    "gm_get_vertex_state": ([_P, _P, _I64, ctypes.c_int], ctypes.c_int),
    "gm_set_vertex_state": ([_P, _P, _I64, ctypes.c_int], ctypes.c_int),
    "gm_get_scalar": ([_P, _I32, _P], ctypes.c_int),
    "gm_set_option": ([_P, _I32, _I64], ctypes.c_int),
    "gm_get_trace": ([_P, _P, _I32, ctypes.POINTER(_I32)], ctypes.c_int),
    "gm_wpagerank_forward": ([_P, _P, ctypes.c_double, _I32, _I32, _P], ctypes.c_int),
    "gm_wpagerank_backward": ([_P, _P, _P], ctypes.c_int),
    "gm_bfs_csr_noalloc": ([_I64, _P, _P, _I32, _P, ctypes.POINTER(_I32), _P], ctypes.c_int),
    "gm_run_batch": ([_P, _I32, _P, _I32, _P, _I32, _P, _P], ctypes.c_int),
    "gm_autotune": ([_P, _I32, _P, _I32, _P], ctypes.c_int),
    "gm_bfs_csr_noalloc_max_vertices": ([], _I64),
    "gm_kernel_launch_count": ([], _U64),
    "gm_debug_fail_allocations_after": ([_I64], None),
    "gm_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "gm_last_error": ([], ctypes.c_char_p),
}


def lib():
    """Load the CUDA library (raises ImportError if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _status_name(s):
    try:
        return lib().gm_status_string(s).decode()
    except Exception:  # pragma: no cover
        return str(s)


def _check(status, where):
    if status != GM_OK:
        raise GMError(status, where, lib().gm_last_error().decode())


def _ptr(a):
    """(pointer, is_device) of a numpy array or torch tensor; None -> (None, 0)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return a.ctypes.data, 0
    # torch tensor
    if not a.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return a.data_ptr(), 1 if a.is_cuda else 0


def _stream_handle(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


class gm_tuning(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("sssp_pull_frac", ctypes.c_double),
                ("bin_small", ctypes.c_int32), ("bin_large", ctypes.c_int32), ("best_ms", ctypes.c_double),
                ("pull_stage", ctypes.c_int32)]


class gm_query(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_int32), ("kind", ctypes.c_int32), ("source", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


def run_batch(graphs, queries, outs, max_iters=-1, stream=None):
    """Run (graph index, kind, source) queries together (gm_run_batch).  `outs`
    are CUDA uint32/int32 tensors of each query graph's n.  Returns superstep counts."""
    ng, nq = len(graphs), len(queries)
    harr = (ctypes.c_void_p * max(ng, 1))(*[g._h.value for g in graphs])
    qarr = (gm_query * max(nq, 1))(*[gm_query(int(gi), int(k), int(s), 0) for gi, k, s in queries])
    oarr = (ctypes.c_void_p * max(nq, 1))(*[o.data_ptr() for o in outs])
    its = (ctypes.c_int32 * max(nq, 1))()
    _check(lib().gm_run_batch(ctypes.cast(harr, ctypes.c_void_p), ng, ctypes.cast(qarr, ctypes.c_void_p), nq,
                              ctypes.cast(oarr, ctypes.c_void_p), max_iters, ctypes.cast(its, ctypes.c_void_p),
                              _stream_handle(stream)), "gm_run_batch")
    return list(its)[:nq]


def bfs_csr_noalloc(row_ptr, col, source, depth, stream=None) -> int:
    """BFS over device CSR tensors into the device uint32 tensor `depth`, with no
    allocation inside the library (see gm_bfs_csr_noalloc).  Returns supersteps."""
    it = ctypes.c_int32()
    n = int(depth.numel())
    _check(lib().gm_bfs_csr_noalloc(n, row_ptr.data_ptr(), col.data_ptr(), int(source), depth.data_ptr(),
                                    ctypes.byref(it), _stream_handle(stream)), "gm_bfs_csr_noalloc")
    return it.value


def kernel_launch_count() -> int:
    return int(lib().gm_kernel_launch_count())


class Graph:
    """A graph handle: CSR + CSC on the GPU plus one vertex program."""

    def __init__(self, n, src, dst, weight=None, flags=GM_DROP_SELF_LOOPS | GM_DEDUP, stream=None, n_left=0):
        L = lib()
        self._keep = (src, dst, weight)
        sp, sdev = _ptr(src)
        dp, ddev = _ptr(dst)
        wp, wdev = _ptr(weight)
        if sdev != ddev or (weight is not None and wdev != sdev):
            raise ValueError("src, dst and weight must all be host arrays or all device tensors")
        wtype = GM_W_NONE
        if weight is not None:
            dt = str(weight.dtype)
            if dt.endswith("uint32"):
                wtype = GM_W_U32
            elif dt.endswith("float32"):
                wtype = GM_W_F32
            elif dt.endswith("int32"):
                wtype = GM_W_U32  # same 4-byte layout; values must be non-negative
            else:
                raise TypeError(f"unsupported weight dtype {dt}")
        m = int(src.shape[0])
        el = gm_edge_list(n, m, sp, dp, wp, wtype, sdev, n_left)
        h = ctypes.c_void_p()
        _check(L.gm_graph_create(ctypes.byref(el), flags, _stream_handle(stream), ctypes.byref(h)),
               "gm_graph_create")
        self._h = h
        self._keep = None
        nv, ne = ctypes.c_int64(), ctypes.c_int64()
        _check(L.gm_graph_info(h, ctypes.byref(nv), ctypes.byref(ne)), "gm_graph_info")
        self.n, self.m = nv.value, ne.value
        self.kind = None
        self.K = 0

    def close(self):
        if getattr(self, "_h", None):
            lib().gm_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- ingest results --------------------------------------------------
    def edges(self):
        s = np.empty(self.m, np.int32)
        d = np.empty(self.m, np.int32)
        _check(lib().gm_graph_get_edges(self._h, s.ctypes.data, d.ctypes.data, None, 0), "gm_graph_get_edges")
        return s, d

    def edge_values(self):
        w = np.empty(self.m, np.uint32)
        _check(lib().gm_graph_get_edges(self._h, None, None, w.ctypes.data, 0), "gm_graph_get_edges")
        return w

    def degrees(self):
        o = np.empty(self.n, np.int32)
        i = np.empty(self.n, np.int32)
        _check(lib().gm_graph_get_degrees(self._h, o.ctypes.data, i.ctypes.data, 0), "gm_graph_get_degrees")
        return o, i

    # -- programs --------------------------------------------------------
    def program_set(self, kind, r=0.15, pr_apply_all=True, K=32, lam=0.05, gamma=1e-3, init_sigma=0.1, seed=0,
                    cf_strata=0):
        p = gm_program_params(r, 1 if pr_apply_all else 0, K, lam, gamma, init_sigma, seed, cf_strata)
        _check(lib().gm_program_set(self._h, kind, ctypes.byref(p)), "gm_program_set")
        self.kind, self.K = kind, K

    def set_active(self, vertices=None):
        if vertices is None:
            _check(lib().gm_set_active(self._h, None, -1, 0), "gm_set_active")
            return
        if isinstance(vertices, np.ndarray) or not hasattr(vertices, "data_ptr"):
            vertices = np.ascontiguousarray(np.atleast_1d(vertices), dtype=np.int32)
        p, dev = _ptr(vertices)
        _check(lib().gm_set_active(self._h, p, int(vertices.shape[0]), dev), "gm_set_active")

    def run(self, max_iters=-1) -> int:
        it = ctypes.c_int32()
        _check(lib().gm_run(self._h, max_iters, ctypes.byref(it)), "gm_run")
        return it.value

    def _state_spec(self):
        if self.kind in (GM_BFS, GM_SSSP, GM_CONNECTED_COMPONENTS):
            return np.uint32, (self.n,)
        if self.kind == GM_PAGERANK:
            return np.float32, (self.n,)
        if self.kind == GM_TRIANGLE_COUNT:
            return np.uint64, (self.n,)
        if self.kind in (GM_CF, GM_CF_SGD):
            return np.float32, (self.n, self.K)
        raise GMError(GM_ERR_STATE, "state", "no program set")

    def state(self, out=None):
        """Vertex properties; into `out` (numpy or CUDA tensor) if given."""
        dt, shape = self._state_spec()
        if out is None:
            out = np.empty(shape, dt)
        p, dev = _ptr(out)
        nbytes = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
        _check(lib().gm_get_vertex_state(self._h, p, nbytes, dev), "gm_get_vertex_state")
        return out

    def set_state(self, values):
        p, dev = _ptr(values)
        nbytes = values.nbytes if isinstance(values, np.ndarray) else values.numel() * values.element_size()
        _check(lib().gm_set_vertex_state(self._h, p, nbytes, dev), "gm_set_vertex_state")

    def scalar(self, which):
        v = _SCALAR_TYPES[which]()
        _check(lib().gm_get_scalar(self._h, which, ctypes.byref(v)), "gm_get_scalar")
        return v.value

    def trace(self):
        """Per-superstep rows of the last profiled run (see gm_get_trace)."""
        k = ctypes.c_int32()
        _check(lib().gm_get_trace(self._h, None, 0, ctypes.byref(k)), "gm_get_trace")
        rows = np.empty((k.value, TRACE_COLS), np.float64)
        if k.value:
            _check(lib().gm_get_trace(self._h, rows.ctypes.data, k.value, ctypes.byref(k)), "gm_get_trace")
        return rows

    # -- weighted PageRank (device tensors) --------------------------------
    def wpagerank_forward(self, w, r=0.15, steps=30, ckpt_every=5):
        import torch
        x = torch.empty(self.n, dtype=torch.float32, device=w.device)
        _check(lib().gm_wpagerank_forward(self._h, w.data_ptr(), r, steps, ckpt_every, x.data_ptr()),
               "gm_wpagerank_forward")
        return x

    def wpagerank_backward(self, dLdx):
        import torch
        g = torch.empty(self.m, dtype=torch.float32, device=dLdx.device)
        _check(lib().gm_wpagerank_backward(self._h, dLdx.contiguous().data_ptr(), g.data_ptr()),
               "gm_wpagerank_backward")
        return g

    def autotune(self, kind, sources):
        """Tune the traversal knobs on sample host sources (gm_autotune); returns the choice."""
        src = np.ascontiguousarray(np.atleast_1d(sources), dtype=np.int32)
        t = gm_tuning()
        _check(lib().gm_autotune(self._h, kind, src.ctypes.data, src.shape[0], ctypes.byref(t)), "gm_autotune")
        return {f: getattr(t, f) for f, _ in gm_tuning._fields_}

    def set_option(self, option, value):
        _check(lib().gm_set_option(self._h, option, int(value)), "gm_set_option")
