"""FP64 CPU oracle for the GraphMat vertex programs -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it, and the
two share no code: the oracle is plain serial C (``graphmat_oracle.c``) compiled
with the host gcc, wrapped here with ctypes and numpy.  For timing on all host
cores, PageRank, BFS and SSSP can also run on OpenMP threads (``threads=``
argument; PageRank as a pull in the serial Reduce order, BFS and SSSP as a push
with an atomic minimum), which gives identical results.

Every function follows a passage of the paper (Sundaram et al., VLDB 2015):
Algorithm 1 (generalized SPMV) inside Algorithm 2 (Run_Graph_Program) for
PageRank (Eq. 1), BFS (Section 3.II) and SSSP (Section 3.V, appendix program);
the two triangle-counting programs of Section 4.2; Eqs. 3-5 for collaborative
filtering (gradient descent, and stochastic gradient descent in a stratified
order); and weighted PageRank with its reverse-mode gradient (an added form
with no counterpart in the paper; pinned by finite differences in the tests).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphmat_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DROP_SELF_LOOPS, DEDUP, SYMMETRIZE, ORIENT_BY_DEGREE = 1, 2, 4, 8
INF_U32 = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (idempotent)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
        try:  # OpenMP for the multi-threaded pull engine; without it that engine runs one thread
            subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    i64, i32, u32, u64, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
    sig = {
        "or_graph_create": ([i64, i64, P, P, P, i32, u32], P),
        "or_graph_destroy": ([P], None),
        "or_graph_m": ([P], i64),
        "or_graph_n": ([P], i64),
        "or_graph_edges": ([P, P, P, P], None),
        "or_graph_degrees": ([P, P, P], None),
        "or_pagerank": ([P, f64, i64, i32, P], i64),
        "or_pagerank_threads": ([P, f64, i64, i32, P, i32], i64),
        "or_bfs": ([P, P, i64, i64, P], i64),
        "or_bfs_threads": ([P, P, i64, i64, P, i32], i64),
        "or_sssp_threads": ([P, P, i64, i64, P, i32], i64),
        "or_openmp": ([], i32),
        "or_connected_components": ([P, i64, P], i64),
        "or_sssp": ([P, P, i64, i64, P], i64),
        "or_reached_edges": ([P, P], i64),
        "or_triangle_count": ([P, P, P], i64),
        "or_normal_draw": ([u64, u64, f64], f64),
        "or_cf_init": ([u64, i64, f64, P], None),
        "or_cf_loss": ([P, i32, f64, P], f64),
        "or_cf_gd": ([P, i32, f64, f64, i64, P, P], i64),
        "or_cf_vertex_step": ([P, i32, f64, f64, P, i64, P], None),
        "or_cf_sgd": ([P, i64, i32, f64, f64, i64, i64, P], i64),
        "or_wpr_forward": ([P, P, f64, i64, P, P], f64),
        "or_wpr_gradient": ([P, P, f64, i64, P, P], f64),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Graph:
    """Cleaned graph held by the oracle (edges sorted by (src, dst))."""

    def __init__(self, n, src, dst, weight=None, flags=DROP_SELF_LOOPS | DEDUP):
        lib = _load()
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        wtype = 0
        if weight is not None:
            weight = np.ascontiguousarray(weight)
            if weight.dtype == np.uint32:
                wtype = 1
            elif weight.dtype == np.float32:
                wtype = 2
            else:
                raise TypeError("weights must be uint32 or float32")
        self._keep = (src, dst, weight)
        h = lib.or_graph_create(n, src.shape[0], _p(src), _p(dst), _p(weight), wtype, flags)
        if not h:
            raise ValueError("oracle: invalid edge list (vertex id out of range) or out of memory")
        self._h = ctypes.c_void_p(h)
        self.n = int(lib.or_graph_n(self._h))
        self.m = int(lib.or_graph_m(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.or_graph_destroy(h)
            self._h = None

    def edges(self):
        s = np.empty(self.m, np.int32)
        d = np.empty(self.m, np.int32)
        v = np.empty(self.m, np.float64)
        _load().or_graph_edges(self._h, _p(s), _p(d), _p(v))
        return s, d, v

    def degrees(self):
        o = np.empty(self.n, np.int64)
        i = np.empty(self.n, np.int64)
        _load().or_graph_degrees(self._h, _p(o), _p(i))
        return o, i

    # -- vertex programs -------------------------------------------------
    # threads=0: the serial engine (Algorithm 1 as a push in source order);
    # threads>=1: a threaded engine on that many OpenMP threads (same results).
    def pagerank(self, r=0.15, iters=20, apply_all_vertices=True, threads=0):
        x = np.empty(self.n, np.float64)
        a = 1 if apply_all_vertices else 0
        lib = _load()
        it = (lib.or_pagerank_threads(self._h, r, iters, a, _p(x), threads) if threads > 0
              else lib.or_pagerank(self._h, r, iters, a, _p(x)))
        return x, int(it)

    def bfs(self, sources, max_iters=-1, threads=0):
        s = np.ascontiguousarray(np.atleast_1d(sources), dtype=np.int32)
        d = np.empty(self.n, np.uint32)
        lib = _load()
        it = (lib.or_bfs_threads(self._h, _p(s), s.shape[0], max_iters, _p(d), threads) if threads > 0
              else lib.or_bfs(self._h, _p(s), s.shape[0], max_iters, _p(d)))
        return d, int(it)

    def connected_components(self, max_iters=-1):
        """Label propagation: (uint32 labels, supersteps)."""
        lab = np.empty(self.n, np.uint32)
        it = _load().or_connected_components(self._h, max_iters, _p(lab))
        return lab, int(it)

    def sssp(self, sources, max_iters=-1, threads=0):
        s = np.ascontiguousarray(np.atleast_1d(sources), dtype=np.int32)
        d = np.empty(self.n, np.uint32)
        lib = _load()
        it = (lib.or_sssp_threads(self._h, _p(s), s.shape[0], max_iters, _p(d), threads) if threads > 0
              else lib.or_sssp(self._h, _p(s), s.shape[0], max_iters, _p(d)))
        return d, int(it)

    def reached_edges(self, dist):
        dist = np.ascontiguousarray(dist, dtype=np.uint32)
        return int(_load().or_reached_edges(self._h, _p(dist)))

    def triangle_count(self):
        pv = np.empty(self.n, np.uint64)
        tot = np.zeros(1, np.uint64)
        _load().or_triangle_count(self._h, _p(pv), _p(tot))
        return pv, int(tot[0])

    def cf_gd(self, K, lam, gamma, iters, p0):
        p = np.array(p0, dtype=np.float64, copy=True).reshape(self.n, K)
        trace = np.empty(iters + 1, np.float64)
        _load().or_cf_gd(self._h, K, lam, gamma, iters, _p(p), _p(trace))
        return p, trace

    def cf_sgd(self, K, lam, gamma, epochs, n_left, P, p0):
        """Stochastic gradient descent (Section 3.III) for `epochs` epochs in the
        stratified order of P blocks (see or_cf_sgd); returns the factors."""
        p = np.array(p0, dtype=np.float64, copy=True).reshape(self.n, K)
        if _load().or_cf_sgd(self._h, n_left, K, lam, gamma, epochs, P, _p(p)) < 0:
            raise ValueError("or_cf_sgd: bad argument")
        return p

    def cf_vertex_step(self, K, lam, gamma, p, v):
        p = np.ascontiguousarray(p, dtype=np.float64)
        out = np.empty(K, np.float64)
        _load().or_cf_vertex_step(self._h, K, lam, gamma, _p(p), v, _p(out))
        return out

    def cf_loss(self, K, lam, p):
        p = np.ascontiguousarray(p, dtype=np.float64)
        return float(_load().or_cf_loss(self._h, K, lam, _p(p)))

    def wpr_forward(self, w, tau, r=0.15, steps=30):
        w = np.ascontiguousarray(w, dtype=np.float64)
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        x = np.empty(self.n, np.float64)
        loss = _load().or_wpr_forward(self._h, _p(w), r, steps, _p(tau), _p(x))
        return x, float(loss)

    def wpr_gradient(self, w, tau, r=0.15, steps=30):
        w = np.ascontiguousarray(w, dtype=np.float64)
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        g = np.empty(self.m, np.float64)
        loss = _load().or_wpr_gradient(self._h, _p(w), r, steps, _p(tau), _p(g))
        return g, float(loss)


def cf_init(n, K, seed, sigma=0.1):
    """Initial CF factors N(0, sigma) from the counter-based draw (SplitMix64 +
    Box-Muller), row-major n x K."""
    out = np.empty(n * K, np.float64)
    _load().or_cf_init(seed, n * K, sigma, _p(out))
    return out.reshape(n, K)


def openmp() -> bool:
    """Whether the oracle's threaded engines were built with OpenMP."""
    return bool(_load().or_openmp())
