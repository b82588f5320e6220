"""Seeded synthetic inputs (RMAT and bipartite Chung-Lu graphs, edge values,
sources, random vectors) for the GraphMat workloads of Section 5.1.

This module holds no vertex-program arithmetic.  It is the one piece shared by
the FP64 oracle and the CUDA library: both take its edge lists as input.  The C
generator is compiled on first use (or by ``build()``) with the host gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

# Seeds: one base seed for every workload, offset by the workload index.
BASE_SEED = 20150325

RMAT_PARAMS = {  # (a, b, c); d = 1 - a - b - c  (Section 5.1)
    "graph500": (0.57, 0.19, 0.19),
    "triangle": (0.45, 0.15, 0.15),
    "sssp24": (0.50, 0.10, 0.10),
}


def build(force: bool = False) -> str:
    """Compile gen.c into libsynth.so (idempotent)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
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
    i64, u64, i32, u32, f64, f32 = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32,
                                    ctypes.c_uint32, ctypes.c_double, ctypes.c_float)
    lib.sy_rmat.argtypes = [i32, i64, f64, f64, f64, u64, P, P]
    lib.sy_rmat.restype = None
    lib.sy_edge_weights_u32.argtypes = [i64, P, P, u64, u32, u32, P]
    lib.sy_edge_weights_u32.restype = None
    lib.sy_uniform_f32.argtypes = [i64, u64, u64, f32, f32, P]
    lib.sy_uniform_f32.restype = None
    lib.sy_uniform_int.argtypes = [i64, u64, u64, i64, i64, P]
    lib.sy_uniform_int.restype = None
    lib.sy_pick_sources.argtypes = [i64, i64, P, P, i64, u64, i64, P]
    lib.sy_pick_sources.restype = i64
    lib.sy_chung_lu_bipartite.argtypes = [i64, i64, f64, f64, u64, P, P, P, i64]
    lib.sy_chung_lu_bipartite.restype = i64
    lib.sy_chung_lu_expected.argtypes = [i64, i64, f64, f64]
    lib.sy_chung_lu_expected.restype = f64
    lib.sy_draw_u64.argtypes = [u64, u64, u64]
    lib.sy_draw_u64.restype = u64
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def rmat(scale: int, edge_factor: int = 16, params=RMAT_PARAMS["graph500"], seed: int = BASE_SEED):
    """Raw RMAT edge list (int32 src, dst): n = 2**scale, m = edge_factor * n,
    self-loops and duplicates included."""
    lib = _load()
    n = 1 << scale
    m = edge_factor * n
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    a, b, c = params
    lib.sy_rmat(scale, m, a, b, c, seed, _p(src), _p(dst))
    return n, src, dst


def edge_weights_u32(src: np.ndarray, dst: np.ndarray, seed: int, lo: int = 1, hi: int = 255):
    """uint32 weight per edge, uniform in [lo, hi], a function of (seed, src, dst)."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    w = np.empty(src.shape[0], dtype=np.uint32)
    lib.sy_edge_weights_u32(src.shape[0], _p(src), _p(dst), seed, lo, hi, _p(w))
    return w


def uniform_f32(count: int, seed: int, stream: int, lo: float, hi: float):
    lib = _load()
    out = np.empty(count, dtype=np.float32)
    lib.sy_uniform_f32(count, seed, stream, lo, hi, _p(out))
    return out


def uniform_int(count: int, seed: int, stream: int, lo: int, hi: int):
    lib = _load()
    out = np.empty(count, dtype=np.int64)
    lib.sy_uniform_int(count, seed, stream, lo, hi, _p(out))
    return out


def pick_sources(n: int, src: np.ndarray, dst: np.ndarray, count: int, seed: int,
                 max_draws: int = 1 << 26):
    """`count` distinct vertices with an out-edge that is not a self-loop."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    out = np.empty(max(count, 1), dtype=np.int32)
    k = lib.sy_pick_sources(n, src.shape[0], _p(src), _p(dst), count, seed, max_draws, _p(out))
    if k < 0:
        raise MemoryError("sy_pick_sources: allocation failed")
    return out[:k].copy()


def chung_lu_expected(n_users: int, n_items: int, alpha: float, c: float) -> float:
    return _load().sy_chung_lu_expected(n_users, n_items, alpha, c)


def chung_lu_calibrate(n_users: int, n_items: int, alpha: float, target_edges: float) -> float:
    """Scale constant c with expected edge count == target (bisection in log c)."""
    lo, hi = 1e-6, 1e12
    for _ in range(200):
        mid = (lo * hi) ** 0.5
        if chung_lu_expected(n_users, n_items, alpha, mid) < target_edges:
            lo = mid
        else:
            hi = mid
        if hi / lo < 1 + 1e-12:
            break
    return (lo * hi) ** 0.5


def chung_lu_bipartite(n_users: int, n_items: int, alpha: float, target_edges: float,
                       seed: int):
    """Bipartite rating graph: (n, src users, dst items offset by n_users,
    uint32 ratings in 1..5).  Zipf(alpha)-shaped degrees on both sides."""
    lib = _load()
    c = chung_lu_calibrate(n_users, n_items, alpha, target_edges)
    cnt = lib.sy_chung_lu_bipartite(n_users, n_items, alpha, c, seed, None, None, None, 0)
    src = np.empty(cnt, dtype=np.int32)
    dst = np.empty(cnt, dtype=np.int32)
    rat = np.empty(cnt, dtype=np.uint32)
    cnt2 = lib.sy_chung_lu_bipartite(n_users, n_items, alpha, c, seed, _p(src), _p(dst), _p(rat), cnt)
    assert cnt2 == cnt
    return n_users + n_items, src, dst, rat


def draw_u64(seed: int, stream: int, counter: int) -> int:
    return int(_load().sy_draw_u64(seed, stream, counter))
