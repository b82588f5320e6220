"""Helpers shared by the GPU parity tests (inputs come from `synth`, expected
values from `oracle`; nothing here does vertex-program arithmetic)."""
import numpy as np

import oracle
import synth

CLEAN = oracle.DROP_SELF_LOOPS | oracle.DEDUP


def rmat_case(scale, ef=16, params=synth.RMAT_PARAMS["graph500"], seed=synth.BASE_SEED, weighted=False):
    n, s, d = synth.rmat(scale, ef, params, seed)
    w = synth.edge_weights_u32(s, d, seed + 1) if weighted else None
    return n, s, d, w


def random_case(rng, n, m, weighted=False, lo=1, hi=255):
    s = rng.integers(0, max(n, 1), m).astype(np.int32)
    d = rng.integers(0, max(n, 1), m).astype(np.int32)
    w = rng.integers(lo, hi + 1, m).astype(np.uint32) if weighted else None
    return n, s, d, w


def check_sssp_certificate(n, src, dst, w, dist, sources):
    """Distances are exact shortest paths iff sources are 0, every edge is
    relaxed (dist[v] <= dist[u] + w) and every other reached vertex has a tight
    in-edge; unreached vertices must have no reached in-neighbour."""
    INF = np.uint64(0xFFFFFFFF)
    d64 = dist.astype(np.uint64)
    assert np.all(d64[sources] == 0)
    reached_u = d64[src] != INF
    cand = np.where(reached_u, d64[src] + w.astype(np.uint64), INF)
    cand = np.minimum(cand, INF)
    assert np.all(d64[dst] <= cand), "an edge is not relaxed"
    best = np.full(n, INF, np.uint64)
    np.minimum.at(best, dst, cand)
    best[sources] = 0
    assert np.array_equal(best, d64), "a vertex lacks a tight in-edge"
