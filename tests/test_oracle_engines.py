"""The oracle's serial engine for Algorithm 2 (a push over the sorted edges) and
its threaded engines (used to time the oracle on every host core: PageRank as a
pull in the same per-destination Reduce order, BFS and SSSP as a push whose
Reduce, an exact minimum, is applied atomically) give identical results: every
property (bit for bit, FP64 PageRank included) and every superstep count."""
import numpy as np
import pytest

import oracle
import synth


def _graphs():
    out = []
    for i, (n, m) in enumerate([(1, 0), (5, 4), (300, 2000), (2000, 30000)]):
        rng = np.random.default_rng(synth.BASE_SEED + 600 + i)
        s = rng.integers(0, n, m).astype(np.int32)
        d = rng.integers(0, n, m).astype(np.int32)
        w = rng.integers(1, 256, m).astype(np.uint32)
        out.append((n, s, d, w))
    n, s, d = synth.rmat(12, 16, synth.RMAT_PARAMS["graph500"], synth.BASE_SEED + 610)
    out.append((n, s, d, synth.edge_weights_u32(s, d, synth.BASE_SEED + 611)))
    return out


@pytest.mark.parametrize("threads", [1, 4])
def test_pull_engine_equals_serial(threads):
    for n, s, d, w in _graphs():
        for flags in (oracle.DROP_SELF_LOOPS | oracle.DEDUP, 0):
            g = oracle.Graph(n, s, d, w, flags=flags)
            srcs = [0, n // 2, n - 1]
            for max_iters in (-1, 1, 3):
                for one in ([srcs[0]], srcs):
                    a = g.bfs(one, max_iters)
                    b = g.bfs(one, max_iters, threads=threads)
                    assert np.array_equal(a[0], b[0]) and a[1] == b[1]
                    a = g.sssp(one, max_iters)
                    b = g.sssp(one, max_iters, threads=threads)
                    assert np.array_equal(a[0], b[0]) and a[1] == b[1]
            for apply_all in (True, False):
                a = g.pagerank(0.15, 7, apply_all)
                b = g.pagerank(0.15, 7, apply_all, threads=threads)
                assert np.array_equal(a[0], b[0]) and a[1] == b[1]
