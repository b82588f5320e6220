"""Triangle counting on the GPU: per-vertex incident counts (uint64) and the
total, bit-exact against the oracle's two vertex programs."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import CLEAN, random_case

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TC_FLAGS = CLEAN | oracle.SYMMETRIZE | oracle.ORIENT_BY_DEGREE


def _tc(gm, n, s, d):
    g = gm.Graph(n, s, d, flags=TC_FLAGS)
    g.program_set(gm.GM_TRIANGLE_COUNT)
    assert g.run() == 2
    return g.state(), g.scalar(gm.GM_SCALAR_TC_TOTAL)


def _check(gm, n, s, d):
    pv, tot = _tc(gm, n, s, d)
    opv, otot = oracle.Graph(n, s, d, flags=TC_FLAGS).triangle_count()
    assert tot == otot
    assert np.array_equal(pv, opv)
    assert int(pv.sum()) == 3 * tot


def test_golden(gm):
    gd = json.load(open(os.path.join(GOLDEN, "triangles_tiny.json")))
    pv, tot = _tc(gm, gd["n"], np.array(gd["src"], np.int32), np.array(gd["dst"], np.int32))
    assert tot == gd["total"] and pv.tolist() == gd["per_vertex_incident"]


@pytest.mark.parametrize("seed", range(4))
def test_random_graphs(gm, seed):
    rng = np.random.default_rng(3000 + seed)
    n, s, d, _ = random_case(rng, int(rng.integers(3, 3000)), int(rng.integers(0, 40000)))
    _check(gm, n, s, d)


@pytest.mark.parametrize("k", [3, 5, 40, 150])
def test_complete_graph(gm, k):
    pairs = np.array([(a, b) for a in range(k) for b in range(k) if a < b], np.int32)
    pv, tot = _tc(gm, k, np.ascontiguousarray(pairs[:, 0]), np.ascontiguousarray(pairs[:, 1]))
    assert tot == math.comb(k, 3) and np.all(pv == math.comb(k - 1, 2))


def test_bipartite_and_empty(gm):
    rng = np.random.default_rng(4)
    s = rng.integers(0, 100, 2000).astype(np.int32)
    d = rng.integers(100, 300, 2000).astype(np.int32)
    pv, tot = _tc(gm, 300, s, d)
    assert tot == 0 and not pv.any()
    pv, tot = _tc(gm, 5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert tot == 0


def test_rmat_scale16(gm):
    n, s, d = synth.rmat(16, 16, synth.RMAT_PARAMS["triangle"])
    _check(gm, n, s, d)


@pytest.mark.slow
def test_rmat_scale20_config(gm):
    """The triangle-counting workload: symmetrised RMAT scale 20 (a/b/c = .45/.15/.15),
    edge factor 16, oriented low-to-high degree; every per-vertex count and the total."""
    n, s, d = synth.rmat(20, 16, synth.RMAT_PARAMS["triangle"])
    _check(gm, n, s, d)
