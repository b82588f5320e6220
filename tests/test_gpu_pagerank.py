"""PageRank (Eq. 1) on the GPU: FP32 ranks within 1e-5 max relative error per
vertex of the FP64 oracle, both apply readings, ragged and degenerate graphs."""
import json
import os

import numpy as np
import pytest

import oracle
from gpu_util import random_case, rmat_case

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = 1e-5  # max relative error per vertex, FP32 GPU vs FP64 oracle


def _pr(gm, g, iters=20, r=0.15, apply_all=True):
    g.program_set(gm.GM_PAGERANK, r=r, pr_apply_all=apply_all)
    assert g.run(iters) == iters
    return g.state().astype(np.float64)


def _relerr(a, b):
    return np.max(np.abs(a - b) / np.abs(b)) if b.size else 0.0


def test_scale16_config(gm):
    n, s, d, _ = rmat_case(16)
    g = gm.Graph(n, s, d)
    og = oracle.Graph(n, s, d)
    ref, _ = og.pagerank(0.15, 20)
    for loop_mode in (0, 1):
        g.set_option(gm.GM_OPT_LOOP_MODE, loop_mode)
        assert _relerr(_pr(gm, g), ref) <= TOL


@pytest.mark.parametrize("apply_all", [True, False])
@pytest.mark.parametrize("seed", range(3))
def test_random_graphs(gm, seed, apply_all):
    rng = np.random.default_rng(2000 + seed)
    n, s, d, _ = random_case(rng, int(rng.integers(1, 4000)), int(rng.integers(0, 60000)))
    g = gm.Graph(n, s, d)
    og = oracle.Graph(n, s, d)
    for iters in (1, 7, 20):
        ref, _ = og.pagerank(0.15, iters, apply_all_vertices=apply_all)
        assert _relerr(_pr(gm, g, iters, apply_all=apply_all), ref) <= TOL


def test_bins_and_hub(gm):
    # a hub with a huge in-degree exercises the CTA-per-vertex bin
    n = 50000
    rng = np.random.default_rng(3)
    s = np.concatenate([np.arange(1, n), rng.integers(0, n, 200000)]).astype(np.int32)
    d = np.concatenate([np.zeros(n - 1), rng.integers(0, n, 200000)]).astype(np.int32)
    g = gm.Graph(n, s, d)
    og = oracle.Graph(n, s, d)
    ref, _ = og.pagerank(0.15, 20)
    for small, large in [(32, 2048), (4, 16), (2, 1 << 20)]:
        g.set_option(gm.GM_OPT_BIN_LARGE, 1 << 30)
        g.set_option(gm.GM_OPT_BIN_SMALL, small)
        g.set_option(gm.GM_OPT_BIN_LARGE, large)
        assert _relerr(_pr(gm, g), ref) <= TOL


def test_golden_and_edge_cases(gm):
    gd = json.load(open(os.path.join(GOLDEN, "pagerank_tiny.json")))
    g = gm.Graph(gd["n"], np.array(gd["src"], np.int32), np.array(gd["dst"], np.int32))
    np.testing.assert_allclose(_pr(gm, g, gd["iters"], gd["r"], True), gd["rank_eq1_all_vertices"], rtol=1e-6)
    np.testing.assert_allclose(_pr(gm, g, gd["iters"], gd["r"], False), gd["rank_alg2_received_only"], rtol=1e-6)
    # zero iterations keep the initial ranks; max_iters = -1 is rejected
    assert np.all(_pr(gm, g, 0) == 1.0)
    with pytest.raises(gm.GMError):
        g.run(-1)
    # regular digraph: ranks stay 1
    n, k = 1000, 7
    src = np.repeat(np.arange(n), k).astype(np.int32)
    dst = ((src + np.tile(np.arange(1, k + 1), n)) % n).astype(np.int32)
    g = gm.Graph(n, src, dst)
    assert np.max(np.abs(_pr(gm, g) - 1.0)) <= 1e-6
    # edgeless graph: every rank is r
    g = gm.Graph(10, np.zeros(0, np.int32), np.zeros(0, np.int32))
    np.testing.assert_allclose(_pr(gm, g), 0.15, rtol=1e-7)
