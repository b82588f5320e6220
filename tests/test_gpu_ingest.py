"""GPU ingest (CSR/CSC build, cleaning, degrees) against the oracle's cleaning."""
import numpy as np
import pytest

import oracle
from gpu_util import CLEAN, random_case, rmat_case

pytestmark = pytest.mark.gpu


def _compare(gm, n, s, d, w, flags):
    g = gm.Graph(n, s, d, w, flags=flags)
    og = oracle.Graph(n, s, d, w, flags=flags)
    assert g.m == og.m
    gs, gd = g.edges()
    os_, od, ov = og.edges()
    assert np.array_equal(gs, os_) and np.array_equal(gd, od)
    if w is not None:
        assert np.array_equal(g.edge_values().astype(np.float64), ov)
    out_deg, in_deg = g.degrees()
    o_out, o_in = og.degrees()
    assert np.array_equal(out_deg, o_out) and np.array_equal(in_deg, o_in)
    g.close()


@pytest.mark.parametrize("seed", range(4))
def test_ingest_random_with_dups_and_loops(gm, seed):
    rng = np.random.default_rng(seed)
    n, s, d, w = random_case(rng, int(rng.integers(1, 3000)), int(rng.integers(0, 20000)), weighted=True)
    _compare(gm, n, s, d, w, CLEAN)


@pytest.mark.parametrize("flags", [0, oracle.DEDUP, oracle.DROP_SELF_LOOPS, CLEAN | oracle.SYMMETRIZE,
                                   CLEAN | oracle.SYMMETRIZE | oracle.ORIENT_BY_DEGREE])
def test_ingest_flags(gm, flags):
    rng = np.random.default_rng(7)
    n, s, d, w = random_case(rng, 500, 6000, weighted=True)
    _compare(gm, n, s, d, w, flags)


def test_ingest_rmat_scale16(gm):
    n, s, d, w = rmat_case(16, weighted=True)
    _compare(gm, n, s, d, w, CLEAN)


def test_ingest_device_inputs(gm):
    import torch
    n, s, d, w = rmat_case(12, weighted=True)
    ts, td = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    tw = torch.from_numpy(w.view(np.int32)).cuda()
    g = gm.Graph(n, ts, td, tw)
    og = oracle.Graph(n, s, d, w)
    gs, gd = g.edges()
    os_, od, ov = og.edges()
    assert np.array_equal(gs, os_) and np.array_equal(gd, od)
    assert np.array_equal(g.edge_values().astype(np.float64), ov)


def test_ingest_empty_and_tiny(gm):
    g = gm.Graph(0, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.n == 0 and g.m == 0
    g = gm.Graph(1, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.m == 0
    g = gm.Graph(1, np.zeros(3, np.int32), np.zeros(3, np.int32))  # only self-loops
    assert g.m == 0


def test_ingest_rejects_bad_ids(gm):
    with pytest.raises(gm.GMError) as ei:
        gm.Graph(4, np.array([0, 4], np.int32), np.array([1, 2], np.int32))
    assert ei.value.status == gm.GM_ERR_INVALID_ARG
    with pytest.raises(gm.GMError):
        gm.Graph(4, np.array([0, -1], np.int32), np.array([1, 2], np.int32))
