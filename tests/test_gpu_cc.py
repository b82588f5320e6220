"""Connected components by label propagation, written with the user-program API
(graphmat_program.cuh), against the FP64 oracle: bit-exact labels and equal
superstep counts on symmetrised and directed graphs."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from gpu_util import CLEAN, random_case, rmat_case

pytestmark = pytest.mark.gpu


def _cc(gm, g, max_iters=-1):
    g.program_set(gm.GM_CONNECTED_COMPONENTS)
    it = g.run(max_iters)
    return g.state(), it


@pytest.mark.parametrize("sym", [True, False])
@pytest.mark.parametrize("seed", range(3))
def test_random_graphs(gm, seed, sym):
    rng = np.random.default_rng(700 + seed)
    n, s, d, _ = random_case(rng, int(rng.integers(2, 6000)), int(rng.integers(0, 30000)))
    flags = CLEAN | (oracle.SYMMETRIZE if sym else 0)
    g = gm.Graph(n, s, d, flags=flags)
    got, it = _cc(gm, g)
    ref, rit = oracle.Graph(n, s, d, flags=flags).connected_components()
    assert np.array_equal(got, ref) and it == rit


@pytest.mark.parametrize("scale,sym", [(14, True), (16, False)])
def test_rmat(gm, scale, sym):
    n, s, d, _ = rmat_case(scale, seed=synth.BASE_SEED + 50 + scale)
    flags = CLEAN | (oracle.SYMMETRIZE if sym else 0)
    g = gm.Graph(n, s, d, flags=flags)
    og = oracle.Graph(n, s, d, flags=flags)
    got, it = _cc(gm, g)
    ref, rit = og.connected_components()
    assert np.array_equal(got, ref) and it == rit
    for k in (1, 2, 3):  # truncated runs end in the same state as the oracle's
        got, it = _cc(gm, g, max_iters=k)
        ref, rit = og.connected_components(max_iters=k)
        assert np.array_equal(got, ref) and it == rit


def test_bins_do_not_change_labels(gm):
    n, s, d, _ = rmat_case(13, seed=synth.BASE_SEED + 60)
    g = gm.Graph(n, s, d, flags=CLEAN | oracle.SYMMETRIZE)
    ref, rit = _cc(gm, g)
    g.set_option(gm.GM_OPT_BIN_LARGE, 1 << 30)
    g.set_option(gm.GM_OPT_BIN_SMALL, 1)  # every destination handled by a warp
    got, it = _cc(gm, g)
    assert np.array_equal(got, ref) and it == rit
    g.set_option(gm.GM_OPT_BIN_SMALL, 4096)  # (almost) every destination by a lane
    got, it = _cc(gm, g)
    assert np.array_equal(got, ref) and it == rit


@pytest.mark.parametrize("n", [2, 33, 1000])
def test_path_superstep_count(gm, n):
    s = np.arange(n - 1, dtype=np.int32)
    g = gm.Graph(n, s, s + 1, flags=CLEAN | oracle.SYMMETRIZE)
    lab, it = _cc(gm, g)
    assert lab.tolist() == [0] * n and it == n


def test_device_view(gm):
    n, s, d, w = rmat_case(10, weighted=True)
    g = gm.Graph(n, s, d, w)
    v = (ctypes.c_int64 * 32)()
    assert gm.lib().gm_graph_device_view(g._h, ctypes.byref(v)) == 0
    vals = list(v)
    assert vals[0] == n and vals[1] == g.m
    # pointers are non-zero device addresses; in_off[3] + zero_in_count == n
    assert all(x != 0 for x in vals[2:9])
    in_off3, zero_count = vals[12], vals[14]
    assert in_off3 + zero_count == n
