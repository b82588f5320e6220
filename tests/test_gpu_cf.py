"""Collaborative filtering (Eqs. 2-5) on the GPU against the FP64 oracle: the
counter-based initial factors, factors after 10 gradient steps within 1e-4
relative, the Eq. 2 loss, and one step on sampled vertices of the full
480,000 x 17,800 / 100M-rating workload."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
LAM = 0.05


def _graph(gm, nu, ni, nr, seed=7):
    n, s, d, r = synth.chung_lu_bipartite(nu, ni, 1.1, nr, seed=seed)
    return n, s, d, r, gm.Graph(n, s, d, r, n_left=nu), oracle.Graph(n, s, d, r)


def _rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_initial_factors_match_generator(gm):
    n, s, d, r, g, og = _graph(gm, 300, 40, 3000)
    for K in (1, 8, 32, 48):
        g.program_set(gm.GM_CF, K=K, lam=LAM, gamma=1e-3, init_sigma=0.1, seed=11)
        np.testing.assert_allclose(g.state(), oracle.cf_init(n, K, 11, 0.1), rtol=0, atol=1e-7)


@pytest.mark.parametrize("K", [4, 32, 64])
def test_ten_steps_match_oracle(gm, K):
    n, s, d, r, g, og = _graph(gm, 3000, 400, 60000)
    gamma = 1e-3
    g.program_set(gm.GM_CF, K=K, lam=LAM, gamma=gamma, init_sigma=0.1, seed=3)
    p0 = g.state().astype(np.float64)
    ref, trace = og.cf_gd(K, LAM, gamma, 10, p0)
    assert np.all(np.diff(trace) < 0), "step size chosen so the loss decreases"
    assert g.run(10) == 10
    got = g.state().astype(np.float64)
    assert _rel_fro(got, ref) <= 1e-4
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))
    assert abs(g.scalar(gm.GM_SCALAR_CF_LOSS) - trace[-1]) <= 1e-5 * trace[-1]


def test_set_state_and_zero_steps(gm):
    n, s, d, r, g, og = _graph(gm, 500, 60, 5000)
    g.program_set(gm.GM_CF, K=16, lam=LAM, gamma=1e-3, seed=1)
    p = (np.arange(n * 16, dtype=np.float32).reshape(n, 16) % 7) * 0.01
    g.set_state(p)
    assert g.run(0) == 0
    assert np.array_equal(g.state(), p)
    assert abs(g.scalar(gm.GM_SCALAR_CF_LOSS) - og.cf_loss(16, LAM, p.astype(np.float64))) <= 1e-5 * og.cf_loss(
        16, LAM, p.astype(np.float64))


def test_rejects_non_bipartite(gm):
    g = gm.Graph(10, np.array([0, 1], np.int32), np.array([1, 2], np.int32), np.array([3, 4], np.uint32))
    with pytest.raises(gm.GMError):
        g.program_set(gm.GM_CF, K=8)


@pytest.mark.slow
def test_full_config_one_step_on_sampled_vertices(gm):
    """480,000 users x 17,800 items, ~100M ratings, K = 32, lambda 0.05, gamma 1e-3:
    after one step, 8 sampled users and 4 sampled items equal the FP64 update of
    Eqs. 3-5 computed from the same initial factors."""
    nu, ni = 480_000, 17_800
    n, s, d, r = synth.chung_lu_bipartite(nu, ni, 1.1, 1e8, seed=synth.BASE_SEED + 2)
    g = gm.Graph(n, s, d, r, n_left=nu)
    og = oracle.Graph(n, s, d, r)
    K, gamma = 32, 1e-3
    g.program_set(gm.GM_CF, K=K, lam=LAM, gamma=gamma, init_sigma=0.1, seed=5)
    p0 = g.state().astype(np.float64)
    g.run(1)
    p1 = g.state().astype(np.float64)
    rng = np.random.default_rng(1)
    for v in list(rng.choice(nu, 8, replace=False)) + list(nu + rng.choice(ni, 4, replace=False)):
        ref = og.cf_vertex_step(K, LAM, gamma, p0, int(v))
        assert np.max(np.abs(p1[v] - ref)) <= 1e-4 * max(np.max(np.abs(ref)), 1e-3)
