"""Collaborative filtering (Eqs. 2-5) on the GPU against the FP64 oracle: the
counter-based initial factors, factors after 10 gradient steps within 1e-4
relative, the Eq. 2 loss, and one step on sampled vertices of the full
480,000 x 17,800 / 100M-rating workload.  Stochastic gradient descent
(GM_CF_SGD) against the oracle's serial SGD in the same stratified order:
every factor after two epochs, for one-block, several-block and default
strata, K with one and two components per lane, item rows in shared memory
and in L2, and one epoch of the full workload.

SGD tolerance: the kernel computes in FP32 with a different dot-product order;
a sequential FP32 replay of the oracle's order differs from FP64 by at most
3e-6 after two epochs of the 150k-rating case and 1.2e-5 after one epoch of the
100M-rating workload, so every factor must lie within 2e-5 + 1e-4 |oracle|."""
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


SGD_ATOL, SGD_RTOL = 2e-5, 1e-4


def _sgd_case(gm, nu, ni, nr, K, gamma, P, epochs=2, seed=7):
    n, s, d, r, g, og = _graph(gm, nu, ni, nr, seed=seed)
    g.program_set(gm.GM_CF_SGD, K=K, lam=LAM, gamma=gamma, init_sigma=0.1, seed=3, cf_strata=P)
    P_used = g.scalar(gm.GM_SCALAR_CF_STRATA)
    p0 = g.state().astype(np.float64)
    np.testing.assert_allclose(p0, oracle.cf_init(n, K, 3, 0.1), rtol=0, atol=1e-7)
    ref = og.cf_sgd(K, LAM, gamma, epochs, nu, P_used, p0)
    assert g.run(epochs) == epochs
    got = g.state().astype(np.float64)
    np.testing.assert_allclose(got, ref, rtol=SGD_RTOL, atol=SGD_ATOL)
    assert abs(g.scalar(gm.GM_SCALAR_CF_LOSS) - og.cf_loss(K, LAM, ref)) <= 1e-4 * og.cf_loss(K, LAM, ref)
    return P_used, g, og, p0, ref


@pytest.mark.parametrize("K,P", [(32, 1), (32, 8), (32, 0), (5, 3), (48, 16), (64, 64)])
def test_sgd_two_epochs_match_oracle(gm, K, P):
    """Skewed 3000 x 500 ratings (the most-rated items are rated by most users);
    P = 0 takes the default."""
    P_used, *_ = _sgd_case(gm, 3000, 500, 1.5e5, K, 1e-2, P)
    assert P_used == (P if P else P_used) and 1 <= P_used <= 4096


def test_sgd_item_rows_in_l2(gm):
    """20,000 items in 2 blocks: a block's item rows do not fit in shared
    memory, so the warps update them in L2."""
    _sgd_case(gm, 400, 20_000, 6e4, 32, 1e-2, 2)


def test_sgd_more_blocks_than_warps(gm):
    """P = 4096 blocks per stratum is more than the resident warps: warps take
    several blocks of a stratum in turn; most blocks are empty."""
    _sgd_case(gm, 5000, 300, 4e4, 16, 1e-2, 4096, epochs=1)


def test_sgd_default_strata_and_epoch_composition(gm):
    n, s, d, r, g, og = _graph(gm, 2000, 300, 5e4)
    g.program_set(gm.GM_CF_SGD, K=32, lam=LAM, gamma=1e-2, seed=4)
    P = g.scalar(gm.GM_SCALAR_CF_STRATA)
    assert P >= 1 and P & (P - 1) == 0
    assert g.run(0) == 0
    p0 = g.state()
    g.run(1)
    g.run(1)
    two = g.state()
    g.set_state(p0)
    g.run(2)
    np.testing.assert_allclose(g.state(), two, rtol=0, atol=1e-6)


def test_sgd_rejects_bad_inputs(gm):
    # an item -> user rating
    g = gm.Graph(5, np.array([0, 3], np.int32), np.array([3, 1], np.int32), np.array([3, 4], np.uint32), n_left=2)
    with pytest.raises(gm.GMError):
        g.program_set(gm.GM_CF_SGD, K=8)
    g2 = gm.Graph(5, np.array([0, 1], np.int32), np.array([3, 4], np.int32), np.array([3, 4], np.uint32), n_left=2)
    with pytest.raises(gm.GMError):
        g2.program_set(gm.GM_CF_SGD, K=8, cf_strata=4097)
    with pytest.raises(gm.GMError):
        g2.program_set(gm.GM_CF_SGD, K=65)
    g2.program_set(gm.GM_CF, K=8)
    with pytest.raises(gm.GMError):
        g2.scalar(gm.GM_SCALAR_CF_STRATA)


def test_sgd_users_without_ratings_and_tiny_graphs(gm):
    """Users and items without ratings keep their factors; a single rating
    matches the hand-worked update of Section 3.III."""
    g = gm.Graph(4, np.array([1], np.int32), np.array([3], np.int32), np.array([3], np.uint32), n_left=2)
    g.program_set(gm.GM_CF_SGD, K=1, lam=0.5, gamma=0.1, cf_strata=2)
    g.set_state(np.array([[7.0], [1.0], [5.0], [2.0]], np.float32))
    g.run(1)
    # e = 3 - 2 = 1; p_1 = 1 + 0.1 (2 - 0.5) = 1.15; p_3 = 2 + 0.1 (1 - 1) = 2
    np.testing.assert_allclose(g.state().ravel(), [7.0, 1.15, 5.0, 2.0], rtol=1e-6)


@pytest.fixture(scope="module")
def full_cf():
    """The 480,000 x 17,800 / ~100M-rating workload and its oracle graph."""
    nu, ni = 480_000, 17_800
    n, s, d, r = synth.chung_lu_bipartite(nu, ni, 1.1, 1e8, seed=synth.BASE_SEED + 2)
    return nu, ni, n, s, d, r, oracle.Graph(n, s, d, r)


@pytest.mark.slow
def test_sgd_full_config_one_epoch(gm, full_cf):
    """One SGD epoch of the full workload (K = 32, lambda 0.05, gamma 1e-3) in
    the default strata: every factor against the oracle's serial epoch in the
    same order."""
    nu, ni, n, s, d, r, og = full_cf
    g = gm.Graph(n, s, d, r, n_left=nu)
    K, gamma = 32, 1e-3
    g.program_set(gm.GM_CF_SGD, K=K, lam=LAM, gamma=gamma, init_sigma=0.1, seed=5)
    P = g.scalar(gm.GM_SCALAR_CF_STRATA)
    p0 = g.state().astype(np.float64)
    g.run(1)
    got = g.state().astype(np.float64)
    ref = og.cf_sgd(K, LAM, gamma, 1, nu, P, p0)
    excess = np.abs(got - ref) - SGD_RTOL * np.abs(ref)
    print(f"full SGD epoch: max |got - ref| {np.max(np.abs(got - ref)):.3e}, "
          f"max |got - ref| - rtol |ref| {excess.max():.3e} (atol {SGD_ATOL})")
    np.testing.assert_allclose(got, ref, rtol=SGD_RTOL, atol=SGD_ATOL)
    assert og.cf_loss(K, LAM, ref) < og.cf_loss(K, LAM, p0)


@pytest.mark.slow
def test_full_config_one_step_on_sampled_vertices(gm, full_cf):
    """480,000 users x 17,800 items, ~100M ratings, K = 32, lambda 0.05, gamma 1e-3:
    after one step, 8 sampled users and 4 sampled items equal the FP64 update of
    Eqs. 3-5 computed from the same initial factors."""
    nu, ni, n, s, d, r, og = full_cf
    g = gm.Graph(n, s, d, r, n_left=nu)
    K, gamma = 32, 1e-3
    g.program_set(gm.GM_CF, K=K, lam=LAM, gamma=gamma, init_sigma=0.1, seed=5)
    p0 = g.state().astype(np.float64)
    g.run(1)
    p1 = g.state().astype(np.float64)
    rng = np.random.default_rng(1)
    for v in list(rng.choice(nu, 8, replace=False)) + list(nu + rng.choice(ni, 4, replace=False)):
        ref = og.cf_vertex_step(K, LAM, gamma, p0, int(v))
        assert np.max(np.abs(p1[v] - ref)) <= 1e-4 * max(np.max(np.abs(ref)), 1e-3)


# Step size of the full-workload gradient-descent check.  With the specified
# gamma = 1e-3 full-batch gradient descent on this workload diverges in FP64 as
# well (the users with ~17,800 ratings take steps that grow their factors
# geometrically; the oracle's loss overflows by the seventh step), and at 1e-4 its
# loss rises again after the seventh step; 1e-5 is the largest power of ten
# <= 1e-3 at which the FP64 oracle's loss decreases in all 10 steps
# (tests/golden/cf_full_gamma_search.json, written by the script beside it).
CF_FULL_GAMMA = 1e-5


@pytest.mark.slow
def test_full_config_ten_steps_match_oracle(gm, full_cf):
    """480,000 users x 17,800 items, ~100M ratings, K = 32, lambda 0.05: ten
    Jacobi gradient steps of Eqs. 3-5 at CF_FULL_GAMMA.  Every factor against
    the FP64 oracle's ten steps from the same initial factors: relative
    Frobenius error and max-abs error over the largest factor both <= 1e-4, the
    change of the factors over the ten steps within 1e-4 (relative Frobenius),
    the Eq. 2 loss within 1e-5 relative, and the oracle's loss decreasing."""
    nu, ni, n, s, d, r, og = full_cf
    g = gm.Graph(n, s, d, r, n_left=nu)
    K = 32
    g.program_set(gm.GM_CF, K=K, lam=LAM, gamma=CF_FULL_GAMMA, init_sigma=0.1, seed=5)
    p0 = g.state().astype(np.float64)
    assert g.run(10) == 10
    got = g.state().astype(np.float64)
    loss = g.scalar(gm.GM_SCALAR_CF_LOSS)
    g.close()
    ref, trace = og.cf_gd(K, LAM, CF_FULL_GAMMA, 10, p0)
    assert np.all(np.diff(trace) < 0), "the oracle's loss decreases at this step size"
    err_fro = _rel_fro(got, ref)
    err_max = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    err_upd = _rel_fro(got - p0, ref - p0)
    print(f"full CF GD: rel fro {err_fro:.3e}, max-abs/max {err_max:.3e}, update rel fro {err_upd:.3e}, "
          f"loss {loss:.6e} vs {trace[-1]:.6e}")
    assert err_fro <= 1e-4
    assert err_max <= 1e-4
    # the ten steps' change of the factors itself, not only the factors (at this
    # step size the change is small next to the initial factors)
    assert err_upd <= 1e-4
    assert abs(loss - trace[-1]) <= 1e-5 * trace[-1]
