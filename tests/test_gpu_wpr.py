"""Differentiable weighted PageRank on the GPU: forward against the FP64 oracle,
the hand-written adjoint against the oracle gradient (itself pinned to central
finite differences on the CPU) and against FP64 finite differences on sampled
edges, independence of the checkpoint interval, and the autograd wrapper."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rmat_case

pytestmark = pytest.mark.gpu
R, STEPS = 0.15, 30


def _setup(gm, scale, seed=5):
    import torch
    n, s, d, _ = rmat_case(scale, 16, seed=synth.BASE_SEED + seed)
    g = gm.Graph(n, s, d)
    og = oracle.Graph(n, s, d)
    w = synth.uniform_f32(g.m, seed=seed, stream=1, lo=0.5, hi=1.5)
    tau = synth.uniform_f32(n, seed=seed, stream=2, lo=0.5, hi=1.5)
    return g, og, w, tau, torch.from_numpy(w).cuda(), torch.from_numpy(tau).cuda()


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("scale", [8, 12, 16])
def test_forward_and_gradient_match_oracle(gm, scale):
    g, og, w, tau, tw, ttau = _setup(gm, scale)
    x = g.wpagerank_forward(tw, R, STEPS, 5)
    xo, loss_o = og.wpr_forward(w.astype(np.float64), tau.astype(np.float64), R, STEPS)
    xg = x.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(xg - xo) / np.abs(xo)) <= 1e-5
    dldx = 2.0 * (x - ttau)
    grad = g.wpagerank_backward(dldx).cpu().numpy().astype(np.float64)
    go, _ = og.wpr_gradient(w.astype(np.float64), tau.astype(np.float64), R, STEPS)
    assert _rel_l2(grad, go) <= 1e-4


@pytest.mark.parametrize("every", [1, 4, 7, 30, 64])
def test_checkpoint_interval_does_not_change_gradient(gm, every):
    g, og, w, tau, tw, ttau = _setup(gm, 10)
    x = g.wpagerank_forward(tw, R, STEPS, 5)
    ref = g.wpagerank_backward(2.0 * (x - ttau)).cpu().numpy()
    x2 = g.wpagerank_forward(tw, R, STEPS, every)
    assert np.array_equal(x.cpu().numpy(), x2.cpu().numpy())
    got = g.wpagerank_backward(2.0 * (x2 - ttau)).cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-9)


def test_gradient_matches_fd_on_sampled_edges(gm):
    """Central differences in FP64 (h = 1e-6) on 64 sampled edges of a scale-10 graph.
    L(w+h) - L(w-h) is evaluated as sum_v (x+ - x-)(x+ + x- - 2 tau), the same
    difference without subtracting two large losses.  At larger scales hub ranks
    of order 1e3 limit FP64 central differences with h = 1e-6 to about 1e-4
    relative, so the full-size check compares with the FP64 adjoint instead."""
    g, og, w, tau, tw, ttau = _setup(gm, 10)
    x = g.wpagerank_forward(tw, R, STEPS, 5)
    grad = g.wpagerank_backward(2.0 * (x - ttau)).cpu().numpy().astype(np.float64)
    w64, tau64 = w.astype(np.float64), tau.astype(np.float64)
    rng = np.random.default_rng(0)
    edges = rng.choice(g.m, 64, replace=False)
    gmax = np.abs(og.wpr_gradient(w64, tau64, R, STEPS)[0]).max()
    h = 1e-6
    for e in edges:
        wp = w64.copy(); wp[e] += h
        wm = w64.copy(); wm[e] -= h
        xp = og.wpr_forward(wp, tau64, R, STEPS)[0]
        xm = og.wpr_forward(wm, tau64, R, STEPS)[0]
        fd = float(np.sum((xp - xm) * (xp + xm - 2.0 * tau64))) / (2 * h)
        assert abs(grad[e] - fd) <= 1e-4 * max(abs(fd), 1e-3 * gmax) + 1e-7


def test_autograd_function(gm):
    import torch
    from paper_1503_07241_gb300.autograd import WeightedPageRank
    g, og, w, tau, tw, ttau = _setup(gm, 11)
    wt = tw.clone().requires_grad_(True)
    x = WeightedPageRank.apply(wt, g, R, STEPS, 5)
    loss = ((x - ttau) ** 2).sum()
    loss.backward()
    go, loss_o = og.wpr_gradient(w.astype(np.float64), tau.astype(np.float64), R, STEPS)
    assert abs(float(loss.detach()) - loss_o) <= 1e-4 * loss_o
    assert _rel_l2(wt.grad.cpu().numpy().astype(np.float64), go) <= 1e-4


def test_backward_before_forward_is_rejected(gm):
    import torch
    g, og, w, tau, tw, ttau = _setup(gm, 6)
    with pytest.raises(gm.GMError) as ei:
        g.wpagerank_backward(torch.zeros(g.n, device="cuda"))
    assert ei.value.status == gm.GM_ERR_STATE


@pytest.mark.slow
def test_scale20_config_gradient(gm):
    """The weighted-PageRank workload: RMAT scale 20, edge factor 16, w ~ U[0.5, 1.5],
    30 supersteps, checkpoints every 5: forward within 1e-5 and the gradient
    within 1e-4 of the FP64 oracle adjoint, both as relative L2 over all edges
    and edge by edge, |g - g*| <= 1e-4 max(|g*|, 1e-3 max|g*|) (the floor of the
    finite-difference check: a per-edge relative error means nothing where the
    gradient is a rounding-level remainder of the row-normalisation term)."""
    g, og, w, tau, tw, ttau = _setup(gm, 20, seed=20)
    x = g.wpagerank_forward(tw, R, STEPS, 5)
    xo, _ = og.wpr_forward(w.astype(np.float64), tau.astype(np.float64), R, STEPS)
    assert np.max(np.abs(x.cpu().numpy() - xo) / np.abs(xo)) <= 1e-5
    grad = g.wpagerank_backward(2.0 * (x - ttau)).cpu().numpy().astype(np.float64)
    go, _ = og.wpr_gradient(w.astype(np.float64), tau.astype(np.float64), R, STEPS)
    assert _rel_l2(grad, go) <= 1e-4
    floor = 1e-3 * np.abs(go).max()
    per_edge = np.abs(grad - go) / np.maximum(np.abs(go), floor)
    worst = int(np.argmax(per_edge))
    print(f"scale-20 gradient: rel L2 {_rel_l2(grad, go):.3e}, worst per-edge {per_edge[worst]:.3e} "
          f"(edge {worst}, g* {go[worst]:.3e}, floor {floor:.3e}), "
          f"edges above the floor {int(np.count_nonzero(np.abs(go) >= floor))} of {g.m}")
    assert per_edge.max() <= 1e-4
