"""Failure paths without a GPU fault: injected allocation failures on the host
side of every entry point, and a bounded device wait made to run out."""
import numpy as np
import pytest

import oracle
from gpu_util import random_case

pytestmark = pytest.mark.gpu


def test_injected_allocation_failures(gm):
    """Every k-th allocation failing makes the call return GM_ERR_OUT_OF_MEMORY
    (nothing else); once the hook is off the library works and matches the oracle."""
    rng = np.random.default_rng(91)
    n, s, d, w = random_case(rng, 3000, 20000, weighted=True)
    failures = 0
    try:
        for k in range(0, 40):
            gm.lib().gm_debug_fail_allocations_after(k)
            try:
                g = gm.Graph(n, s, d, w)
                for kind in (gm.GM_BFS, gm.GM_SSSP):
                    g.program_set(kind)
                    g.set_active([0])
                    g.run(-1)
                g.close()
            except gm.GMError as e:
                assert e.status == gm.GM_ERR_OUT_OF_MEMORY
                failures += 1
    finally:
        gm.lib().gm_debug_fail_allocations_after(-1)
    assert failures > 10
    g = gm.Graph(n, s, d, w)
    og = oracle.Graph(n, s, d, w)
    for kind, ref in ((gm.GM_BFS, og.bfs), (gm.GM_SSSP, og.sssp)):
        g.program_set(kind)
        g.set_active([0])
        it = g.run(-1)
        want, wit = ref([0])
        assert np.array_equal(g.state(), want) and it == wit


def test_staging_wait_runs_out(gm):
    """The SSSP pull's staging barrier is made to wait for bytes that never come:
    every CTA gives up after its bounded wait, gathers from global memory instead,
    the superstep's result is still exact and gm_run reports GM_ERR_TIMEOUT; the
    handle keeps working afterwards."""
    rng = np.random.default_rng(92)
    n, s, d, w = random_case(rng, 4000, 40000, weighted=True)
    g = gm.Graph(n, s, d, w)
    og = oracle.Graph(n, s, d, w)
    g.set_option(gm.GM_OPT_DIRECTION, 2)  # pull from the first superstep
    g.set_option(gm.GM_OPT_TEST_STALL_STAGE, 1)
    g.program_set(gm.GM_SSSP)
    g.set_active([0])
    with pytest.raises(gm.GMError) as ei:
        g.run(1)
    assert ei.value.status == gm.GM_ERR_TIMEOUT
    want, _ = og.sssp([0], max_iters=1)
    assert np.array_equal(g.state(), want)
    g.set_option(gm.GM_OPT_TEST_STALL_STAGE, 0)
    g.program_set(gm.GM_SSSP)
    g.set_active([0])
    it = g.run(-1)
    want, wit = og.sssp([0])
    assert np.array_equal(g.state(), want) and it == wit


def test_sgd_grid_barrier_wait_runs_out(gm):
    """The grid barrier between SGD strata is made to wait for a CTA that never
    arrives (test hook GM_OPT_TEST_STALL_SGD: the last CTA skips its arrival at
    the first barrier and the wait limit drops to half a second): every CTA's
    bounded wait gives up, the kernel ends, gm_run reports GM_ERR_TIMEOUT, and
    after the hook is cleared the same handle runs two epochs that equal the
    oracle's serial SGD (Section 3.III; stratified order)."""
    import synth
    nu, ni = 2000, 300
    n, s, d, r = synth.chung_lu_bipartite(nu, ni, 1.1, 5e4, seed=17)
    g = gm.Graph(n, s, d, r, n_left=nu)
    og = oracle.Graph(n, s, d, r)
    g.set_option(gm.GM_OPT_TEST_STALL_SGD, 1)
    g.program_set(gm.GM_CF_SGD, K=32, lam=0.05, gamma=1e-2, init_sigma=0.1, seed=3, cf_strata=64)
    with pytest.raises(gm.GMError) as ei:
        g.run(1)
    assert ei.value.status == gm.GM_ERR_TIMEOUT
    assert "never arrived" in str(ei.value)
    g.set_option(gm.GM_OPT_TEST_STALL_SGD, 0)
    g.program_set(gm.GM_CF_SGD, K=32, lam=0.05, gamma=1e-2, init_sigma=0.1, seed=3, cf_strata=64)
    p0 = g.state().astype(np.float64)
    ref = og.cf_sgd(32, 0.05, 1e-2, 2, nu, 64, p0)
    assert g.run(2) == 2
    np.testing.assert_allclose(g.state().astype(np.float64), ref, rtol=1e-4, atol=2e-5)


def test_failed_layout_builds_recover_on_the_same_handle(gm):
    """An allocation failure while the SSSP pull's ranks and in-edge layout are
    built (gm_program_set) or rebuilt (the layout option) leaves the handle
    without a layout: gm_run refuses with an error instead of running, and the
    next successful gm_program_set builds it again; the same handle then matches
    the oracle."""
    rng = np.random.default_rng(93)
    n, s, d, w = random_case(rng, 3000, 20000, weighted=True)
    og = oracle.Graph(n, s, d, w)
    want, wit = og.sssp([0])
    recovered = 0
    for k in range(12):
        g = gm.Graph(n, s, d, w)
        g.program_set(gm.GM_BFS)
        gm.lib().gm_debug_fail_allocations_after(k)
        try:
            g.program_set(gm.GM_SSSP)
            failed = False
        except gm.GMError as e:
            assert e.status == gm.GM_ERR_OUT_OF_MEMORY
            failed = True
        finally:
            gm.lib().gm_debug_fail_allocations_after(-1)
        if failed:
            with pytest.raises(gm.GMError):
                g.run(-1)
            g.program_set(gm.GM_SSSP)
            recovered += 1
        g.set_active([0])
        it = g.run(-1)
        assert np.array_equal(g.state(), want) and it == wit
    assert recovered >= 3
    # the layout option's rebuild fails: no run until the next program_set
    g = gm.Graph(n, s, d, w)
    g.program_set(gm.GM_SSSP)
    gm.lib().gm_debug_fail_allocations_after(0)
    try:
        with pytest.raises(gm.GMError) as ei:
            g.set_option(gm.GM_OPT_PULL_PACKED, 0)
        assert ei.value.status == gm.GM_ERR_OUT_OF_MEMORY
    finally:
        gm.lib().gm_debug_fail_allocations_after(-1)
    g.set_active([0])
    with pytest.raises(gm.GMError) as ei:
        g.run(-1)
    assert ei.value.status == gm.GM_ERR_STATE
    g.program_set(gm.GM_SSSP)
    g.set_active([0])
    it = g.run(-1)
    assert np.array_equal(g.state(), want) and it == wit
