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
