"""BFS and SSSP on the GPU against the FP64 oracle: bit-exact properties and
identical superstep counts (Algorithm 2 semantics), every direction mode and
loop mode, edge cases, and the scale-22 workload."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import CLEAN, check_sssp_certificate, random_case, rmat_case

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

DIRS = [0, 1, 2]  # auto, push only, pull only


def _run(gm, g, kind, sources, max_iters=-1):
    g.program_set(kind)
    g.set_active(sources)
    it = g.run(max_iters)
    return g.state(), it


@pytest.mark.parametrize("direction", DIRS)
@pytest.mark.parametrize("kind", ["bfs", "sssp"])
def test_rmat_small_parity(gm, kind, direction):
    n, s, d, w = rmat_case(12, weighted=True)
    g = gm.Graph(n, s, d, w)
    g.set_option(gm.GM_OPT_DIRECTION, direction)
    og = oracle.Graph(n, s, d, w)
    for src in synth.pick_sources(n, s, d, 4, seed=11):
        if kind == "bfs":
            got, it = _run(gm, g, gm.GM_BFS, [src])
            ref, rit = og.bfs([src])
        else:
            got, it = _run(gm, g, gm.GM_SSSP, [src])
            ref, rit = og.sssp([src])
        assert np.array_equal(got, ref)
        assert it == rit


@pytest.mark.parametrize("packed", [1, 0])
@pytest.mark.parametrize("stage", [40960, 0])
def test_sssp_pull_in_edge_layouts(gm, packed, stage):
    """The SSSP pull over the octet layout (each in-edge one word, source rank
    << 8 | weight, column lists padded to whole octets) and over separate rank
    and one-byte weight arrays, with and without the shared-memory stage,
    forced to pull every superstep and automatic: exact distances and
    superstep counts on an RMAT graph of several thousand warp tiles and a
    ragged last tile.  The layout option switched back and forth on one handle
    rebuilds the in-edge stream."""
    n, s, d, w = rmat_case(14, weighted=True)
    g = gm.Graph(n, s, d, w)
    og = oracle.Graph(n, s, d, w)
    assert g.m % 256 != 0
    g.program_set(gm.GM_SSSP)  # ranks and the default (packed) layout
    g.set_option(gm.GM_OPT_PULL_PACKED, 1 - packed)
    g.set_option(gm.GM_OPT_PULL_PACKED, packed)
    g.set_option(gm.GM_OPT_PULL_STAGE, stage)
    for direction in (2, 0):
        g.set_option(gm.GM_OPT_DIRECTION, direction)
        for src in synth.pick_sources(n, s, d, 3, seed=12):
            got, it = _run(gm, g, gm.GM_SSSP, [src])
            ref, rit = og.sssp([src])
            assert np.array_equal(got, ref) and it == rit


@pytest.mark.parametrize("packed", [1, 0])
def test_sssp_pull_column_shapes(gm, packed):
    """In-degrees that meet the octet layout's edges: columns of exactly 8, 16
    and 256 in-edges (whole octets, a whole tile of 32 octets), one of 8k + 1,
    a hub spanning several tiles, single-edge columns, and a graph whose octets
    fill less than one tile; forced pull from the first superstep and the
    automatic switch, against the oracle."""
    rng = np.random.default_rng(77)
    n = 3000
    parts = [(np.arange(1, 1001), 0), (np.arange(1001, 1009), 1), (np.arange(1009, 1025), 2),
             (np.arange(1025, 1281), 3), (np.arange(1281, 1298), 4), (np.arange(1298, 1299), 5)]
    src = np.concatenate([p for p, _ in parts] + [rng.integers(0, n, 20000)]).astype(np.int32)
    dst = np.concatenate([np.full(len(p), v) for p, v in parts] + [rng.integers(0, n, 20000)]).astype(np.int32)
    w = rng.integers(1, 256, len(src)).astype(np.uint32)
    cases = [(n, src, dst, w), (40, np.array([1, 2, 3, 4, 5, 6, 7, 8, 9, 0, 0], np.int32),
                                np.array([0, 0, 0, 0, 0, 0, 0, 0, 0, 9, 10], np.int32),
                                np.arange(1, 12, dtype=np.uint32))]
    for nn, ss, dd, ww in cases:
        g = gm.Graph(nn, ss, dd, ww)
        og = oracle.Graph(nn, ss, dd, ww)
        g.program_set(gm.GM_SSSP)
        g.set_option(gm.GM_OPT_PULL_PACKED, packed)
        for direction in (2, 0):
            g.set_option(gm.GM_OPT_DIRECTION, direction)
            for seeds in ([int(ss[0])], [int(x) for x in ss[:5]], [0]):
                got, it = _run(gm, g, gm.GM_SSSP, seeds)
                ref, rit = og.sssp(seeds)
                assert np.array_equal(got, ref) and it == rit


@pytest.mark.parametrize("direction", DIRS)
@pytest.mark.parametrize("kind", ["bfs", "sssp"])
def test_sorted_list_sparse_vector(gm, kind, direction):
    """GM_OPT_SPARSE_LIST (the ablation of Section 4.3.2's sparse-vector form):
    each pull superstep looks its sources up by binary search in a sorted
    (index, value) list of the frontier instead of the bitvector / dense message
    array.  Properties and superstep counts equal the oracle's on an RMAT graph
    (n not a multiple of the 2048-index list tile) and on a graph whose frontier
    holds a single vertex, from one and from several sources."""
    n, s, d, w = rmat_case(13, weighted=True)
    n += 77  # isolated vertices past the RMAT range: a ragged last list tile
    g = gm.Graph(n, s, d, w)
    og = oracle.Graph(n, s, d, w)
    g.set_option(gm.GM_OPT_SPARSE_LIST, 1)
    g.set_option(gm.GM_OPT_DIRECTION, direction)
    srcs = synth.pick_sources(n, s, d, 3, seed=21)
    prog, ref_fn = (gm.GM_BFS, og.bfs) if kind == "bfs" else (gm.GM_SSSP, og.sssp)
    for src in [[int(srcs[0])], [int(srcs[1])], srcs.tolist()]:
        got, it = _run(gm, g, prog, src)
        ref, rit = ref_fn(src)
        assert np.array_equal(got, ref) and it == rit
    # a path 0 -> 1 -> ... -> 9: every frontier is one vertex
    ps, pd = np.arange(9, dtype=np.int32), np.arange(1, 10, dtype=np.int32)
    pw = np.full(9, 3, np.uint32)
    gp = gm.Graph(10, ps, pd, pw)
    gp.set_option(gm.GM_OPT_SPARSE_LIST, 1)
    gp.set_option(gm.GM_OPT_DIRECTION, direction)
    opg = oracle.Graph(10, ps, pd, pw)
    got, it = _run(gm, gp, prog, [0])
    ref, rit = (opg.bfs if kind == "bfs" else opg.sssp)([0])
    assert np.array_equal(got, ref) and it == rit


@pytest.mark.parametrize("loop_mode", [0, 1])
@pytest.mark.parametrize("seed", range(3))
def test_random_graphs_multi_source(gm, seed, loop_mode):
    rng = np.random.default_rng(1000 + seed)
    n, s, d, w = random_case(rng, int(rng.integers(2, 5000)), int(rng.integers(1, 40000)), weighted=True)
    g = gm.Graph(n, s, d, w)
    g.set_option(gm.GM_OPT_LOOP_MODE, loop_mode)
    og = oracle.Graph(n, s, d, w)
    srcs = rng.choice(n, size=min(n, 3), replace=False).astype(np.int32)
    got, it = _run(gm, g, gm.GM_BFS, srcs)
    ref, rit = og.bfs(srcs)
    assert np.array_equal(got, ref) and it == rit
    got, it = _run(gm, g, gm.GM_SSSP, srcs)
    ref, rit = og.sssp(srcs)
    assert np.array_equal(got, ref) and it == rit


def test_bin_thresholds_do_not_change_results(gm):
    n, s, d, w = rmat_case(13, weighted=True)
    g = gm.Graph(n, s, d, w)
    og = oracle.Graph(n, s, d, w)
    src = synth.pick_sources(n, s, d, 1, seed=3)
    ref, rit = og.sssp(src)
    for small, large in [(2, 4), (8, 64), (32, 2048), (64, 1 << 20)]:
        g.set_option(gm.GM_OPT_BIN_LARGE, 1 << 30)
        g.set_option(gm.GM_OPT_BIN_SMALL, small)
        g.set_option(gm.GM_OPT_BIN_LARGE, large)
        for direction in DIRS:
            g.set_option(gm.GM_OPT_DIRECTION, direction)
            got, it = _run(gm, g, gm.GM_SSSP, src)
            assert np.array_equal(got, ref) and it == rit


def test_max_iters_truncates_like_oracle(gm):
    n, s, d, w = rmat_case(11, weighted=True)
    g = gm.Graph(n, s, d, w)
    og = oracle.Graph(n, s, d, w)
    src = synth.pick_sources(n, s, d, 1, seed=5)
    for k in (0, 1, 2, 3, 5):
        got, it = _run(gm, g, gm.GM_SSSP, src, max_iters=k)
        ref, rit = og.sssp(src, max_iters=k)
        assert it == rit
        if k > 0:
            assert np.array_equal(got, ref)


def test_golden_tiny(gm):
    gd = json.load(open(os.path.join(GOLDEN, "sssp_bfs_tiny.json")))
    g = gm.Graph(gd["n"], np.array(gd["src"], np.int32), np.array(gd["dst"], np.int32),
                 np.array(gd["w"], np.uint32))
    for loop_mode in (0, 1):
        g.set_option(gm.GM_OPT_LOOP_MODE, loop_mode)
        got, it = _run(gm, g, gm.GM_SSSP, [gd["source"]])
        assert got.tolist() == gd["sssp_dist"] and it == gd["sssp_supersteps"]
        got, it = _run(gm, g, gm.GM_BFS, [gd["source"]])
        assert got.tolist() == gd["bfs_depth"] and it == gd["bfs_supersteps"]


@pytest.mark.parametrize("packed", [1, 0])
def test_pull_on_graphs_without_in_edges(gm, packed):
    """SSSP and BFS forced to pull on graphs whose pull has nothing to stream: no
    edges, only self-loops (removed by cleaning), a single vertex.  The octet
    layout then has no tile; results and superstep counts equal the oracle's."""
    cases = [(6, np.zeros(0, np.int32), np.zeros(0, np.int32)),
             (4, np.array([0, 1, 2], np.int32), np.array([0, 1, 2], np.int32)),
             (1, np.zeros(0, np.int32), np.zeros(0, np.int32))]
    for n, s, d in cases:
        w = np.full(len(s), 7, np.uint32)
        g = gm.Graph(n, s, d, w)
        og = oracle.Graph(n, s, d, w)
        g.program_set(gm.GM_SSSP)
        g.set_option(gm.GM_OPT_PULL_PACKED, packed)
        g.set_option(gm.GM_OPT_DIRECTION, 2)
        for kind, ref_fn in ((gm.GM_SSSP, og.sssp), (gm.GM_BFS, og.bfs)):
            got, it = _run(gm, g, kind, [0])
            ref, rit = ref_fn([0])
            assert np.array_equal(got, ref) and it == rit


def test_edge_cases(gm):
    # isolated source: one superstep that finds nothing
    g = gm.Graph(5, np.array([1], np.int32), np.array([2], np.int32))
    got, it = _run(gm, g, gm.GM_BFS, [0])
    assert it == 1 and got.tolist() == [0] + [gm.INF_U32] * 4
    # no active vertex
    g.program_set(gm.GM_SSSP)
    assert g.run() == 1
    assert np.all(g.state() == gm.INF_U32)
    # unweighted SSSP is BFS
    n, s, d, _ = rmat_case(10)
    g = gm.Graph(n, s, d)
    a, _ = _run(gm, g, gm.GM_SSSP, [1])
    b, _ = _run(gm, g, gm.GM_BFS, [1])
    assert np.array_equal(a, b)
    # all vertices active: every property 0, one superstep... plus convergence
    g.program_set(gm.GM_BFS)
    g.set_active(None)
    g.run()
    assert np.all(g.state() == 0)
    # duplicate sources
    a, _ = _run(gm, g, gm.GM_BFS, [1, 1, 1])
    b, _ = _run(gm, g, gm.GM_BFS, [1])
    assert np.array_equal(a, b)
    # bad source id
    g.program_set(gm.GM_BFS)
    with pytest.raises(gm.GMError):
        g.set_active([n])
    # run before program_set
    g2 = gm.Graph(3, np.array([0], np.int32), np.array([1], np.int32))
    with pytest.raises(gm.GMError) as ei:
        g2.run()
    assert ei.value.status == gm.GM_ERR_STATE


def test_saturating_weights(gm):
    big = np.array([0xFFFFFFF0, 0x20], np.uint32)
    g = gm.Graph(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32), big)
    got, _ = _run(gm, g, gm.GM_SSSP, [0])
    assert got.tolist() == [0, 0xFFFFFFF0, gm.INF_U32]


@pytest.mark.parametrize("direction", DIRS)
def test_weight_width(gm, direction):
    """Weights below 256 are read as one byte by the SSSP pull, wider ones as four;
    both give the oracle's distances and superstep counts."""
    rng = np.random.default_rng(77)
    n, s, d, _ = rmat_case(12)
    for hi, width in ((255, 1), (1 << 20, 4)):
        w = rng.integers(1, hi + 1, len(s)).astype(np.uint32)
        g = gm.Graph(n, s, d, w)
        assert g.scalar(gm.GM_SCALAR_PULL_WEIGHT_BYTES) == width
        g.set_option(gm.GM_OPT_DIRECTION, direction)
        og = oracle.Graph(n, s, d, w)
        for src in synth.pick_sources(n, s, d, 2, seed=78):
            got, it = _run(gm, g, gm.GM_SSSP, [src])
            ref, rit = og.sssp([src])
            assert np.array_equal(got, ref) and it == rit
    assert gm.Graph(n, s, d).scalar(gm.GM_SCALAR_PULL_WEIGHT_BYTES) == 0


@pytest.mark.parametrize("stage", [0, 1000, 49152])
@pytest.mark.parametrize("direction", [0, 2])
def test_sssp_staged_and_gathered_messages(gm, direction, stage):
    """At scale 17 (n = 131,072) the SSSP pull stages the messages of the `stage`
    highest-out-degree sources in shared memory and gathers the rest: both kinds
    of source, one-byte and four-byte weights, match the oracle."""
    n, s, d, w = rmat_case(17, weighted=True, seed=synth.BASE_SEED + 17)
    rng = np.random.default_rng(17)
    for ww in (w, rng.integers(1, 1 << 24, len(s)).astype(np.uint32)):
        g = gm.Graph(n, s, d, ww)
        g.set_option(gm.GM_OPT_DIRECTION, direction)
        g.set_option(gm.GM_OPT_PULL_STAGE, stage)
        og = oracle.Graph(n, s, d, ww)
        for src in synth.pick_sources(n, s, d, 2, seed=170):
            got, it = _run(gm, g, gm.GM_SSSP, [src])
            ref, rit = og.sssp([src])
            assert np.array_equal(got, ref) and it == rit


@pytest.mark.parametrize("direction", [0, 2])
def test_sssp_distances_beyond_16_bits(gm, direction):
    """The octet pull stages its hot messages as signed 16 bits (finite values
    below 32,767).  A chain of 600 vertices joined by weight-255 edges carries
    distances up to 152,745, past what the stage holds (from superstep 129 on);
    those pulls must take every message from global memory instead.  Beside the chain, a random graph with
    small weights whose distances stay low.  Forced pull and the automatic
    switch, from the chain's head and from the random part, against the oracle."""
    rng = np.random.default_rng(1616)
    L, n = 600, 3000
    chain_s = np.arange(0, L - 1, dtype=np.int32)
    chain_d = chain_s + 1
    rs = rng.integers(L, n, 15000).astype(np.int32)
    rd = rng.integers(L, n, 15000).astype(np.int32)
    src = np.concatenate([chain_s, rs, np.array([L], np.int32)])
    dst = np.concatenate([chain_d, rd, np.array([0], np.int32)])
    w = np.concatenate([np.full(L - 1, 255, np.uint32), rng.integers(1, 8, 15000).astype(np.uint32),
                        np.array([3], np.uint32)])
    g = gm.Graph(n, src, dst, w)
    og = oracle.Graph(n, src, dst, w)
    g.program_set(gm.GM_SSSP)
    g.set_option(gm.GM_OPT_DIRECTION, direction)
    for seeds in ([0], [int(L) + 5], [0, int(L) + 5]):
        got, it = _run(gm, g, gm.GM_SSSP, seeds)
        ref, rit = og.sssp(seeds)
        assert np.array_equal(got, ref) and it == rit
        if seeds == [0]:
            assert int(ref[L - 1]) == 255 * (L - 1) > 0xFFFF


def test_symmetrized_bfs(gm):
    n, s, d, _ = rmat_case(12)
    flags = CLEAN | oracle.SYMMETRIZE
    g = gm.Graph(n, s, d, flags=flags)
    og = oracle.Graph(n, s, d, flags=flags)
    src = synth.pick_sources(n, s, d, 2, seed=9)
    got, it = _run(gm, g, gm.GM_BFS, src[:1])
    ref, rit = og.bfs(src[:1])
    assert np.array_equal(got, ref) and it == rit


@pytest.mark.slow
def test_scale22_workload(gm):
    """The benchmark workload: RMAT scale 22, edge factor 16, uint32 weights in
    [1, 255].  BFS depths and superstep counts match the oracle on two sources;
    SSSP matches the oracle on one source and passes the exact shortest-path
    certificate (relaxed + tight edges) on two more."""
    n, s, d, w = rmat_case(22, weighted=True)
    g = gm.Graph(n, s, d, w)
    og = oracle.Graph(n, s, d, w)
    cs, cd, cv = og.edges()
    srcs = synth.pick_sources(n, s, d, 16, seed=synth.BASE_SEED + 1)
    for src in srcs[:2]:
        got, it = _run(gm, g, gm.GM_BFS, [src])
        ref, rit = og.bfs([src])
        assert np.array_equal(got, ref) and it == rit
    got, it = _run(gm, g, gm.GM_SSSP, [srcs[0]])
    ref, rit = og.sssp([srcs[0]])
    assert np.array_equal(got, ref) and it == rit
    for src in srcs[1:3]:
        got, _ = _run(gm, g, gm.GM_SSSP, [src])
        check_sssp_certificate(n, cs, cd, cv.astype(np.uint32), got, np.array([src]))


@pytest.mark.slow
@pytest.mark.parametrize("scale,params", [(23, "graph500"), (24, "sssp24")])
def test_paper_rmat_shapes(gm, scale, params):
    """The paper's larger RMAT graphs (Section 5.1): RMAT-23 with a/b/c = .57/.19/.19
    (BFS and SSSP) and RMAT-24 with .50/.10/.10 (SSSP), one source each, bit-exact
    against the oracle with the same superstep counts."""
    n, s, d, w = rmat_case(scale, weighted=True, params=synth.RMAT_PARAMS[params], seed=synth.BASE_SEED + scale)
    g = gm.Graph(n, s, d, w)
    og = oracle.Graph(n, s, d, w)
    src = synth.pick_sources(n, s, d, 2, seed=synth.BASE_SEED + 200 + scale)
    if scale == 23:
        got, it = _run(gm, g, gm.GM_BFS, [src[0]])
        ref, rit = og.bfs([src[0]])
        assert np.array_equal(got, ref) and it == rit
    got, it = _run(gm, g, gm.GM_SSSP, [src[1]])
    ref, rit = og.sssp([src[1]])
    assert np.array_equal(got, ref) and it == rit


def test_autotune_keeps_results(gm):
    n, s, d, w = rmat_case(14, weighted=True)
    g = gm.Graph(n, s, d, w)
    og = oracle.Graph(n, s, d, w)
    srcs = synth.pick_sources(n, s, d, 3, seed=17)
    for kind, ref_fn in ((gm.GM_SSSP, og.sssp), (gm.GM_BFS, og.bfs)):
        choice = g.autotune(kind, srcs[:2])
        assert choice["best_ms"] > 0 and 1 <= choice["bin_small"] <= choice["bin_large"]
        got, it = _run(gm, g, kind, [srcs[2]])
        ref, rit = ref_fn([srcs[2]])
        assert np.array_equal(got, ref) and it == rit


def _stats(gm, g):
    return [g.scalar(x) for x in (gm.GM_SCALAR_SUPERSTEPS, gm.GM_SCALAR_PUSH_STEPS, gm.GM_SCALAR_PULL_STEPS,
                                  gm.GM_SCALAR_SCANNED_EDGES, gm.GM_SCALAR_PROCESSED_VERTICES)]


@pytest.mark.parametrize("kind", ["bfs", "sssp"])
def test_small_supersteps_match_host_loop(gm, kind):
    """The device loop runs supersteps with tiny frontiers in one CTA (trav_small),
    the host loop never does: properties, superstep counts, push/pull counts,
    edges scanned and vertices processed agree, with and without max_iters, on
    an RMAT graph (small heads and tails around large supersteps), a long path
    (every superstep small) and a graph whose frontier has large-degree hubs."""
    k = gm.GM_BFS if kind == "bfs" else gm.GM_SSSP
    n, s, d, w = rmat_case(14, weighted=True)
    n2 = 3000
    ps, pd = np.arange(n2 - 1, dtype=np.int32), np.arange(1, n2, dtype=np.int32)
    hs = np.concatenate([np.zeros(5000, np.int32), np.arange(1, 5001, dtype=np.int32)])
    hd = np.concatenate([np.arange(1, 5001, dtype=np.int32), (np.arange(5000, dtype=np.int32) * 7 + 3) % 5001])
    # a star of 3000 leaves of which only the first 40 have an out-edge (to 40
    # vertices chained one after another): the superstep over the centre sets 3000
    # frontier bits (more than the small kernel lists), the following ones are
    # small and must clear that bitvector whole
    ss_ = np.concatenate([np.zeros(3000, np.int32), np.arange(1, 41, dtype=np.int32),
                          np.arange(3001, 3040, dtype=np.int32)])
    sd_ = np.concatenate([np.arange(1, 3001, dtype=np.int32), np.arange(3001, 3041, dtype=np.int32),
                          np.arange(3002, 3041, dtype=np.int32)])
    cases = [(n, s, d, w, list(synth.pick_sources(n, s, d, 4, seed=31))),
             (n2, ps, pd, (ps % 7 + 1).astype(np.uint32), [0, 1500]),
             (5001, hs, hd, ((hs + hd) % 11 + 1).astype(np.uint32), [0, 17]),
             (3041, ss_, sd_, ((ss_ * 3 + sd_) % 13 + 1).astype(np.uint32), [0])]
    for nn, ss, dd, ww, srcs in cases:
        g = gm.Graph(nn, ss, dd, ww)
        og = oracle.Graph(nn, ss, dd, ww)
        for src in srcs:
            for max_iters in (-1, 1, 2, 5):
                res = []
                for loop_mode in (0, 1):
                    g.set_option(gm.GM_OPT_LOOP_MODE, loop_mode)
                    l0 = gm.kernel_launch_count()
                    got, it = _run(gm, g, k, [int(src)], max_iters)
                    res.append((got, it, _stats(gm, g)))
                    if nn == n2 and loop_mode == 0 and max_iters == -1:  # one loop iteration ran them all
                        assert it > 1000 and gm.kernel_launch_count() - l0 < 100  # vs about 4 per superstep
                assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]
                assert res[0][2] == res[1][2], (nn, src, max_iters, res[0][2], res[1][2])
                if max_iters == -1:
                    ref, rit = (og.bfs if kind == "bfs" else og.sssp)([int(src)])
                    assert np.array_equal(res[0][0], ref) and res[0][1] == rit
        g.close()


def test_reached_edges_counter(gm):
    """GM_SCALAR_REACHED_EDGES is kept by the traversal kernels (a vertex's
    out-degree is added when its property first becomes finite: seeding, push,
    pull, the small-superstep kernel); it must equal the sum of out-degrees over
    the finite properties after every call sequence: one or several sources,
    repeated and already-reached sources, continued runs, max_iters, every
    direction, all vertices active, program switches and a caller-written state."""
    n, s, d, w = rmat_case(13, weighted=True)
    g = gm.Graph(n, s, d, w)
    od, _ = g.degrees()
    srcs = [int(x) for x in synth.pick_sources(n, s, d, 6, seed=41)]

    def expect():
        st = g.state()
        return int(od[st != gm.INF_U32].astype(np.int64).sum())

    for kind in (gm.GM_BFS, gm.GM_SSSP):
        for direction in DIRS:
            g.set_option(gm.GM_OPT_DIRECTION, direction)
            g.program_set(kind)
            assert g.scalar(gm.GM_SCALAR_REACHED_EDGES) == 0
            g.set_active(srcs[:1])
            g.run(2)
            assert g.scalar(gm.GM_SCALAR_REACHED_EDGES) == expect()
            g.set_active(srcs[1:3] + srcs[1:2])  # a repeated source
            g.run(-1)
            assert g.scalar(gm.GM_SCALAR_REACHED_EDGES) == expect()
            g.set_active(srcs[:4])  # sources already reached
            g.run(3)
            assert g.scalar(gm.GM_SCALAR_REACHED_EDGES) == expect()
            g.set_active(srcs[4:5])
            assert g.scalar(gm.GM_SCALAR_REACHED_EDGES) == expect()  # seeds pending: counted from the state
            g.run(-1)
            assert g.scalar(gm.GM_SCALAR_REACHED_EDGES) == expect()
        g.set_option(gm.GM_OPT_DIRECTION, 0)
        g.program_set(kind)
        g.set_active(np.arange(0, n, 97, dtype=np.int32))
        g.run(0)
        assert g.scalar(gm.GM_SCALAR_REACHED_EDGES) == expect()
        g.run(-1)
        assert g.scalar(gm.GM_SCALAR_REACHED_EDGES) == expect()
        g.program_set(kind)
        g.set_active()  # every vertex
        g.run(2)
        assert g.scalar(gm.GM_SCALAR_REACHED_EDGES) == expect() == int(od.astype(np.int64).sum())
        st = g.state()
        st[:n // 2] = gm.INF_U32
        g.set_state(st)
        assert g.scalar(gm.GM_SCALAR_REACHED_EDGES) == expect()
        g.set_active(srcs[5:6])
        g.run(-1)
        assert g.scalar(gm.GM_SCALAR_REACHED_EDGES) == expect()
    g.close()
