"""Batched BFS/SSSP (gm_run_batch) on the GPU: every query bit-exact (values and
superstep counts) against the same query run alone and against the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _graphs(gm, scales, seed):
    out = []
    for i, sc in enumerate(scales):
        n, s, d = synth.rmat(int(sc), 16, synth.RMAT_PARAMS["graph500"], seed + i)
        w = synth.edge_weights_u32(s, d, seed + 1000 + i)
        out.append((n, s, d, w, gm.Graph(n, s, d, w)))
    return out


def _queries(graphs, per_graph, seed):
    q = []
    for gi, (n, s, d, w, g) in enumerate(graphs):
        src = synth.pick_sources(n, s, d, 2 * per_graph, seed=seed + gi)
        q += [(gi, 1, int(x)) for x in src[:per_graph]]        # GM_BFS
        q += [(gi, 2, int(x)) for x in src[per_graph:]]        # GM_SSSP
    return q


def _single(gm, g, kind, src):
    g.program_set(kind)
    g.set_active([src])
    it = g.run(-1)
    return g.state(), it


def _run(gm, graphs, queries, max_iters=-1):
    import torch
    outs = [torch.empty(graphs[gi][0], dtype=torch.int32, device="cuda") for gi, _, _ in queries]
    its = gm.run_batch([t[4] for t in graphs], queries, outs, max_iters)
    return [o.cpu().numpy().view(np.uint32) for o in outs], its


def test_small_batch_matches_single_and_oracle(gm):
    graphs = _graphs(gm, [6, 9, 12, 10], synth.BASE_SEED + 70)
    queries = _queries(graphs, 3, 71)
    res, its = _run(gm, graphs, queries)
    for (gi, kind, src), got, it in zip(queries, res, its):
        n, s, d, w, g = graphs[gi]
        ref, rit = _single(gm, g, kind, src)
        assert np.array_equal(got, ref) and it == rit
        og = oracle.Graph(n, s, d, w)
        oref, oit = (og.bfs if kind == 1 else og.sssp)([src])
        assert np.array_equal(got, oref) and it == oit


def test_batch_max_iters_and_repeat(gm):
    graphs = _graphs(gm, [11], synth.BASE_SEED + 80)
    queries = _queries(graphs, 2, 81)
    n, s, d, w, g = graphs[0]
    og = oracle.Graph(n, s, d, w)
    for k in (1, 2, 4):
        res, its = _run(gm, graphs, queries, max_iters=k)
        for (gi, kind, src), got, it in zip(queries, res, its):
            oref, oit = (og.bfs if kind == 1 else og.sssp)([src], max_iters=k)
            assert np.array_equal(got, oref) and it == oit
    a, ia = _run(gm, graphs, queries)
    b, ib = _run(gm, graphs, queries)
    assert all(np.array_equal(x, y) for x, y in zip(a, b)) and ia == ib


def test_batch_edge_cases(gm):
    import torch
    g = gm.Graph(4, np.array([0, 1], np.int32), np.array([1, 2], np.int32), np.array([5, 7], np.uint32))
    outs = [torch.empty(4, dtype=torch.int32, device="cuda") for _ in range(3)]
    its = gm.run_batch([g], [(0, 1, 3), (0, 2, 0), (0, 1, 0)], outs)
    assert [o.cpu().numpy().view(np.uint32).tolist() for o in outs] == [
        [gm.INF_U32, gm.INF_U32, gm.INF_U32, 0], [0, 5, 12, gm.INF_U32], [0, 1, 2, gm.INF_U32]]
    assert its == [1, 3, 3]
    with pytest.raises(gm.GMError):
        gm.run_batch([g], [(0, 1, 4)], outs[:1])
    with pytest.raises(gm.GMError):
        gm.run_batch([g], [(1, 1, 0)], outs[:1])


@pytest.mark.slow
def test_batch_config_64_graphs_1024_queries(gm):
    """The batched workload: 64 RMAT graphs with scales drawn from U{12..20}, edge
    factor 16, weights in [1, 255]; 8 BFS + 8 SSSP queries per graph (512 + 512).
    Every query equals the single-query run; a sample also equals the oracle."""
    scales = synth.uniform_int(64, synth.BASE_SEED + 4, 0, 12, 20)
    graphs = _graphs(gm, scales, synth.BASE_SEED + 400)
    queries = _queries(graphs, 8, 401)
    assert len(queries) == 1024
    res, its = _run(gm, graphs, queries)
    for (gi, kind, src), got, it in zip(queries, res, its):
        ref, rit = _single(gm, graphs[gi][4], kind, src)
        assert np.array_equal(got, ref) and it == rit
    small = [i for i, (gi, _, _) in enumerate(queries) if scales[gi] <= 13][:6]
    for i in small:
        gi, kind, src = queries[i]
        n, s, d, w, g = graphs[gi]
        oref, oit = (oracle.Graph(n, s, d, w).bfs if kind == 1 else oracle.Graph(n, s, d, w).sssp)([src])
        assert np.array_equal(res[i], oref) and its[i] == oit


def test_batch_full_bundles_duplicates_and_unweighted(gm):
    """More than eight queries of one program on one graph (several bundles, one
    partly filled), repeated sources inside a bundle, interleaved programs, an
    unweighted graph next to a weighted one, and a graph of one vertex."""
    n, s, d = synth.rmat(10, 16, synth.RMAT_PARAMS["graph500"], synth.BASE_SEED + 90)
    w = synth.edge_weights_u32(s, d, synth.BASE_SEED + 91)
    gw = gm.Graph(n, s, d, w)
    gu = gm.Graph(n, s, d)
    g1 = gm.Graph(1, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    src = synth.pick_sources(n, s, d, 12, seed=92)
    queries = []
    for i in range(21):
        queries.append((0, 2 if i % 3 else 1, int(src[i % 12])))
        queries.append((1, 1 if i % 2 else 2, int(src[(5 * i) % 12])))
    queries += [(2, 1, 0), (2, 2, 0)]
    graphs = [(n, s, d, w, gw), (n, s, d, None, gu), (1, None, None, None, g1)]
    res, its = _run(gm, graphs, queries)
    og = {0: oracle.Graph(n, s, d, w), 1: oracle.Graph(n, s, d)}
    for (gi, kind, x), got, it in zip(queries, res, its):
        if gi == 2:
            assert got.tolist() == [0] and it == 1
            continue
        oref, oit = (og[gi].bfs if kind == 1 else og[gi].sssp)([x])
        assert np.array_equal(got, oref) and it == oit


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_batch_every_direction(gm, direction):
    """Bundles push or pull per superstep from the handle's switch point: forced
    push, forced pull and the automatic switch all give every query's exact
    result and superstep count (with and without max_iters), on graphs where the
    automatic switch does both."""
    graphs = _graphs(gm, [9, 12], synth.BASE_SEED + 120)
    for t in graphs:
        t[4].set_option(gm.GM_OPT_DIRECTION, direction)
    queries = _queries(graphs, 9, 121)  # 9 per program and graph: a full bundle and one more
    for max_iters in (-1, 3):
        res, its = _run(gm, graphs, queries, max_iters)
        for (gi, kind, src), got, it in zip(queries, res, its):
            n, s, d, w, g = graphs[gi]
            og = oracle.Graph(n, s, d, w)
            oref, oit = (og.bfs if kind == 1 else og.sssp)([src], max_iters=max_iters)
            assert np.array_equal(got, oref) and it == oit, (direction, max_iters, gi, kind, src)
