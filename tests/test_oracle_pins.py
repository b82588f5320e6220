"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks an oracle function against a textbook or library routine
(queue BFS, Dijkstra, a dense linear solve, networkx triangle counts, finite
differences), a closed form, an invariant, or a hand-worked fixture under
tests/golden/.  A dropped term, a wrong sign or a transposed operand in the
oracle fails at least one of them.
"""
import heapq
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = oracle.INF_U32
CLEAN = oracle.DROP_SELF_LOOPS | oracle.DEDUP


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _random_graph(rng, n, m, loops=True):
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    if not loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    return src, dst


# ---------------------------------------------------------------- cleaning
@pytest.mark.parametrize("seed", range(5))
def test_cleaning_matches_numpy_unique(seed):
    rng = np.random.default_rng(seed)
    n = 40
    src, dst = _random_graph(rng, n, 400)
    w = rng.integers(1, 1000, src.shape[0]).astype(np.uint32)
    g = oracle.Graph(n, src, dst, w, flags=CLEAN)
    s, d, v = g.edges()
    keep = src != dst
    key = src[keep].astype(np.int64) * n + dst[keep]
    uk, first = np.unique(key, return_index=True)  # first occurrence in input order
    assert np.array_equal(s.astype(np.int64) * n + d, uk)
    assert np.array_equal(v, w[keep][first].astype(np.float64))
    out_deg, in_deg = g.degrees()
    assert np.array_equal(out_deg, np.bincount(s, minlength=n))
    assert np.array_equal(in_deg, np.bincount(d, minlength=n))


def test_cleaning_flags_off_keeps_everything():
    src = np.array([0, 0, 1, 1], np.int32)
    dst = np.array([0, 1, 0, 0], np.int32)
    g = oracle.Graph(2, src, dst, flags=0)
    assert g.m == 4
    g = oracle.Graph(2, src, dst, flags=oracle.DEDUP)
    assert g.m == 3
    g = oracle.Graph(2, src, dst, flags=oracle.DROP_SELF_LOOPS)
    assert g.m == 3


def test_invalid_vertex_id_rejected():
    with pytest.raises(ValueError):
        oracle.Graph(3, np.array([0, 3], np.int32), np.array([1, 1], np.int32))


@pytest.mark.parametrize("seed", range(3))
def test_symmetrize_and_orient(seed):
    rng = np.random.default_rng(seed)
    n = 30
    src, dst = _random_graph(rng, n, 200)
    g = oracle.Graph(n, src, dst, flags=CLEAN | oracle.SYMMETRIZE)
    s, d, _ = g.edges()
    und = {(min(a, b), max(a, b)) for a, b in zip(src, dst) if a != b}
    assert set(zip(s.tolist(), d.tolist())) == und | {(b, a) for a, b in und}
    deg = np.bincount(s, minlength=n)
    go = oracle.Graph(n, src, dst, flags=CLEAN | oracle.SYMMETRIZE | oracle.ORIENT_BY_DEGREE)
    so, do, _ = go.edges()
    assert go.m == len(und)
    for a, b in zip(so, do):
        assert (deg[a], a) < (deg[b], b)


# ---------------------------------------------------------------- BFS
def _scipy_dist(n, s, d, w, sources, unweighted):
    A = sp.csr_matrix((w if w is not None else np.ones(len(s)), (s, d)), shape=(n, n))
    D = csg.shortest_path(A, method="D", directed=True, unweighted=unweighted, indices=sources)
    D = np.atleast_2d(D).min(axis=0)
    out = np.full(n, INF, np.uint32)
    fin = np.isfinite(D)
    out[fin] = D[fin].astype(np.uint64).astype(np.uint32)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_bfs_matches_scipy_breadth_first(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 80))
    src, dst = _random_graph(rng, n, int(rng.integers(1, 4 * n)))
    g = oracle.Graph(n, src, dst)
    s, d, _ = g.edges()
    sources = rng.choice(n, size=int(rng.integers(1, 3)), replace=False).astype(np.int32)
    depth, iters = g.bfs(sources)
    ref = _scipy_dist(n, s, d, None, sources, unweighted=True)
    assert np.array_equal(depth, ref)
    # supersteps: one per BFS level plus the converging one
    assert iters == int(depth[depth != INF].max()) + 1
    # edge invariant depth(v) <= depth(u) + 1
    fin = depth[s] != INF
    assert np.all(depth[d[fin]].astype(np.int64) <= depth[s[fin]].astype(np.int64) + 1)


def test_bfs_max_iters_truncates():
    src = np.arange(0, 9, dtype=np.int32)
    dst = np.arange(1, 10, dtype=np.int32)
    g = oracle.Graph(10, src, dst)
    depth, iters = g.bfs([0], max_iters=3)
    assert iters == 3
    assert depth.tolist() == [0, 1, 2, 3] + [INF] * 6


def test_bfs_sssp_golden():
    gd = _golden("sssp_bfs_tiny.json")
    g = oracle.Graph(gd["n"], np.array(gd["src"], np.int32), np.array(gd["dst"], np.int32),
                     np.array(gd["w"], np.uint32))
    dist, it = g.sssp([gd["source"]])
    assert dist.tolist() == gd["sssp_dist"]
    assert it == gd["sssp_supersteps"]
    depth, it = g.bfs([gd["source"]])
    assert depth.tolist() == gd["bfs_depth"]
    assert it == gd["bfs_supersteps"]


# ---------------------------------------------------------------- SSSP
def _dijkstra_hops(n, s, d, w, source):
    """Dijkstra on (distance, hops): the hop count of the fewest-edge shortest path."""
    adj = [[] for _ in range(n)]
    for a, b, c in zip(s.tolist(), d.tolist(), w.tolist()):
        adj[a].append((b, c))
    best = {source: (0, 0)}
    pq = [(0, 0, source)]
    done = set()
    while pq:
        dd, hh, u = heapq.heappop(pq)
        if u in done:
            continue
        done.add(u)
        for v, c in adj[u]:
            cand = (dd + c, hh + 1)
            if v not in best or cand < best[v]:
                best[v] = cand
                heapq.heappush(pq, (cand[0], cand[1], v))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_sssp_matches_dijkstra(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(2, 70))
    src, dst = _random_graph(rng, n, int(rng.integers(1, 5 * n)))
    w = synth.edge_weights_u32(src, dst, seed=seed, lo=1, hi=255)
    g = oracle.Graph(n, src, dst, w)
    s, d, v = g.edges()
    source = int(rng.integers(0, n))
    dist, iters = g.sssp([source])
    ref = _scipy_dist(n, s, d, v, [source], unweighted=False)
    assert np.array_equal(dist, ref)
    # Bellman-Ford rounds: the last change happens in superstep h*-1 where h* is the
    # largest fewest-edge shortest-path length; one more superstep finds no change.
    best = _dijkstra_hops(n, s, d, v.astype(np.int64), source)
    assert iters == max(h for _, h in best.values()) + 1
    fin = dist[s] != INF
    assert np.all(dist[d[fin]].astype(np.int64) <= dist[s[fin]].astype(np.int64) + v[fin].astype(np.int64))


def test_sssp_saturates_at_infinity():
    big = np.array([0xFFFFFFF0, 0x20], np.uint32)
    g = oracle.Graph(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32), big)
    dist, _ = g.sssp([0])
    assert dist.tolist() == [0, 0xFFFFFFF0, INF]


def test_sssp_multi_source_is_min_of_single():
    n, src, dst = synth.rmat(8, 8)
    w = synth.edge_weights_u32(src, dst, 7)
    g = oracle.Graph(n, src, dst, w)
    a, _ = g.sssp([3])
    b, _ = g.sssp([17])
    ab, _ = g.sssp([3, 17])
    assert np.array_equal(ab, np.minimum(a, b))


# ---------------------------------------------------------------- PageRank
def test_pagerank_golden_both_readings():
    gd = _golden("pagerank_tiny.json")
    g = oracle.Graph(gd["n"], np.array(gd["src"], np.int32), np.array(gd["dst"], np.int32))
    x, it = g.pagerank(gd["r"], gd["iters"], apply_all_vertices=True)
    assert it == gd["iters"]
    np.testing.assert_allclose(x, gd["rank_eq1_all_vertices"], rtol=0, atol=1e-15)
    x, _ = g.pagerank(gd["r"], gd["iters"], apply_all_vertices=False)
    np.testing.assert_allclose(x, gd["rank_alg2_received_only"], rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_pagerank_fixed_point_is_linear_solve(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(3, 50))
    src, dst = _random_graph(rng, n, 4 * n)
    g = oracle.Graph(n, src, dst)
    s, d, _ = g.edges()
    out_deg, _ = g.degrees()
    r = 0.15
    P = np.zeros((n, n))
    for a, b in zip(s, d):
        P[a, b] += 1.0 / out_deg[a]
    ref = np.linalg.solve(np.eye(n) - (1 - r) * P.T, r * np.ones(n))
    x, _ = g.pagerank(r, 500)
    np.testing.assert_allclose(x, ref, rtol=1e-12, atol=1e-12)


def test_pagerank_regular_digraph_stays_one():
    n, k = 64, 5  # circulant: v -> v+1..v+k, in- and out-degree k
    src = np.repeat(np.arange(n), k).astype(np.int32)
    dst = ((src + np.tile(np.arange(1, k + 1), n)) % n).astype(np.int32)
    g = oracle.Graph(n, src, dst)
    x, _ = g.pagerank(0.15, 20)
    assert np.all(x == 1.0)


def test_pagerank_in_degree_closed_form():
    """With r = 0 and every out-degree 1, one step gives y = G^T 1 (Figure 1)."""
    rng = np.random.default_rng(5)
    n = 50
    src = np.arange(n, dtype=np.int32)
    dst = rng.integers(0, n, n).astype(np.int32)
    dst[dst == src] = (dst[dst == src] + 1) % n
    g = oracle.Graph(n, src, dst)
    x, _ = g.pagerank(0.0, 1)
    assert np.array_equal(x, np.bincount(dst, minlength=n).astype(np.float64))


# ---------------------------------------------------------------- triangles
def test_triangles_golden():
    gd = _golden("triangles_tiny.json")
    g = oracle.Graph(gd["n"], np.array(gd["src"], np.int32), np.array(gd["dst"], np.int32),
                     flags=CLEAN | oracle.SYMMETRIZE | oracle.ORIENT_BY_DEGREE)
    pv, tot = g.triangle_count()
    assert tot == gd["total"]
    assert pv.tolist() == gd["per_vertex_incident"]


@pytest.mark.parametrize("seed", range(5))
def test_triangles_brute_force(seed):
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(3, 45))
    src, dst = _random_graph(rng, n, int(rng.integers(n, 6 * n)))
    adj = np.zeros((n, n), bool)
    for a, b in zip(src, dst):
        if a != b:
            adj[a, b] = adj[b, a] = True
    brute_total = 0
    brute_pv = np.zeros(n, np.int64)
    for u, v, w in itertools.combinations(range(n), 3):  # u < v < w, Section 3.IV
        if adj[u, v] and adj[v, w] and adj[u, w]:
            brute_total += 1
            brute_pv[[u, v, w]] += 1
    g = oracle.Graph(n, src, dst, flags=CLEAN | oracle.SYMMETRIZE | oracle.ORIENT_BY_DEGREE)
    pv, tot = g.triangle_count()
    assert tot == brute_total
    assert np.array_equal(pv.astype(np.int64), brute_pv)
    assert int(pv.sum()) == 3 * tot


def test_triangles_networkx_per_vertex():
    nx = pytest.importorskip("networkx")
    n, src, dst = synth.rmat(9, 8, synth.RMAT_PARAMS["triangle"])
    g = oracle.Graph(n, src, dst, flags=CLEAN | oracle.SYMMETRIZE | oracle.ORIENT_BY_DEGREE)
    pv, tot = g.triangle_count()
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from((a, b) for a, b in zip(src.tolist(), dst.tolist()) if a != b)
    t = nx.triangles(G)
    assert pv.tolist() == [t[v] for v in range(n)]
    assert tot == sum(t.values()) // 3


@pytest.mark.parametrize("k", [3, 4, 7, 12])
def test_triangles_complete_graph(k):
    pairs = np.array([(a, b) for a in range(k) for b in range(k) if a < b], np.int32).reshape(-1, 2)
    g = oracle.Graph(k, pairs[:, 0], pairs[:, 1], flags=CLEAN | oracle.SYMMETRIZE | oracle.ORIENT_BY_DEGREE)
    pv, tot = g.triangle_count()
    assert tot == math.comb(k, 3)
    assert np.all(pv == math.comb(k - 1, 2))


def test_triangles_bipartite_is_zero():
    rng = np.random.default_rng(9)
    src = rng.integers(0, 20, 300).astype(np.int32)
    dst = rng.integers(20, 45, 300).astype(np.int32)
    g = oracle.Graph(45, src, dst, flags=CLEAN | oracle.SYMMETRIZE | oracle.ORIENT_BY_DEGREE)
    pv, tot = g.triangle_count()
    assert tot == 0 and not pv.any()


# ---------------------------------------------------------------- CF
def test_cf_golden_hand_step():
    gd = _golden("cf_k1_tiny.json")
    g = oracle.Graph(gd["n"], np.array(gd["src"], np.int32), np.array(gd["dst"], np.int32),
                     np.array(gd["rating"], np.uint32))
    p0 = np.array(gd["p0"]).reshape(gd["n"], gd["K"])
    p1, trace = g.cf_gd(gd["K"], gd["lambda"], gd["gamma"], 1, p0)
    np.testing.assert_allclose(p1.ravel(), gd["p1"], rtol=0, atol=1e-15)
    assert trace[0] == pytest.approx(gd["loss0"], abs=1e-15)


def _bipartite(rng, nu, ni, m):
    u = rng.integers(0, nu, m).astype(np.int32)
    v = rng.integers(nu, nu + ni, m).astype(np.int32)
    r = rng.integers(1, 6, m).astype(np.uint32)
    return u, v, r


def test_cf_step_is_half_gradient_of_loss():
    """Eqs. 3-5 move every factor by -gamma/2 times the gradient of the Eq. 2 loss
    (regulariser once per vertex); checked with central differences."""
    rng = np.random.default_rng(11)
    nu, ni, K, lam = 7, 5, 3, 0.05
    u, v, r = _bipartite(rng, nu, ni, 25)
    g = oracle.Graph(nu + ni, u, v, r)
    p0 = rng.normal(0, 0.5, (nu + ni, K))
    gamma = 1e-3
    p1, _ = g.cf_gd(K, lam, gamma, 1, p0)
    step = (p1 - p0) / gamma
    h = 1e-6
    grad = np.zeros_like(p0)
    for i in range(p0.shape[0]):
        for k in range(K):
            pp = p0.copy(); pp[i, k] += h
            pm = p0.copy(); pm[i, k] -= h
            grad[i, k] = (g.cf_loss(K, lam, pp) - g.cf_loss(K, lam, pm)) / (2 * h)
    np.testing.assert_allclose(step, -0.5 * grad, rtol=1e-6, atol=1e-7)


def test_cf_vertex_step_matches_full_step():
    rng = np.random.default_rng(13)
    nu, ni, K = 15, 9, 4
    u, v, r = _bipartite(rng, nu, ni, 80)
    g = oracle.Graph(nu + ni, u, v, r)
    p0 = rng.normal(0, 0.3, (nu + ni, K))
    p1, _ = g.cf_gd(K, 0.05, 0.01, 1, p0)
    for vert in range(nu + ni):
        np.testing.assert_allclose(g.cf_vertex_step(K, 0.05, 0.01, p0, vert), p1[vert], rtol=1e-13, atol=1e-15)


def test_cf_loss_decreases_at_small_step():
    rng = np.random.default_rng(12)
    nu, ni, K = 60, 20, 8
    u, v, r = _bipartite(rng, nu, ni, 600)
    g = oracle.Graph(nu + ni, u, v, r)
    p0 = oracle.cf_init(nu + ni, K, seed=3)
    _, trace = g.cf_gd(K, 0.05, 1e-3, 20, p0)
    assert np.all(np.diff(trace) < 0)


def test_cf_init_normal_moments():
    p = oracle.cf_init(4000, 32, seed=1, sigma=0.1).ravel()
    assert abs(p.mean()) < 3 * 0.1 / math.sqrt(p.size)
    assert abs(p.std() - 0.1) < 0.002
    assert np.array_equal(p[:64], oracle.cf_init(2, 32, seed=1).ravel())


# ---------------------------------------------------------------- CF by SGD
@pytest.mark.parametrize("case", range(2))
def test_cf_sgd_golden_hand_steps(case):
    gd = _golden("cf_sgd_tiny.json")["cases"][case]
    g = oracle.Graph(gd["n"], np.array(gd["src"], np.int32), np.array(gd["dst"], np.int32),
                     np.array(gd["rating"], np.uint32))
    p0 = np.array(gd["p0"]).reshape(gd["n"], gd["K"])
    p1 = g.cf_sgd(gd["K"], gd["lambda"], gd["gamma"], 1, gd["n_left"], gd["P"], p0)
    np.testing.assert_allclose(p1.ravel(), gd["p1"], rtol=0, atol=1e-15)


def _perfect_matching(rng, n_pairs):
    u = np.arange(n_pairs, dtype=np.int32)
    v = (n_pairs + rng.permutation(n_pairs)).astype(np.int32)
    r = rng.integers(1, 6, n_pairs).astype(np.uint32)
    return u, v, r


@pytest.mark.parametrize("P", [1, 2, 3, 7, 64])
def test_cf_sgd_epoch_on_a_perfect_matching_is_one_gd_step(P):
    """When every user and every item has exactly one rating, no two updates
    touch the same vector: one SGD epoch in any order is one Jacobi GD step of
    Eqs. 3-5 (regulariser once per vertex = once per rating)."""
    rng = np.random.default_rng(21)
    n_pairs, K = 40, 5
    u, v, r = _perfect_matching(rng, n_pairs)
    g = oracle.Graph(2 * n_pairs, u, v, r)
    p0 = rng.normal(0, 0.5, (2 * n_pairs, K))
    gd, _ = g.cf_gd(K, 0.05, 0.02, 1, p0)
    sgd = g.cf_sgd(K, 0.05, 0.02, 1, n_pairs, P, p0)
    np.testing.assert_allclose(sgd, gd, rtol=1e-14, atol=1e-15)


def test_cf_sgd_epoch_is_gd_step_to_first_order_in_gamma():
    """With lambda = 0, an epoch applies every rating's gradient once: it differs
    from one GD step by O(gamma^2) (a dropped or doubled rating would leave an
    O(gamma) gap)."""
    rng = np.random.default_rng(22)
    nu, ni, K = 12, 6, 4
    u, v, r = _bipartite(rng, nu, ni, 50)
    g = oracle.Graph(nu + ni, u, v, r)
    p0 = rng.normal(0, 0.5, (nu + ni, K))
    gaps = []
    for gamma in (1e-3, 5e-4, 2.5e-4):
        gd, _ = g.cf_gd(K, 0.0, gamma, 1, p0)
        sgd = g.cf_sgd(K, 0.0, gamma, 1, nu, 5, p0)
        gaps.append(np.abs(sgd - gd).max())
    assert gaps[0] > 0
    for a, b in zip(gaps, gaps[1:]):
        assert 3.5 < a / b < 4.5


@pytest.mark.parametrize("P", [3, 5])
def test_cf_sgd_visits_ratings_in_the_stratified_order(P):
    """Every user rates one item and items are shared, so the result depends on
    the order.  The order is enumerated here by nested loops (stratum, then user
    block, then edge-list position); relabelling the users in that order and
    running with P = 1 (plain edge-list order) must give the same factors."""
    rng = np.random.default_rng(25)
    nu, ni, K = 40, 6, 3
    u = np.arange(nu, dtype=np.int32)
    v = rng.integers(nu, nu + ni, nu).astype(np.int32)
    r = rng.integers(1, 6, nu).astype(np.uint32)
    g = oracle.Graph(nu + ni, u, v, r)
    p0 = rng.normal(0, 0.5, (nu + ni, K))
    want = g.cf_sgd(K, 0.05, 0.05, 1, nu, P, p0)
    order = [e for s in range(P) for b in range(P) for e in range(nu)
             if u[e] % P == b and (v[e] - nu) % P == (b + s) % P]
    assert sorted(order) == list(range(nu))
    label = np.empty(nu, np.int32)
    label[order] = np.arange(nu)  # the rating of user order[i] becomes user i's
    g2 = oracle.Graph(nu + ni, label, v, r)
    p0_2 = p0.copy()
    p0_2[label] = p0[:nu]
    got = g2.cf_sgd(K, 0.05, 0.05, 1, nu, 1, p0_2)
    np.testing.assert_array_equal(got[label], want[:nu])
    np.testing.assert_array_equal(got[nu:], want[nu:])
    assert not np.array_equal(want, g.cf_sgd(K, 0.05, 0.05, 1, nu, 1, p0))


@pytest.mark.parametrize("P", [2, 5, 16])
def test_cf_sgd_strata_blocks_are_disjoint(P):
    """The blocks of one stratum share no user and no item, so the blocks of a
    stratum may run at the same time and give the serial order's result."""
    rng = np.random.default_rng(23)
    nu, ni = 50, 30
    u, v, _ = _bipartite(rng, nu, ni, 400)
    bu, bv = u % P, (v - nu) % P
    stratum = (bv - bu) % P
    for s in range(P):
        sel = stratum == s
        for b in range(P):
            mine = sel & (bu == b)
            other = sel & (bu != b)
            assert not np.isin(u[mine], u[other]).any()
            assert not np.isin(v[mine], v[other]).any()


def test_cf_sgd_fits_a_rank_one_matrix():
    """Fully observed rank-1 ratings G_uv = a_u b_v, K = 1, lambda = 0: SGD at a
    small step drives the Eq. 2 loss towards 0."""
    a = np.array([1, 2, 3, 2])
    b = np.array([2, 1, 3])
    uu, vv = np.meshgrid(np.arange(4), np.arange(3), indexing="ij")
    g = oracle.Graph(7, uu.ravel().astype(np.int32), (4 + vv.ravel()).astype(np.int32),
                     (a[uu] * b[vv]).ravel().astype(np.uint32))
    p0 = np.full((7, 1), 1.0)
    loss0 = g.cf_loss(1, 0.0, p0)
    p = g.cf_sgd(1, 0.0, 0.01, 400, 4, 3, p0)
    assert g.cf_loss(1, 0.0, p) < 1e-6 * loss0


def test_cf_sgd_epochs_compose_and_arguments_are_checked():
    rng = np.random.default_rng(24)
    nu, ni, K = 10, 8, 3
    u, v, r = _bipartite(rng, nu, ni, 60)
    g = oracle.Graph(nu + ni, u, v, r)
    p0 = rng.normal(0, 0.3, (nu + ni, K))
    two = g.cf_sgd(K, 0.05, 0.01, 2, nu, 4, p0)
    np.testing.assert_array_equal(two, g.cf_sgd(K, 0.05, 0.01, 1, nu, 4, g.cf_sgd(K, 0.05, 0.01, 1, nu, 4, p0)))
    with pytest.raises(ValueError):
        g.cf_sgd(K, 0.05, 0.01, 1, nu, 0, p0)
    with pytest.raises(ValueError):
        g.cf_sgd(K, 0.05, 0.01, 1, nu - 1, 4, p0)  # a user would be an item
    empty = oracle.Graph(nu + ni, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    np.testing.assert_array_equal(empty.cf_sgd(K, 0.05, 0.01, 3, nu, 4, p0), p0)  # no rating, no update


# ---------------------------------------------------------------- weighted PageRank
@pytest.mark.parametrize("seed", range(3))
def test_wpr_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(500 + seed)
    n = 12
    src, dst = _random_graph(rng, n, 40)
    g = oracle.Graph(n, src, dst)
    w = rng.uniform(0.5, 1.5, g.m)
    tau = rng.uniform(0.5, 1.5, n)
    grad, loss = g.wpr_gradient(w, tau, 0.15, 30)
    _, loss_f = g.wpr_forward(w, tau, 0.15, 30)
    assert loss == pytest.approx(loss_f, rel=1e-14)
    h = 1e-6
    fd = np.empty(g.m)
    for e in range(g.m):
        wp = w.copy(); wp[e] += h
        wm = w.copy(); wm[e] -= h
        fd[e] = (g.wpr_forward(wp, tau, 0.15, 30)[1] - g.wpr_forward(wm, tau, 0.15, 30)[1]) / (2 * h)
    scale = max(np.abs(fd).max(), 1e-12)
    assert np.all(np.abs(grad - fd) <= 1e-6 * scale + 1e-9)


def test_wpr_uniform_weights_is_pagerank():
    n, src, dst = synth.rmat(8, 8)
    g = oracle.Graph(n, src, dst)
    x_pr, _ = g.pagerank(0.15, 30)
    x_w, _ = g.wpr_forward(np.full(g.m, 0.7), np.zeros(n), 0.15, 30)
    np.testing.assert_allclose(x_w, x_pr, rtol=1e-13)


# ---- connected components by label propagation (a program outside the paper's five) ----

@pytest.mark.parametrize("seed", range(4))
def test_components_match_scipy_on_symmetrised_graphs(seed):
    """On a symmetrised graph the label of v is the smallest id in its connected
    component (scipy's weak components)."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(5, 400))
    s, d = _random_graph(rng, n, int(rng.integers(0, 2 * n)))
    g = oracle.Graph(n, s, d, flags=CLEAN | oracle.SYMMETRIZE)
    lab, _ = g.connected_components()
    cs, cd, _ = g.edges()
    A = sp.csr_matrix((np.ones(len(cs)), (cs, cd)), shape=(n, n))
    ncomp, comp = csg.connected_components(A, directed=False)
    smallest = np.full(ncomp, n, np.int64)
    np.minimum.at(smallest, comp, np.arange(n))
    assert np.array_equal(lab.astype(np.int64), smallest[comp])


@pytest.mark.parametrize("seed", range(4))
def test_components_directed_brute_force(seed):
    """On a directed graph the label of v is the smallest id of any vertex with a
    path to v (v included): brute force by a BFS from every vertex."""
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(3, 40))
    s, d = _random_graph(rng, n, int(rng.integers(0, 3 * n)))
    g = oracle.Graph(n, s, d, flags=CLEAN)
    lab, _ = g.connected_components()
    adj = [[] for _ in range(n)]
    for a, b in zip(s.tolist(), d.tolist()):
        adj[a].append(b)
    want = np.arange(n)
    for u in range(n):
        seen, stack = {u}, [u]
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if y not in seen:
                    seen.add(y)
                    stack.append(y)
        for v in seen:
            want[v] = min(want[v], u)
    assert np.array_equal(lab.astype(np.int64), want)


@pytest.mark.parametrize("n", [2, 7, 30])
def test_components_path_superstep_count(n):
    """A symmetric path 0 - 1 - ... - n-1: the label 0 needs n-1 supersteps to
    reach the far end, and one more superstep finds no change: n in all."""
    s = np.arange(n - 1, dtype=np.int32)
    g = oracle.Graph(n, s, s + 1, flags=CLEAN | oracle.SYMMETRIZE)
    lab, it = g.connected_components()
    assert lab.tolist() == [0] * n and it == n


def test_components_without_edges():
    g = oracle.Graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    lab, it = g.connected_components()
    assert lab.tolist() == list(range(5)) and it == 1
