"""Seeded input generator (CPU only): determinism, shapes and distributions."""
import numpy as np

import synth


def test_rmat_deterministic_and_in_range():
    n, s1, d1 = synth.rmat(10, 16, seed=1)
    _, s2, d2 = synth.rmat(10, 16, seed=1)
    _, s3, _ = synth.rmat(10, 16, seed=2)
    assert n == 1024 and s1.shape == (16 * 1024,)
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)
    assert not np.array_equal(s1, s3)
    assert s1.min() >= 0 and s1.max() < n and d1.min() >= 0 and d1.max() < n


def test_rmat_quadrant_frequencies():
    a, b, c = synth.RMAT_PARAMS["graph500"]
    n, s, d = synth.rmat(12, 16)
    top_s = s >> 11  # most significant level
    top_d = d >> 11
    m = s.shape[0]
    freq = [np.mean((top_s == i) & (top_d == j)) for i, j in ((0, 0), (0, 1), (1, 0), (1, 1))]
    np.testing.assert_allclose(freq, [a, b, c, 1 - a - b - c], atol=4 / np.sqrt(m))


def test_weights_depend_only_on_endpoints():
    s = np.array([3, 5, 3, 9], np.int32)
    d = np.array([4, 6, 4, 1], np.int32)
    w = synth.edge_weights_u32(s, d, seed=7)
    assert w[0] == w[2]
    n, s, d = synth.rmat(12)
    w = synth.edge_weights_u32(s, d, seed=7)
    assert w.min() == 1 and w.max() == 255


def test_sources_are_distinct_and_non_isolated():
    n, s, d = synth.rmat(12)
    src = synth.pick_sources(n, s, d, 16, seed=3)
    assert len(set(src.tolist())) == 16
    has_out = np.zeros(n, bool)
    has_out[s[s != d]] = True
    assert has_out[src].all()


def test_chung_lu_bipartite_count_and_shape():
    nu, ni = 3000, 400
    target = 60000
    n, s, d, r = synth.chung_lu_bipartite(nu, ni, 1.1, target, seed=4)
    assert n == nu + ni
    assert abs(len(s) - target) < 6 * np.sqrt(target)
    assert s.min() >= 0 and s.max() < nu and d.min() >= nu and d.max() < n
    assert r.min() == 1 and r.max() == 5
    key = s.astype(np.int64) * n + d
    assert np.unique(key).size == key.size  # simple graph
    deg_u = np.bincount(s, minlength=nu)
    assert deg_u[:10].mean() > deg_u[-1000:].mean()


def test_uniform_f32_range():
    x = synth.uniform_f32(10000, seed=1, stream=0, lo=0.5, hi=1.5)
    assert x.min() >= 0.5 and x.max() < 1.5 and abs(x.mean() - 1.0) < 0.02
