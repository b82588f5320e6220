"""The closed form of an SGD window whose users are distinct (CPU).

Within such a window every user row keeps its value from before the window, so
with c = 1 - gamma lambda the row of an item before its t-th rating in the
window is c^k (v0 + gamma sum_s E_s a_s) over its earlier ratings s, with
E_s = e_s / c^(k_s + 1).  Then e_t = r_t - c^k_t (a_t.v0 + gamma sum_s (a_t.a_s) E_s)
needs only dot products that are independent of each other, plus a scalar
recurrence.  This is the identity a faster SGD kernel can use; here it is
checked against the oracle's serial SGD (Section 3.III: the updates of Eqs. 4-5
without their sums, rating by rating)."""
import numpy as np
import pytest

import oracle


def _closed_form_window(p, users, items, ratings, gamma, lam):
    p = p.copy()
    c = 1.0 - gamma * lam
    W = len(users)
    A = p[users].copy()
    v0 = {v: p[v].copy() for v in set(items)}
    k = np.zeros(W, int)
    seen = {}
    for t, v in enumerate(items):
        k[t] = seen.get(v, 0)
        seen[v] = k[t] + 1
    G = A @ A.T
    D = np.array([A[t] @ v0[items[t]] for t in range(W)])
    E = np.zeros(W)
    S = np.zeros(W)
    e = np.zeros(W)
    for t in range(W):  # the serial part: one scalar per rating
        e[t] = ratings[t] - c ** k[t] * (D[t] + gamma * S[t])
        E[t] = e[t] / c ** (k[t] + 1)
        for t2 in range(t + 1, W):
            if items[t2] == items[t]:
                S[t2] += G[t2, t] * E[t]
    for t in range(W):
        before = v0[items[t]] + gamma * sum(E[s] * A[s] for s in range(t) if items[s] == items[t])
        p[users[t]] = c * A[t] + gamma * e[t] * c ** k[t] * before
    for v in v0:
        p[v] = c ** seen[v] * (v0[v] + gamma * sum(E[s] * A[s] for s in range(W) if items[s] == v))
    return p


@pytest.mark.parametrize("seed", range(4))
def test_window_with_distinct_users_equals_serial_sgd(seed):
    rng = np.random.default_rng(seed)
    nu, ni, K, gamma, lam = 32, 4, 32, 1e-2, 0.05
    items = (nu + rng.choice([0, 0, 0, 1, 2, 3], nu)).astype(np.int32)  # one item takes about half
    r = rng.integers(1, 6, nu).astype(np.uint32)
    users = np.arange(nu, dtype=np.int32)  # one rating per user: edge-list order is user order
    g = oracle.Graph(nu + ni, users, items, r)
    p0 = rng.normal(0, 0.3, (nu + ni, K))
    want = g.cf_sgd(K, lam, gamma, 1, nu, 1, p0)
    got = _closed_form_window(p0, users, items, r.astype(np.float64), gamma, lam)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)
