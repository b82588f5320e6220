"""bench.py helpers that run on the host: the oracle's bounded SGD sample."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_cf_sgd_oracle_sample_counts_the_chosen_users():
    import bench
    import synth
    nu, ni = 3000, 500
    n, s, d, r = synth.chung_lu_bipartite(nu, ni, 1.1, 5e4, seed=9)
    order = np.lexsort((d, s))
    s, d, r = s[order], d[order], r[order]
    out = bench.cf_sgd_oracle_sample(s, d, r, nu, n, 8, lo=1000, count=500, K=8)
    want = int(((s >= 1000) & (s < 1500)).sum())
    assert want > 0
    assert out["kind"] == "oracle" and out["cores"] == 1 and out["unit"] == "ratings/s"
    assert out["value"] > 0
    assert f"the {want} ratings of users 1000..1499" in out["sample"]
