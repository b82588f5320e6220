"""Writes cf_full_gamma_search.json: the FP64 oracle's Eq. 2 loss over ten Jacobi
gradient steps of Eqs. 3-5 on the 480,000 x 17,800 / ~1e8-rating workload
(K = 32, lambda = 0.05, initial factors N(0, 0.1) with seed 5) for the step sizes
1e-3, 1e-4, 1e-5 and 1e-6, and the largest of them at which the loss decreases
in every step.  Calls only the seeded generator and the oracle; takes a few
minutes (one process per step size).

    python tests/golden/make_cf_full_gamma_search.py
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

GAMMAS = (1e-3, 1e-4, 1e-5, 1e-6)
NU, NI, K, LAM, SEED, SIGMA, STEPS = 480_000, 17_800, 32, 0.05, 5, 0.1, 10


def loss_trace(gamma):
    import oracle
    import synth
    n, s, d, r = synth.chung_lu_bipartite(NU, NI, 1.1, 1e8, seed=synth.BASE_SEED + 2)
    og = oracle.Graph(n, s, d, r)
    p0 = oracle.cf_init(og.n, K, SEED, SIGMA)
    _, trace = og.cf_gd(K, LAM, gamma, STEPS, p0)
    return og.m, [float(x) for x in trace]


def main():
    with mp.get_context("spawn").Pool(len(GAMMAS)) as pool:
        res = pool.map(loss_trace, GAMMAS)
    rows = []
    for gamma, (m, tr) in zip(GAMMAS, res):
        t = np.array(tr)
        rows.append({"gamma": gamma, "loss": tr, "finite": bool(np.all(np.isfinite(t))),
                     "decreasing": bool(np.all(np.isfinite(t)) and np.all(np.diff(t) < 0))})
    chosen = max(r["gamma"] for r in rows if r["decreasing"])
    out = {"citation": "Eqs. 2-5 (gradient descent on the CF loss, regulariser once per vertex), Section 3.III; "
                       "reading: the largest power of ten <= 1e-3 at which the FP64 loss decreases in all 10 "
                       "steps is the step size of the full-workload parity check",
           "workload": {"users": NU, "items": NI, "ratings": res[0][0], "K": K, "lambda": LAM,
                        "init": f"N(0, {SIGMA}) seed {SEED}", "steps": STEPS},
           "runs": rows, "chosen_gamma": chosen}
    with open(os.path.join(HERE, "cf_full_gamma_search.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({"chosen_gamma": chosen}))


if __name__ == "__main__":
    main()
