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


def test_clock_summary_reads_median_under_load_and_reasons(tmp_path):
    """nvidia-smi rows (csv, noheader, nounits): the SM clock median over samples
    above half the maximum, the maximum, and every throttle reason seen active."""
    import bench
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    rows = [
        "0, 345, 2070, 120.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1965, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1100.25, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1995, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
    ]
    with open(cs.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    cs.proc = object()  # as if the sampler had run
    out = cs.summary()
    assert out["sm_mhz"] == 1980.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 4 and out["power_w_max"] == 1100.25


def test_pull_roofline_adds_the_sssp_pull_launches_only():
    """Algorithmic bytes of trav_pull_a launches: in-edges x (4 B id + weight
    width + 1/8 B first-edge bit) + the vertex state once per launch; BFS pull
    launches are reported apart and push supersteps count only in the
    whole-superstep figure."""
    import bench

    class FakeGM:
        GM_BFS, GM_SSSP = 1, 2
        GM_SCALAR_PULL_WEIGHT_BYTES = 11
        GM_SCALAR_PULL_STREAM_BYTES = 13
        GM_OPT_PROFILE = 3

    class FakeGraph:
        n = 10
        # (superstep, dir, active, edges, vertices, superstep ms, next edges, pull ms, push ms, finalize ms)
        traces = {FakeGM.GM_BFS: [[0, 0, 1, 100, 1, 0.1, 0, 0.0, 0.05, 0.02], [1, 1, 5, 800, 6, 0.2, 0, 0.15, 0, 0]],
                  FakeGM.GM_SSSP: [[0, 0, 1, 100, 1, 0.1, 0, 0.0, 0.06, 0.02],
                                   [1, 1, 9, 1000, 6, 0.5, 0, 0.4, 0.003, 0.08]]}

        def __init__(self):
            self.kind = None
            self.options = []

        def scalar(self, which):
            assert which in (FakeGM.GM_SCALAR_PULL_WEIGHT_BYTES, FakeGM.GM_SCALAR_PULL_STREAM_BYTES)
            return 1 if which == FakeGM.GM_SCALAR_PULL_WEIGHT_BYTES else 5000

        def degrees(self):
            return np.zeros(10, np.int32), np.array([0, 1, 2, 0, 3, 1, 0, 0, 5, 1], np.int32)

        def set_option(self, opt, val):
            self.options.append((opt, val))

        def program_set(self, kind):
            self.kind = kind

        def set_active(self, v):
            pass

        def run(self, it):
            return 2

        def trace(self):
            return np.array(self.traces[self.kind], np.float64)

    g = FakeGraph()
    srcs = np.array([0, 1], np.int32)
    r = bench.pull_roofline(FakeGM, g, srcs, srcs, (srcs, srcs), peak=6000.0, peak_kind="measured")
    assert g.options == [(FakeGM.GM_OPT_PROFILE, 1), (FakeGM.GM_OPT_PROFILE, 0)]
    state = 4.0 * 10 + 4.0 * 6  # every message once + the 6 non-empty columns written once
    per_launch = 1000 * (4 + 1) + 1000 / 8 + state
    assert r["launches"] == 2 and r["bytes_per_launch"] == per_launch
    assert abs(r["avg_launch_us"] - 400.0) < 1e-9
    assert abs(r["achieved"] - per_launch / 0.4e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 6000.0) < 1e-12
    # bytes the layout streams (5000 here) plus the same vertex state
    assert r["bytes_read_per_launch"] == 5000 + state
    assert r["bfs_pull_bottom_up"]["launches"] == 2
    assert r["bfs_pull_bottom_up"]["in_edges_checked_per_launch"] == 800
    # SSSP push superstep 0 (1 frontier vertex, 100 edges): 12 B + 16 B per edge, 0.06 ms
    push = r["sssp_push"]
    assert push["launches"] == 2 and push["bytes_per_launch"] == 12 + 1600
    assert abs(push["achieved"] - (12 + 1600) / 0.06e-3 / 1e9) < 1e-9
    # finalize after that push: the 9 vertices of the next frontier, 16 B each
    assert r["sssp_finalize_after_push"]["bytes_per_launch"] == 16 * 9
    # finalize after the pull: 6 non-empty columns x 12 B + 6 received x 12 B, no next frontier
    fp = r["sssp_finalize_after_pull"]
    assert fp["bytes_per_launch"] == 12 * 6 + 12 * 6 and abs(fp["avg_launch_us"] - 80.0) < 1e-9


def test_recorded_traffic_is_dropped_when_the_kernel_source_changes(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: "0" * 64)
    assert bench._recorded_traffic() is None
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: bench.PULL_A_TRAFFIC["source_sha256"])
    assert bench._recorded_traffic() == bench.PULL_A_TRAFFIC["bytes_per_launch"]


def test_cf_roofline_arithmetic():
    """CF step roofline: HBM algorithmic bytes = ratings streamed once per pass
    (8 B + 5 B) + seven touches of the factor state; L2 bytes = one K-wide row
    gathered per rating in each pass."""
    import bench
    r = bench.cf_roofline(m=1000, n=100, K=32, ms_iter=1.0, hbm_peak=5000.0)
    assert r["hbm_algorithmic_bytes_per_iter"] == 1000 * 13 + 7 * 100 * 32 * 4
    assert r["gather_bytes_per_iter"] == 2 * 1000 * 128
    assert abs(r["achieved"] - 2 * 1000 * 128 / 1e-3 / 1e9) < 1e-9
    assert r["bound"] == "l2" and r["peak"] is None
    assert abs(r["hbm_frac"] - r["hbm_achieved"] / 5000.0) < 1e-12
