#!/usr/bin/env python3
"""Benchmark: BFS and SSSP supersteps on a scale-22 RMAT graph on one GB300.

One step = 16 BFS + 16 SSSP queries (uint32 weights in [1, 255]) from seeded
non-isolated sources, run one at a time through the C ABI on a graph already
ingested into HBM (ingest is timed separately, as the paper excludes graph
load).  The metric is GTEPS = sum over queries of the edges of reached vertices
(Graph500 convention) / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own queries on
its own GPU (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SCALE, EDGE_FACTOR, N_QUERIES = 22, 16, 16
METRIC = "GTEPS plain vs batched/adjoint on 1 GB300 at oracle accuracy; HBM % of peak"
WORKLOAD = ("bfs16+sssp16 on RMAT scale 22, edge factor 16, a/b/c/d=.57/.19/.19/.05, "
            "self-loops and duplicates removed, uint32 weights in [1,255]")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out" if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else "",
                                 f".clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
            os.remove(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        smax = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [x for x in sm if x > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def make_workload(rank):
    import synth
    n, s, d = synth.rmat(SCALE, EDGE_FACTOR, synth.RMAT_PARAMS["graph500"], synth.BASE_SEED + 1)
    w = synth.edge_weights_u32(s, d, synth.BASE_SEED + 2)
    srcs = synth.pick_sources(n, s, d, 2 * N_QUERIES, seed=synth.BASE_SEED + 100 + rank)
    return n, s, d, w, srcs[:N_QUERIES], srcs[N_QUERIES:2 * N_QUERIES]


def run_queries(gm, g, bfs_src, sssp_src, src_dev, out_host=None):
    """One step: every query through the C ABI.  Returns edges traversed."""
    edges = 0
    for kind, srcs, dev in ((gm.GM_BFS, bfs_src, src_dev[0]), (gm.GM_SSSP, sssp_src, src_dev[1])):
        for i in range(len(srcs)):
            g.program_set(kind)
            g.set_active(dev[i:i + 1] if dev is not None else srcs[i:i + 1])
            g.run(-1)
            edges += g.scalar(gm.GM_SCALAR_REACHED_EDGES)
            if out_host is not None:
                g.state(out_host)
    return edges


def cpu_baseline(n, s, d, w, bfs_src, sssp_src, n_pairs=1):
    """The FP64 oracle as it stands (single thread) on a bounded sample."""
    import oracle
    og = oracle.Graph(n, s, d, w)
    t = 0.0
    edges = 0
    for i in range(n_pairs):
        t0 = time.perf_counter()
        dd, _ = og.bfs([bfs_src[i]])
        t += time.perf_counter() - t0
        edges += og.reached_edges(dd)
        t0 = time.perf_counter()
        dd, _ = og.sssp([sssp_src[i]])
        t += time.perf_counter() - t0
        edges += og.reached_edges(dd)
    return {"value": edges / t / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{n_pairs} BFS + {n_pairs} SSSP queries of the same scale-22 graph "
                      f"({t:.1f} s of single-thread FP64 oracle time; graph build excluded)"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n, s, d, w, bfs_src, sssp_src = make_workload(0)
    import oracle
    og = oracle.Graph(n, s, d, w)
    both = (args.steps + args.warmup) <= 20
    per = []
    edges_total, t_total = 0, 0.0
    for step in range(args.warmup + args.steps):
        i = step % N_QUERIES
        t0 = time.perf_counter()
        dd, _ = og.bfs([bfs_src[i]])
        e = og.reached_edges(dd)
        if both:
            dd, _ = og.sssp([sssp_src[i]])
            e += og.reached_edges(dd)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            edges_total += e
            t_total += dt
            per.append(dt)
    val = edges_total / t_total / 1e9
    sample = ("1 BFS + 1 SSSP query" if both else "1 BFS query") + " of the scale-22 workload per step"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle (oracle/)"},
            "cpu_baseline": {"value": val, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1)
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import __graft_entry__ as ge
    ge.build_cuda_library()
    import paper_1503_07241_gb300 as gm

    n, s, d, w, bfs_src, sssp_src = make_workload(rank)
    stream = torch.cuda.Stream()
    # ---- ingest (timed separately, excluded from the metric as in the paper) ----
    ts, td = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    tw = torch.from_numpy(w.view(np.int32)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = gm.Graph(n, ts, td, tw, stream=stream)
    ingest_s = time.perf_counter() - t0
    del ts, td, tw
    src_dev = (torch.from_numpy(bfs_src).cuda(), torch.from_numpy(sssp_src).cuda())

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    for _ in range(args.warmup):
        run_queries(gm, g, bfs_src, sssp_src, src_dev)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = gm.kernel_launch_count()
    edges = 0
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            edges += run_queries(gm, g, bfs_src, sssp_src, src_dev)
        ev1.record(stream)
        barrier()
    launches = gm.kernel_launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    tmax = ms
    edges_all = edges
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tmax = float(t.item())
        e = torch.tensor([float(edges)], device="cuda", dtype=torch.float64)
        dist.all_reduce(e)
        edges_all = float(e.item())
    value = edges_all / (tmax / 1e3) / 1e9

    # ---- dominant kernel: relax launches timed with CUDA events (profile mode) ----
    g.set_option(gm.GM_OPT_PROFILE, 1)
    relax_ms, relax_launches, scanned_e, scanned_v = 0.0, 0, 0, 0
    bytes_alg = 0.0
    for kind, srcs in ((gm.GM_BFS, bfs_src), (gm.GM_SSSP, sssp_src)):
        for i in range(len(srcs)):
            g.program_set(kind)
            g.set_active(src_dev[0 if kind == gm.GM_BFS else 1][i:i + 1])
            g.run(-1)
            relax_ms += g.scalar(gm.GM_SCALAR_RELAX_MS)
            relax_launches += g.scalar(gm.GM_SCALAR_RELAX_LAUNCHES)
            e = g.scalar(gm.GM_SCALAR_SCANNED_EDGES)
            v = g.scalar(gm.GM_SCALAR_PROCESSED_VERTICES)
            scanned_e += e
            scanned_v += v
            # algorithmic bytes: edge stream (int32 ids + uint32 weights for SSSP)
            # + per processed vertex an offset pair and a list/queue id
            bytes_alg += e * (4 + (4 if kind == gm.GM_SSSP else 0)) + v * 12
    g.set_option(gm.GM_OPT_PROFILE, 0)
    peak, peak_kind = _peaks()
    achieved = bytes_alg / (relax_ms / 1e3) / 1e9 if relax_ms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": None,
                "kernel": "trav_relax", "peak_source": peak_kind,
                "bytes_per_launch": bytes_alg / max(relax_launches, 1),
                "avg_launch_us": 1e3 * relax_ms / max(relax_launches, 1), "launches": relax_launches}

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(a).pin_memory()
        hs, hd, hw = pin(s), pin(d), pin(w.view(np.int32))
        out = torch.empty(n, dtype=torch.int32).pin_memory()
        barrier()
        t0 = time.perf_counter()
        e_edges = 0
        for _ in range(args.e2e_steps):
            g2 = gm.Graph(n, hs, hd, hw, stream=stream)
            e_edges += run_queries(gm, g2, bfs_src, sssp_src, (None, None), out_host=out)
            g2.close()
        barrier()
        e_t = time.perf_counter() - t0
        if dist:
            t = torch.tensor([e_t], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_t = float(t.item())
            e = torch.tensor([float(e_edges)], device="cuda", dtype=torch.float64)
            dist.all_reduce(e)
            e_edges = float(e.item())
        e2e = {"value": e_edges / e_t / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": int(s.nbytes + d.nbytes + w.nbytes + 8 * N_QUERIES),
               "d2h_bytes_per_step": int(2 * N_QUERIES * 4 * n), "steps": args.e2e_steps,
               "includes": "graph ingest from pinned host edge list + 32 queries + results to host"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n, s, d, w, bfs_src, sssp_src, n_pairs=1)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tmax / max(args.steps, 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": n, "m": g.m, "queries_per_step": 2 * N_QUERIES,
                           "ingest_ms": 1e3 * ingest_s, "l2": "inputs larger than L2 (CSR+CSC+weights ~1.05 GB)",
                           "parallelism": f"replicas{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
