"""bench.py's multi-process path on the CPU: two gloo ranks (127.0.0.1) combine
their numbers as the job's (slowest rank's time, all ranks' edges), and every rank
draws its own sources (independent queries: weak scaling, no data-path
collective)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, e = bench.combine_ranks(dist, [3.5, 7.25][rank], [1000, 2345][rank], "cpu")
    results[rank] = (t, e)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_time_and_edges():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, results)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert results[0] == results[1] == (7.25, 3345.0)


def test_one_process_passes_numbers_through():
    import bench
    assert bench.combine_ranks(None, 1.5, 42, "cpu") == (1.5, 42)


def test_ranks_draw_their_own_sources():
    import bench
    import synth
    n, s, d = synth.rmat(10, 16, synth.RMAT_PARAMS["graph500"], synth.BASE_SEED + 1)
    out_deg = np.bincount(s, minlength=n)
    per_rank = [bench.rank_sources(n, s, d, r, count=8) for r in range(2)]
    for bfs, sssp in per_rank:
        both = np.concatenate([bfs, sssp])
        assert len(both) == 16 and (out_deg[both] > 0).all()
    assert not np.array_equal(np.concatenate(per_rank[0]), np.concatenate(per_rank[1]))
