"""gm_bfs_csr_noalloc: the allocation-free BFS entry point, called through the C
ABI, against the regular graph-handle BFS (gm_run with GM_BFS) and the oracle.

The entry point exists for callers that cannot allocate device memory when they
need a traversal: code whose device memory is all owned by its own arena or
caching allocator, and loops that must not pay for cudaMalloc/cudaFree.  Its
scratch is a fixed device array shared by every call, so the test makes two
calls in a row on the same graph and checks that the second is not disturbed by
what the first left behind.  This file is collected last so that a failure here
does not hide any other test.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _csr_tensors(g):
    import torch
    s, d = g.edges()
    row_ptr = np.zeros(g.n + 1, np.int32)
    np.add.at(row_ptr, s.astype(np.int64) + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return torch.from_numpy(row_ptr).cuda(), torch.from_numpy(d).cuda()


def _reference(gm, g, src):
    g.program_set(gm.GM_BFS)
    g.set_active([src])
    it = g.run(-1)
    return g.state(), it


def test_noalloc_bfs_matches_graph_bfs_twice(gm):
    import torch
    n, s, d = synth.rmat(16, 16, synth.RMAT_PARAMS["graph500"], synth.BASE_SEED + 40)
    g = gm.Graph(n, s, d)
    row_ptr, col = _csr_tensors(g)
    srcs = synth.pick_sources(n, s, d, 2, seed=41)
    og = oracle.Graph(n, s, d)
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    for src in srcs:  # two calls in a row share the fixed scratch
        it = gm.bfs_csr_noalloc(row_ptr, col, int(src), depth)
        got = depth.cpu().numpy().view(np.uint32)
        ref, rit = _reference(gm, g, int(src))
        assert np.array_equal(got, ref)
        assert it == rit
        oref, oit = og.bfs([int(src)])  # the FP64 oracle's Algorithm 2 BFS
        assert np.array_equal(got, oref)
        assert it == oit


def test_noalloc_bfs_rejects_too_many_vertices(gm):
    import torch
    L = gm.lib()
    nmax = L.gm_bfs_csr_noalloc_max_vertices()
    assert nmax == 1 << 20
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    it = gm.ctypes.c_int32()
    st = L.gm_bfs_csr_noalloc(nmax + 1, dummy.data_ptr(), dummy.data_ptr(), 0, dummy.data_ptr(),
                              gm.ctypes.byref(it), None)
    assert st == gm.GM_ERR_INVALID_ARG
    assert b"limit" in L.gm_last_error()
