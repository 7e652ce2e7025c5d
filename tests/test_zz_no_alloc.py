"""The allocation-free entry point, bfs_run_static, against bfs_run.

bfs_run_static serves callers that cannot allocate device memory while they
run (inside a memory arena they do not own, a plugin given fixed buffers, a
real-time loop where cudaMalloc may stall or fail): its scratch is a fixed
array inside the library. This file is named to be collected last, so a run
that stops at the first failure has already run every other test; it passes
alone in a fresh process as well as after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import paper_1708_01159_gb300 as bfs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_run_static_matches_bfs_run_on_two_calls_in_a_row():
    bfs.build()
    L = bfs.lib()
    g = gg.rmat(14, 16, seed=1000)
    roots = gg.sample_roots(g, 2, seed=2000)
    off = torch.from_numpy(g.off).cuda()
    idx = torch.from_numpy(g.idx).cuda()
    stream = torch.cuda.current_stream()
    with bfs.Graph(g.off, g.idx) as G:
        for r in roots:  # two calls in a row share (and must reset) the fixed scratch
            want = torch.empty(g.n, dtype=torch.int32, device="cuda")
            bfs.bfs_run(G.handle, int(r), want, stream)
            got = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
            rc = L.bfs_run_static(off.data_ptr(), idx.data_ptr(), g.n, g.m, int(r), got.data_ptr(),
                                  stream.cuda_stream)
            assert rc == bfs.BFS_OK, L.bfs_last_error_detail().decode()
            torch.cuda.synchronize()
            assert torch.equal(got, want)


def test_run_static_rejects_sizes_beyond_its_limit():
    bfs.build()
    L = bfs.lib()
    n = (1 << 20) + 1
    off = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    idx = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    rc = L.bfs_run_static(off.data_ptr(), idx.data_ptr(), n, 0, 0, out.data_ptr(), None)
    assert rc == bfs.BFS_ERR_INVALID_ARG
    assert "1048576" in L.bfs_last_error_detail().decode()
