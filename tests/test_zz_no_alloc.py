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


def _static(g, root):
    off = torch.from_numpy(g.off).cuda()
    idx = torch.from_numpy(g.idx if g.m else np.zeros(1, np.int32)).cuda()
    out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
    rc = bfs.lib().bfs_run_static(off.data_ptr(), idx.data_ptr(), g.n, g.m, int(root), out.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rc, out.cpu().numpy()


def test_run_static_against_the_oracle_at_the_size_limit_and_after_it():
    """n = 1,048,576 exactly (a permuted 1024 x 1024 grid: the fixed queues at
    capacity, hundreds of levels), then a scale-10 R-MAT graph: the second call
    reuses the array the first one filled, and both equal the oracle."""
    import oracle
    bfs.build()
    big = gg.grid(1024, 1024, 0.1, seed=77)
    assert big.n == 1 << 20
    small = gg.rmat(10, 16, seed=78)
    for g, r in ((big, int(gg.sample_roots(big, 1, seed=79, giant=True)[0])),
                 (small, int(gg.sample_roots(small, 1, seed=80)[0]))):
        rc, got = _static(g, r)
        assert rc == bfs.BFS_OK, bfs.lib().bfs_last_error_detail().decode()
        assert np.array_equal(got, oracle.bfs(g.off, g.idx, r).depth)


def test_run_static_directed_graph_and_isolated_root():
    import oracle
    bfs.build()
    rng = np.random.default_rng(81)
    n = 3000
    g = gg.from_edges(n, rng.integers(0, n - 10, 9000), rng.integers(0, n - 10, 9000), symmetrize=False)
    iso = n - 1  # no edges reach or leave the last vertices
    for r in (int(gg.sample_roots(g, 1, seed=82)[0]), iso):
        rc, got = _static(g, r)
        assert rc == bfs.BFS_OK, bfs.lib().bfs_last_error_detail().decode()
        assert np.array_equal(got, oracle.bfs(g.off, g.idx, r).depth)
    rc, got = _static(g, iso)
    assert got[iso] == 0 and (np.delete(got, iso) == -1).all()


def test_run_static_rejects_a_malformed_csr_and_the_next_call_works():
    import oracle
    bfs.build()
    g = gg.rmat(11, 8, seed=83)
    bad_idx = g.idx.copy()
    bad_idx[len(bad_idx) // 2] = g.n  # one index out of range
    rc, _ = _static(gg.Graph(g.off, bad_idx), 0)
    assert rc == bfs.BFS_ERR_BAD_GRAPH
    bad_off = g.off.copy()
    bad_off[5], bad_off[6] = bad_off[6], bad_off[5] - 1  # offsets decreasing
    rc, _ = _static(gg.Graph(bad_off, g.idx), 0)
    assert rc == bfs.BFS_ERR_BAD_GRAPH
    r = int(gg.sample_roots(g, 1, seed=84)[0])
    rc, got = _static(g, r)
    assert rc == bfs.BFS_OK
    assert np.array_equal(got, oracle.bfs(g.off, g.idx, r).depth)
