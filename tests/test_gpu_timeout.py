"""Bounded device-side waits, run out on purpose through the library's test
hook (bfs_debug_stall_next_launch): a grid barrier or level barrier that
expects one arrival more than the grid has, or a staged adjacency copy whose
barrier expects 16 bytes more than are copied. Every wait of the library gives
up after about 2 s, so nothing hangs and nothing faults: the kernel records
BFS_ERR_TIMEOUT in its status word, returns, and the host reports it. The next
launch on the same graph must then be exact again (the kernel resets the
barrier state a failed run leaves)."""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1708_01159_gb300 as bfs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    bfs.build()
    bfs.bfs_load_tree(None)
    yield
    bfs.bfs_debug_stall_next_launch(0)


def exact(G, g, root, **kw):
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    st = bfs.bfs_run_ex(G.handle, int(root), d, stats=True, mode=bfs.MODE_PERSISTENT, **kw)
    ref = oracle.bfs(g.off, g.idx, int(root))
    return np.array_equal(d.cpu().numpy(), ref.depth) and st["edges_reached"] == ref.edges_reached


def timed_out(fn):
    t0 = time.perf_counter()
    with pytest.raises(bfs.BFSError) as e:
        fn()
    dt = time.perf_counter() - t0
    assert e.value.code == bfs.BFS_ERR_TIMEOUT, str(e.value)
    assert dt < 30.0
    return dt


@pytest.mark.parametrize("mode", [1, 2])
def test_barrier_wait_runs_out_then_next_run_is_exact(mode):
    g = gg.rmat(13, 16, seed=41)
    roots = gg.sample_roots(g, 2, seed=42, giant=True)
    with bfs.Graph(g.off, g.idx) as G:
        assert exact(G, g, roots[0])
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        bfs.bfs_debug_stall_next_launch(mode)
        dt = timed_out(lambda: bfs.bfs_run_ex(G.handle, int(roots[1]), d, stats=True, mode=bfs.MODE_PERSISTENT))
        assert dt >= 1.0  # the wait ran to its limit
        for r in roots:
            assert exact(G, g, r)


def test_staged_copy_wait_runs_out_then_next_run_is_exact():
    # a hub of degree 5000: the CTA push streams its list through shared memory
    n = 5003
    s = np.concatenate([np.zeros(n - 3, np.int32), [n - 3, n - 2]]).astype(np.int32)
    t = np.concatenate([np.arange(1, n - 2, dtype=np.int32), [n - 2, n - 1]]).astype(np.int32)
    g = gg.from_edges(n, s, t, name="hub")
    with bfs.Graph(g.off, g.idx) as G:
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        bfs.bfs_debug_stall_next_launch(3)
        timed_out(lambda: bfs.bfs_run_ex(G.handle, 0, d, stats=True, mode=bfs.MODE_PERSISTENT,
                                         forced_variant=bfs.VARIANTS.index("push_cta")))
        assert exact(G, g, 0, forced_variant=bfs.VARIANTS.index("push_cta"))
        assert exact(G, g, n - 1)


def test_multi_source_barrier_wait_runs_out_then_next_wave_is_exact():
    g = gg.rmat(12, 16, seed=43)
    roots = gg.sample_roots(g, 64, seed=44)
    with bfs.Graph(g.off, g.idx) as G:
        out = torch.empty(64 * g.n, dtype=torch.int32, device="cuda")
        bfs.bfs_debug_stall_next_launch(1)
        timed_out(lambda: bfs.bfs_run_batch(G.handle, roots, out, edges=True))
        edges = bfs.bfs_run_batch(G.handle, roots, out, edges=True)
        D, E = oracle.bfs_batch(g.off, g.idx, roots)
        assert np.array_equal(out.cpu().numpy().reshape(64, g.n), D)
        assert np.array_equal(edges, E)
