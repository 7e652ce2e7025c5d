"""Serving loop (continuous batching over resident graphs): every query's result
equals the same query run alone, whatever else shares the GPU; admission
respects the memory budget; shutdown cancels what never ran. Depths are
integers: the tolerance is zero."""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1708_01159_gb300 as bfs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def graphs():
    bfs.build()
    gs = [gg.rmat(14, 16, seed=501), gg.grid(120, 90, 0.1, seed=502), gg.erdos_renyi(30000, 6.0, seed=503),
          gg.rmat(12, 8, seed=504, permute=True)]
    Gs = [bfs.Graph(g.off, g.idx) for g in gs]
    yield gs, Gs
    for G in Gs:
        G.close()


def alone(G, n, root):
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    bfs.bfs_run(G.handle, int(root), d)
    torch.cuda.synchronize()
    return d.cpu().numpy()


@pytest.mark.parametrize("merge,policy", [(0, 0), (16, 1), (16, 0)])
def test_mixed_results_equal_alone(graphs, merge, policy):
    """policy 1 merges wherever it can; policy 0 merges only graphs whose
    registration probe found waves cheaper (each graph's query block count is
    probed too): either way every result equals the query run alone."""
    gs, Gs = graphs
    rng = np.random.default_rng(7 + merge + policy)
    s = bfs.bfs_serve_create(max_inflight=12, num_streams=6, merge_batch=merge, merge_policy=policy)
    try:
        ids = [bfs.bfs_serve_add_graph(s, G.handle) for G in Gs]
        plan = []
        for q in range(240):
            gi = int(rng.integers(0, len(gs)))
            root = int(gg.sample_roots(gs[gi], 1, seed=1000 + q)[0])
            plan.append((gi, root, torch.full((gs[gi].n,), -7, dtype=torch.int32, device="cuda")))
        # the server's streams do not wait on the caller's: buffers must be ready when submitted
        torch.cuda.synchronize()
        jobs = [(gi, root, out, bfs.bfs_serve_submit(s, ids[gi], root, out)) for gi, root, out in plan]
        for gi, root, out, t in jobs:
            assert bfs.bfs_serve_wait(s, t) == bfs.BFS_OK
        torch.cuda.synchronize()
        for gi, root, out, t in jobs:
            assert np.array_equal(out.cpu().numpy(), alone(Gs[gi], gs[gi].n, root))
        # a sample also against the oracle
        for gi, root, out, t in jobs[:12]:
            assert np.array_equal(out.cpu().numpy(), oracle.bfs(gs[gi].off, gs[gi].idx, root).depth)
        st = bfs.bfs_serve_stats(s)
        assert st["completed"] == 240 and st["failed"] == 0 and st["admitted"] == 240
        assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"] and st["qps"] > 0 and st["gteps"] > 0
        assert 0 <= st["wait_p50_ms"] <= st["wait_p99_ms"] <= st["max_ms"]
        if merge and policy == 1:
            assert st["merged_waves"] >= 1
        for gi in ids:
            shape = bfs.bfs_serve_graph_shape(s, gi)
            assert 1 <= shape["query_blocks"] <= 8 * torch.cuda.get_device_properties(0).multi_processor_count
        with pytest.raises(bfs.BFSError):
            bfs.bfs_serve_graph_shape(s, len(ids))
        for _, _, _, t in jobs[:3]:
            assert bfs.bfs_serve_poll(s, t) == (0, bfs.BFS_OK)
    finally:
        bfs.bfs_serve_destroy(s)


def test_memory_budget_admission(graphs):
    """Admission by memory: with a budget that fits two of the largest queries at
    once, the memory held by admitted queries never exceeds it, although the
    slot limit alone would admit eight."""
    gs, Gs = graphs
    probe = bfs.bfs_serve_create(max_inflight=1, num_streams=1)
    try:
        need = [bfs.bfs_serve_query_bytes(probe, bfs.bfs_serve_add_graph(probe, G.handle)) for G in Gs]
    finally:
        bfs.bfs_serve_destroy(probe)
    budget = 2 * max(need) + 1
    s = bfs.bfs_serve_create(mem_budget_bytes=budget, max_inflight=8, num_streams=4)
    try:
        ids = [bfs.bfs_serve_add_graph(s, G.handle) for G in Gs]
        assert [bfs.bfs_serve_query_bytes(s, i) for i in ids] == need
        assert all(bfs.bfs_serve_query_bytes(s, i, with_output=True) < need[k] for k, i in enumerate(ids))
        tickets = []
        for q in range(40):
            gi = q % len(gs)
            tickets.append(bfs.bfs_serve_submit(s, ids[gi], int(gg.sample_roots(gs[gi], 1, seed=q)[0])))
        for t in tickets:
            assert bfs.bfs_serve_wait(s, t) == bfs.BFS_OK
        st = bfs.bfs_serve_stats(s)
        assert st["completed"] == 40
        assert min(need) <= st["peak_bytes_inflight"] <= budget
        with pytest.raises(bfs.BFSError) as e:
            bfs.bfs_serve_query_bytes(s, len(ids))
        assert e.value.code == bfs.BFS_ERR_NOT_FOUND
    finally:
        bfs.bfs_serve_destroy(s)


def test_over_budget_query_runs_alone_and_shutdown_cancels(graphs):
    gs, Gs = graphs
    s = bfs.bfs_serve_create(mem_budget_bytes=1, max_inflight=1, num_streams=1, queue_capacity=4)
    try:
        gid = bfs.bfs_serve_add_graph(s, Gs[0].handle)
        root = int(gg.sample_roots(gs[0], 1, seed=3)[0])
        t = bfs.bfs_serve_submit(s, gid, root)
        assert bfs.bfs_serve_wait(s, t, 10_000_000) == bfs.BFS_OK  # larger than the budget: runs when idle
        with pytest.raises(bfs.BFSError) as e:
            bfs.bfs_serve_submit(s, 99, root)
        assert e.value.code == bfs.BFS_ERR_NOT_FOUND
        with pytest.raises(bfs.BFSError):
            bfs.bfs_serve_poll(s, 123456789)
        # fill the queue faster than one slot drains it: some submissions are refused
        accepted, busy = [], 0
        for q in range(64):
            try:
                accepted.append(bfs.bfs_serve_submit(s, gid, root))
            except bfs.BFSError as err:
                assert err.code == bfs.BFS_ERR_BUSY
                busy += 1
        assert bfs.bfs_serve_stats(s)["rejected"] == busy
    finally:
        bfs.bfs_serve_destroy(s)  # running queries finish, queued ones are cancelled


def test_wait_timeout():
    bfs.build()
    g = gg.grid(400, 400, 0.1, seed=9)  # hundreds of levels: a query takes a while
    with bfs.Graph(g.off, g.idx) as G:
        s = bfs.bfs_serve_create(max_inflight=1, num_streams=1)
        try:
            gid = bfs.bfs_serve_add_graph(s, G.handle)
            r = int(gg.sample_roots(g, 1, seed=1, giant=True)[0])
            ts = [bfs.bfs_serve_submit(s, gid, r) for _ in range(8)]
            assert bfs.bfs_serve_wait(s, ts[-1], 0) == bfs.BFS_ERR_TIMEOUT
            for t in ts:
                assert bfs.bfs_serve_wait(s, t) == bfs.BFS_OK
        finally:
            bfs.bfs_serve_destroy(s)


def test_cancel_queued_and_stats_window():
    """Load shedding cancels exactly the queries not yet admitted; running ones
    finish; a statistics reset starts a new window."""
    bfs.build()
    g = gg.grid(400, 400, 0.1, seed=9)  # hundreds of levels: a query takes a while
    with bfs.Graph(g.off, g.idx) as G:
        s = bfs.bfs_serve_create(max_inflight=1, num_streams=1)
        try:
            gid = bfs.bfs_serve_add_graph(s, G.handle)
            r = int(gg.sample_roots(g, 1, seed=1, giant=True)[0])
            ts = [bfs.bfs_serve_submit(s, gid, r) for _ in range(10)]
            k = bfs.bfs_serve_cancel_queued(s)
            assert 1 <= k <= 9  # at least one was admitted, the tail of the queue was not
            statuses = [bfs.bfs_serve_wait(s, t) for t in ts]
            assert statuses.count(bfs.BFS_ERR_CANCELLED) == k
            assert statuses.count(bfs.BFS_OK) == 10 - k
            st = bfs.bfs_serve_stats(s)
            assert st["completed"] == 10 - k and st["submitted"] == 10
            bfs.bfs_serve_reset_stats(s)
            st = bfs.bfs_serve_stats(s)
            assert st["submitted"] == 0 and st["completed"] == 0 and st["p50_ms"] == 0
            t = bfs.bfs_serve_submit(s, gid, r)
            assert bfs.bfs_serve_wait(s, t) == bfs.BFS_OK
            st = bfs.bfs_serve_stats(s)
            assert st["submitted"] == 1 and st["completed"] == 1 and st["p50_ms"] > 0
        finally:
            bfs.bfs_serve_destroy(s)
