"""GPU parity at the benchmark's full sizes for the multi-source batches and the
query server: every depth row the benchmark's launch configuration produces is
compared with the CPU oracle element by element (integers: bit-exact).

- ER 2^22, average degree 8: 64 giant-component roots in one tuned
  multi-source launch (a 1.07 GB depth output).
- The 32 uneven R-MAT graphs (scale 12-20, edge factor 8-32): 64 roots per
  graph in one launch each, tuned like the benchmark, launches overlapping on
  8 streams.
- The eight resident graphs of the query server (R-MAT up to scale 24, the
  2048^2 and 4096^2 permuted grids, ER 2^21): a mix of queries with and
  without same-graph merging, each result against the oracle.

The oracle runs on every host core (one thread per chunk of roots; its C code
runs outside the interpreter lock)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1708_01159_gb300 as bfs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

CORES = os.cpu_count() or 1


def oracle_rows(g, roots):
    """(depth[k, n], edges[k]) of the oracle, roots split over the host cores."""
    roots = np.asarray(roots, dtype=np.int32)
    chunks = [c for c in np.array_split(roots, min(CORES, len(roots))) if c.size]
    with ThreadPoolExecutor(max_workers=len(chunks)) as ex:
        parts = list(ex.map(lambda c: oracle.bfs_batch(g.off, g.idx, c), chunks))
    return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])


@pytest.fixture(scope="module", autouse=True)
def built():
    bfs.build()
    bfs.bfs_load_tree(None)
    yield


def test_er_2p22_wave_of_64_full_size():
    """ER 2^22 (average degree 8), 64 giant-component roots, one multi-source
    launch in the configuration the autotuner picks (as the benchmark runs it)."""
    g = gg.er_2p22_d8()
    roots = gg.sample_roots(g, 64, seed=gg.SEED_ROOTS + 3, giant=True)
    with bfs.Graph(g.off, g.idx) as G:
        out = torch.empty(64 * g.n, dtype=torch.int32, device="cuda")
        bfs.bfs_batch_tune(G.handle, roots, out)
        out.fill_(-7)
        edges = bfs.bfs_run_batch(G.handle, roots, out, edges=True)
        got = out.cpu().numpy().reshape(64, g.n)
    del out
    D, E = oracle_rows(g, roots)
    for i in range(64):
        assert np.array_equal(got[i], D[i]), f"root {roots[i]}: {int((got[i] != D[i]).sum())} depths differ"
    assert np.array_equal(edges, E)


def test_rmat_batch_of_32_graphs_full_size():
    """The benchmark's 32 uneven R-MAT graphs, 64 giant-component roots each,
    one launch per graph (graphs of scale 16 and up tuned for 8 waves at once),
    the launches spread over 8 streams so that they overlap: every row against
    the oracle."""
    specs = gg.rmat_batch_specs()
    streams = [torch.cuda.Stream() for _ in range(8)]
    gs, Gs, roots, outs = [], [], [], []
    try:
        for sc, ef, gseed, rseed in specs:
            g = gg.rmat(sc, ef, seed=gseed)
            G = bfs.Graph(g.off, g.idx)
            r = gg.sample_roots(g, 64, seed=rseed, giant=True)
            out = torch.empty(64 * g.n, dtype=torch.int32, device="cuda")
            if sc >= 16:  # as the benchmark: tuned for 8 waves at once
                bfs.bfs_batch_tune(G.handle, r, out, concurrency=len(streams))
            gs.append(g)
            Gs.append(G)
            roots.append(r)
            outs.append(out)
        for out in outs:
            out.fill_(-7)
        torch.cuda.synchronize()
        for i, G in enumerate(Gs):
            bfs.bfs_run_batch(G.handle, roots[i], outs[i], streams[i % len(streams)])
        torch.cuda.synchronize()
        for i, g in enumerate(gs):
            got = outs[i].cpu().numpy().reshape(len(roots[i]), g.n)
            D, _ = oracle_rows(g, roots[i])
            assert np.array_equal(got, D), f"graph {i} {specs[i]}: {int((got != D).sum())} depths differ"
    finally:
        for G in Gs:
            G.close()


@pytest.fixture(scope="module")
def serve_graphs():
    specs = gg.serve_graph_specs()
    gs = [mk() for _, mk in specs]
    Gs = [bfs.Graph(g.off, g.idx) for g in gs]
    yield [name for name, _ in specs], gs, Gs
    for G in Gs:
        G.close()


@pytest.mark.parametrize("merge_policy", [0, 1])
def test_serve_eight_resident_graphs_full_size(serve_graphs, merge_policy):
    """The query server over its eight resident graphs (R-MAT 16-24, the two
    permuted grids, ER 2^21), 80 queries submitted at once with output buffers
    (graph and root seeded): every result equals the oracle's. merge_policy 0
    merges where registration found waves cheaper; 1 merges every graph's
    queued queries (multi-source waves on R-MAT 24 and the 4096^2 grid)."""
    names, gs, Gs = serve_graphs
    rng = np.random.default_rng(5100 + merge_policy)
    s = bfs.bfs_serve_create(max_inflight=64, num_streams=16, queue_capacity=4096, merge_batch=64,
                             merge_policy=merge_policy)
    try:
        ids = [bfs.bfs_serve_add_graph(s, G.handle) for G in Gs]
        plan = []
        for q in range(80):
            gi = q % len(gs) if q < 16 else int(rng.integers(0, len(gs)))
            cand = np.nonzero(np.diff(gs[gi].off) > 0)[0]
            root = int(cand[int(rng.integers(0, len(cand)))])
            plan.append((gi, root, torch.full((gs[gi].n,), -7, dtype=torch.int32, device="cuda")))
        torch.cuda.synchronize()  # the server's streams do not wait on the caller's
        jobs = [(gi, root, out, bfs.bfs_serve_submit(s, ids[gi], root, out)) for gi, root, out in plan]
        for _, _, _, t in jobs:
            assert bfs.bfs_serve_wait(s, t) == bfs.BFS_OK
        st = bfs.bfs_serve_stats(s)
        assert st["completed"] == 80 and st["failed"] == 0
        if merge_policy == 1:
            assert st["merged_waves"] >= 1
        torch.cuda.synchronize()

        def check(job):
            gi, root, out, _ = job
            ref = oracle.bfs(gs[gi].off, gs[gi].idx, root)
            return gi, root, bool(np.array_equal(out.cpu().numpy(), ref.depth))

        with ThreadPoolExecutor(max_workers=CORES) as ex:
            bad = [(names[gi], root) for gi, root, ok in ex.map(check, jobs) if not ok]
        assert not bad, f"results differ from the oracle: {bad}"
    finally:
        bfs.bfs_serve_destroy(s)
