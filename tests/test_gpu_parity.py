"""GPU parity: depths from the CUDA path (through the C ABI) equal the CPU
oracle's element by element, on every variant, under tree switching, on edge
cases and at full workload sizes. Integer results: the bar is bit-exact."""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1708_01159_gb300 as bfs
from tests import graphs_closed_form as cf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
V = bfs.NUM_VARIANTS


@pytest.fixture(scope="module", autouse=True)
def built():
    bfs.build()
    bfs.bfs_load_tree(None)
    yield


def make(g, flags=bfs.BFS_SYMMETRIC):
    return bfs.Graph(g.off, g.idx, flags)


def run(G, root, variant=bfs.VARIANT_TREE, log=64, mode=bfs.MODE_DEFAULT):
    d = torch.empty(G.n, dtype=torch.int32, device="cuda")
    st = bfs.bfs_run_ex(G.handle, int(root), d, forced_variant=variant, stats=True, log_capacity=log, mode=mode)
    return d.cpu().numpy(), st


def assert_parity(g, G, root, variant=bfs.VARIANT_TREE, mode=bfs.MODE_DEFAULT):
    ref = oracle.bfs(g.off, g.idx, int(root))
    dep, st = run(G, root, variant, log=max(ref.num_levels + 1, 1), mode=mode)
    assert np.array_equal(dep, ref.depth), f"root {root} variant {variant}: depth mismatch " \
        f"({int((dep != ref.depth).sum())} entries)"
    assert st["edges_reached"] == ref.edges_reached
    assert st["vertices_reached"] == int((ref.depth >= 0).sum())
    assert st["levels"] == ref.num_levels
    assert st["status"] == 0
    k = min(ref.num_levels, len(st["frontier"]))
    assert np.array_equal(st["frontier"][:k], ref.level_count[:k])
    assert np.array_equal(st["frontier_edges"][:k], ref.level_edges[:k])
    if variant >= 0:
        assert np.all(st["variant"][:k] == variant)
    return ref, st


# ------------------------------------------------------------- small graphs

def test_rmat_s14_push_thread_16_roots():
    """R-MAT scale 14, edge factor 16, 16 seeded roots of nonzero degree, one
    fixed top-down push kernel: bit-exact depths."""
    g = gg.rmat_s14_ef16()
    roots = gg.sample_roots(g, 16, seed=gg.SEED_ROOTS)
    with make(g) as G:
        for r in roots:
            assert_parity(g, G, r, variant=0)


@pytest.mark.parametrize("variant", range(V))
@pytest.mark.parametrize("which", ["rmat13", "grid70x53", "er9000", "rmat12_perm"])
def test_each_variant(which, variant):
    g = {"rmat13": lambda: gg.rmat(13, 16, seed=11), "grid70x53": lambda: gg.grid(70, 53, 0.1, seed=12),
         "er9000": lambda: gg.erdos_renyi(9000, 6.0, seed=13),
         "rmat12_perm": lambda: gg.rmat(12, 8, seed=14, permute=True)}[which]()
    with make(g) as G:
        for r in gg.sample_roots(g, 3, seed=5):
            assert_parity(g, G, r, variant)


@pytest.mark.parametrize("mode", [bfs.MODE_PERSISTENT, bfs.MODE_GRAPH, bfs.MODE_HOST_LOOP])
@pytest.mark.parametrize("variant", [bfs.VARIANT_EDGE_LIST, bfs.VARIANT_REVERSE_EDGE_LIST])
def test_edge_list_variants(mode, variant):
    """Section 3.1.1's whole-edge-list kernels (forced only): bit-exact on
    skewed, high-diameter, directed (separate transpose origins) graphs and
    closed forms, in every driver; the tree cannot predict them."""
    rng = np.random.default_rng(5)
    n = 2000
    directed = gg.from_edges(n, rng.integers(0, n, 9000), rng.integers(0, n, 9000), symmetrize=False)
    for g, flags in ((gg.rmat(12, 16, seed=61), bfs.BFS_SYMMETRIC), (gg.grid(40, 30, 0.1, seed=62), bfs.BFS_SYMMETRIC),
                     (directed, 0), (cf.star(50)[0], bfs.BFS_SYMMETRIC)):
        with make(g, flags) as G:
            for r in gg.sample_roots(g, 2, seed=12):
                assert_parity(g, G, r, variant, mode)
    with pytest.raises(bfs.BFSError) as e:
        with make(gg.rmat(8, 8, seed=1)) as G:
            run(G, 0, bfs.NUM_FORCED_VARIANTS)
    assert e.value.code == bfs.BFS_ERR_INVALID_ARG


@pytest.mark.parametrize("count_mode", [1, 2])
def test_count_modes(count_mode):
    """Section 3.1.4's frontier-count alternatives (warp-aggregated and
    per-vertex atomics) in the vertex push: identical depths and per-level
    counts; the other drivers reject them."""
    for g in (gg.rmat(12, 16, seed=71), gg.grid(40, 30, 0.1, seed=72), gg.erdos_renyi(5000, 6.0, seed=73)):
        with make(g) as G:
            for r in gg.sample_roots(g, 2, seed=14):
                ref = oracle.bfs(g.off, g.idx, int(r))
                for v in (0, bfs.VARIANT_TREE):  # vertex push forced, and tree switching
                    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
                    st = bfs.bfs_run_ex(G.handle, int(r), d, forced_variant=v, mode=bfs.MODE_HOST_LOOP,
                                        count_mode=count_mode, stats=True, log_capacity=ref.num_levels + 1)
                    assert np.array_equal(d.cpu().numpy(), ref.depth)
                    assert np.array_equal(st["frontier"][:ref.num_levels], ref.level_count)
            for m in (bfs.MODE_PERSISTENT, bfs.MODE_GRAPH):
                with pytest.raises(bfs.BFSError) as e:
                    bfs.bfs_run_ex(G.handle, 0, d, mode=m, count_mode=count_mode)
                assert e.value.code == bfs.BFS_ERR_INVALID_ARG


@pytest.mark.parametrize("mode", [bfs.MODE_PERSISTENT, bfs.MODE_GRAPH, bfs.MODE_HOST_LOOP])
@pytest.mark.parametrize("variant", [bfs.VARIANT_TREE] + list(range(V)))
def test_execution_modes_agree(mode, variant):
    """The persistent kernel, the CUDA graph and the host loop run the same level
    code: identical depths, counts, and (under the tree) identical schedules."""
    for g in (gg.rmat(13, 16, seed=81), gg.grid(45, 61, 0.1, seed=82)):
        with make(g) as G:
            for r in gg.sample_roots(g, 2, seed=11):
                ref, st = assert_parity(g, G, r, variant, mode)
                if variant == bfs.VARIANT_TREE and mode != bfs.MODE_PERSISTENT:
                    _, st2 = run(G, r, variant, log=ref.num_levels + 1, mode=bfs.MODE_PERSISTENT)
                    assert st2["variant"].tolist() == st["variant"].tolist()


@pytest.mark.parametrize("name", sorted(cf.ALL))
def test_closed_forms_all_variants(name):
    g, fn = cf.ALL[name]()
    with make(g) as G:
        for r in range(0, g.n, max(1, g.n // 5)):
            for v in [bfs.VARIANT_TREE] + list(range(V)):
                dep, st = run(G, r, v)
                assert np.array_equal(dep, fn(r)), (name, r, v)


def test_directed_graph_uses_transpose():
    rng = np.random.default_rng(3)
    n = 3000
    s = rng.integers(0, n, 12000)
    t = rng.integers(0, n, 12000)
    g = gg.from_edges(n, s, t, symmetrize=False, name="directed")
    with make(g, flags=0) as G:
        assert not G.info()["symmetric"]
        for r in gg.sample_roots(g, 4, seed=1):
            for v in [bfs.VARIANT_TREE] + list(range(V)):
                assert_parity(g, G, r, v)


@pytest.mark.parametrize("mode", [bfs.MODE_PERSISTENT, bfs.MODE_GRAPH])
def test_sources_and_isolated_vertices(mode):
    """Isolated vertices start out marked visited (pull skips them, and whole
    bitmap words of them); sources (out-edges, no in-edges) must not be: they
    stay unreached unless they are the root, and are never taken for frontier
    in-neighbours by pull."""
    rng = np.random.default_rng(11)
    n = 4096
    sources = np.arange(0, n, 3)
    isolated = np.concatenate([np.arange(2048, 2112), np.arange(3001, n, 7)])  # two whole words + scattered
    sources = np.setdiff1d(sources, isolated)
    rest = np.setdiff1d(np.arange(n), np.concatenate([sources, isolated]))
    s = np.concatenate([rng.choice(sources, 6000), rng.choice(rest, 20000)])
    t = rng.choice(rest, 26000)
    g = gg.from_edges(n, s, t, symmetrize=False, name="sources")
    deg_in = np.bincount(g.idx, minlength=n)
    assert (deg_in[sources] == 0).all() and (np.diff(g.off)[isolated] == 0).all() and (deg_in[isolated] == 0).all()
    with make(g, flags=0) as G:
        for r in (0, 1023, int(rest[5]), 2050):
            for v in [bfs.VARIANT_TREE] + list(range(V)):
                ref, _ = assert_parity(g, G, r, v, mode=mode)
                assert (ref.depth[sources[sources != r]] == -1).all()


def test_hub_star_exercises_staged_cta_path():
    # one hub of degree 200k (staged through shared memory in many chunks) plus a tail
    n = 200_003
    s = np.zeros(n - 3, np.int32)
    t = np.arange(1, n - 2, dtype=np.int32)
    s = np.concatenate([s, [n - 3, n - 2]]).astype(np.int32)
    t = np.concatenate([t, [n - 2, n - 1]]).astype(np.int32)
    g = gg.from_edges(n, s, t, name="hub")
    with make(g) as G:
        for r in (0, 5, n - 1):
            for v in range(V):
                assert_parity(g, G, r, v)


# ------------------------------------------------------------------ edge cases

def test_edge_cases():
    # single vertex, no edges
    g = gg.Graph(np.array([0, 0], np.int32), np.zeros(0, np.int32))
    with make(g) as G:
        dep, st = run(G, 0)
        assert dep.tolist() == [0] and st["edges_reached"] == 0 and st["levels"] == 1
    # isolated root in a larger graph; ragged n (not a multiple of 32 or 4)
    g = gg.rmat(10, 4, seed=3)
    iso = int(np.nonzero(g.degrees() == 0)[0][0])
    with make(g) as G:
        for v in [bfs.VARIANT_TREE] + list(range(V)):
            dep, st = run(G, iso, v)
            exp = np.full(g.n, -1, np.int32)
            exp[iso] = 0
            assert np.array_equal(dep, exp) and st["edges_reached"] == 0
        with pytest.raises(bfs.BFSError) as e:
            run(G, g.n)
        assert e.value.code == bfs.BFS_ERR_INVALID_ARG
        with pytest.raises(bfs.BFSError):
            run(G, -1)
    g, fn = cf.path(37)
    with make(g) as G:
        dep, _ = run(G, 36)
        assert np.array_equal(dep, fn(36))


def test_unaligned_depth_output_and_host_output():
    g = gg.rmat(11, 8, seed=9)
    r = int(gg.sample_roots(g, 1, seed=2)[0])
    ref = oracle.bfs(g.off, g.idx, r)
    with make(g) as G:
        buf = torch.empty(g.n + 1, dtype=torch.int32, device="cuda")
        bfs.bfs_run(G.handle, r, buf[1:])  # 4-byte aligned only: scalar init path
        torch.cuda.synchronize()
        assert np.array_equal(buf[1:].cpu().numpy(), ref.depth)
        host = np.empty(g.n, np.int32)
        bfs.bfs_run_ex(G.handle, r, host, depth_on_host=True)
        assert np.array_equal(host, ref.depth)
        pinned = torch.empty(g.n, dtype=torch.int32).pin_memory()
        bfs.bfs_run_ex(G.handle, r, pinned, depth_on_host=True)
        assert np.array_equal(pinned.numpy(), ref.depth)


def test_host_output_async_on_two_streams():
    """host_async: each call returns once its copy is enqueued; 12 roots
    alternating between two streams, each into its own pinned buffer, equal
    the oracle once both streams are synchronised. host_async needs host
    output and no statistics."""
    g = gg.rmat(13, 16, seed=19)
    roots = [int(r) for r in gg.sample_roots(g, 12, seed=20)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    with make(g) as G:
        bufs = [torch.full((g.n,), -7, dtype=torch.int32).pin_memory() for _ in roots]
        torch.cuda.synchronize()
        for i, r in enumerate(roots):
            bfs.bfs_run_ex(G.handle, r, bufs[i], streams[i & 1], depth_on_host=True, host_async=True)
        for st in streams:
            st.synchronize()
        for r, b in zip(roots, bufs):
            assert np.array_equal(b.numpy(), oracle.bfs(g.off, g.idx, r).depth)
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for kw in ({"host_async": True}, {"host_async": True, "depth_on_host": True, "stats": True}):
            with pytest.raises(bfs.BFSError) as e:
                bfs.bfs_run_ex(G.handle, roots[0], d if "depth_on_host" not in kw else bufs[0], **kw)
            assert e.value.code == bfs.BFS_ERR_INVALID_ARG


def test_bad_graphs_rejected_on_device():
    off = np.array([0, 2, 3], np.int32)
    with pytest.raises(bfs.BFSError) as e:
        bfs.Graph(off, np.array([1, 5, 0], np.int32))  # index out of range
    assert e.value.code == bfs.BFS_ERR_BAD_GRAPH
    with pytest.raises(bfs.BFSError):
        bfs.Graph(np.array([0, 3, 2], np.int32), np.array([1, 0, 1], np.int32))  # decreasing offsets
    with pytest.raises(bfs.BFSError):
        bfs.Graph(np.array([1, 2, 3], np.int32), np.array([1, 0, 1], np.int32))  # off[0] != 0


def test_device_input_and_graph_info():
    g = gg.rmat(12, 16, seed=21)
    off = torch.from_numpy(g.off).cuda()
    idx = torch.from_numpy(g.idx).cuda()
    with bfs.Graph(off, idx) as G:
        info = G.info()
        assert info["n"] == g.n and info["m"] == g.m
        st = oracle.degree_stats(g.off)
        assert info["deg_summary"] == st[:5] and info["deg_sd256"] == st[5]
        for r in gg.sample_roots(g, 2, seed=4):
            assert_parity(g, G, r)


@pytest.mark.parametrize("symmetric", [True, False])
def test_in_and_total_degree_statistics_match_the_oracle(symmetric):
    """Section 4.1's in- and total-degree summaries, computed on the device at
    graph creation (the transpose's row lengths, and their sum with the
    out-degrees), equal the oracle's; a profiled level reports them too."""
    rng = np.random.default_rng(31)
    n = 20000
    g = (gg.rmat(13, 8, seed=32) if symmetric else
         gg.from_edges(n, rng.zipf(1.7, 90000) % n, rng.integers(0, n, 90000), symmetrize=False))
    F = oracle.F
    with make(g, flags=bfs.BFS_SYMMETRIC if symmetric else 0) as G:
        info = G.info()
        r = int(gg.sample_roots(g, 1, seed=33)[0])
        ref = oracle.bfs(g.off, g.idx, r)
        x = oracle.level_features(g.off, g.idx, ref)[0]
        assert info["in_deg_summary"] + [info["in_deg_sd256"]] == x[F["in_deg_min"]:F["in_deg_sd256"] + 1]
        assert info["tot_deg_summary"] + [info["tot_deg_sd256"]] == x[F["tot_deg_min"]:F["tot_deg_sd256"] + 1]
        feats, _, _ = bfs.bfs_profile_levels(G.handle, r, reps=1)
        assert feats.tolist() == oracle.level_features(g.off, g.idx, ref)


def test_injected_oom_is_reported():
    g = gg.rmat(10, 8, seed=3)
    bfs.lib().bfs_debug_fail_alloc_after(1)
    try:
        with pytest.raises(bfs.BFSError) as e:
            make(g)
        assert e.value.code == bfs.BFS_ERR_OOM
    finally:
        bfs.lib().bfs_debug_fail_alloc_after(0)
    with make(g) as G:  # the library is still usable
        assert_parity(g, G, int(gg.sample_roots(g, 1)[0]))


# -------------------------------------------------- switching and the schedule

def test_tree_schedule_matches_oracle_walk():
    """The variant log of a switched run equals the oracle's walk of the same
    tree over the oracle's per-level features, unknown-prediction rule included."""
    from paper_1708_01159_gb300 import buildlib
    rows = buildlib.parse_tree_text(open(bfs.DEFAULT_TREE).read())
    tree = {"nodes": [{"f": f, "t": t, "l": l, "r": r, "v": v} for f, t, l, r, v in rows]}
    for g in (gg.rmat(14, 16, seed=31), gg.grid(60, 60, 0.1, seed=32), gg.erdos_renyi(20000, 10.0, seed=33)):
        with make(g) as G:
            for r in gg.sample_roots(g, 3, seed=6):
                ref, st = assert_parity(g, G, r)
                feats = oracle.level_features(g.off, g.idx, ref)
                want = oracle.predict_schedule(tree, feats)
                assert st["variant"][:len(want)].tolist() == want


def test_custom_tree_file_with_unknown_leaves(tmp_path):
    # unknown at level 0 -> edge list default; unknown later -> repeat previous
    p = tmp_path / "t.tree"
    p.write_text("bfs-tree 1 5\n13 0 1 2 -1\n-1 0 -1 -1 -1\n8 50 3 4 -1\n-1 0 -1 -1 -1\n-1 0 -1 -1 4\n")
    tree = {"nodes": [{"f": 13, "t": 0, "l": 1, "r": 2, "v": -1}, {"f": -1, "t": 0, "l": -1, "r": -1, "v": -1},
                      {"f": 8, "t": 50, "l": 3, "r": 4, "v": -1}, {"f": -1, "t": 0, "l": -1, "r": -1, "v": -1},
                      {"f": -1, "t": 0, "l": -1, "r": -1, "v": 4}]}
    bfs.bfs_load_tree(str(p))
    try:
        g = gg.rmat(13, 16, seed=41)
        with make(g) as G:
            for r in gg.sample_roots(g, 3, seed=7):
                ref, st = assert_parity(g, G, r)
                want = oracle.predict_schedule(tree, oracle.level_features(g.off, g.idx, ref))
                assert st["variant"][:len(want)].tolist() == want
    finally:
        bfs.bfs_load_tree(None)


def _random_tree(rng, depth, feats_pool, node_limit=None):
    """A random integer tree (breadth-first numbering, children after parents)
    whose thresholds are drawn from observed feature values, so both branches
    of most nodes are taken; some leaves unknown (-1)."""
    nodes = [None]
    frontier = [(0, 0)]
    while frontier:
        i, d = frontier.pop(0)
        if d == depth or (node_limit and len(nodes) + 2 > node_limit):
            nodes[i] = {"f": -1, "t": 0, "l": -1, "r": -1, "v": int(rng.integers(-1, V))}
            continue
        f = int(rng.integers(0, len(oracle.FEATURES)))
        vals = [row[f] for row in feats_pool]
        t = int(rng.choice(vals)) if vals else 0
        l, r = len(nodes), len(nodes) + 1
        nodes += [None, None]
        nodes[i] = {"f": f, "t": t, "l": l, "r": r, "v": -1}
        frontier += [(l, d + 1), (r, d + 1)]
    return {"nodes": nodes}


@pytest.mark.parametrize("depth", [1, 4, 6, 7])
def test_random_trees_schedule_matches_oracle_walk(tmp_path, depth):
    """Random trees of depth 1-7: up to 64 leaves use the persistent kernel's
    bit-parallel evaluation, 128 leaves its walk; every driver's schedule equals
    the oracle's walk of the tree over the oracle's per-level features."""
    rng = np.random.default_rng(100 + depth)
    gs = [gg.rmat(13, 16, seed=43), gg.grid(50, 40, 0.1, seed=44), gg.erdos_renyi(8000, 5.0, seed=45),
          gg.rmat(12, 16, seed=46, directed=True, b=0.3, c=0.08)]
    pool = []
    refs = []
    for g in gs:
        for r in gg.sample_roots(g, 2, seed=depth):
            ref = oracle.bfs(g.off, g.idx, int(r))
            refs.append((g, int(r), ref))
            pool += oracle.level_features(g.off, g.idx, ref)
    for k in range(3):
        tree = _random_tree(rng, depth, pool)
        p = tmp_path / f"r{k}.tree"
        p.write_text(f"bfs-tree 1 {len(tree['nodes'])}\n" + "".join(
            f"{n['f']} {n['t']} {n['l']} {n['r']} {n['v']}\n" for n in tree["nodes"]))
        bfs.bfs_load_tree(str(p))
        try:
            for g, r, ref in refs:
                want = oracle.predict_schedule(tree, oracle.level_features(g.off, g.idx, ref))
                with make(g, flags=0 if g.name.endswith("-dir") else bfs.BFS_SYMMETRIC) as G:
                    for mode in (bfs.MODE_PERSISTENT, bfs.MODE_GRAPH):
                        _, st = assert_parity(g, G, r, mode=mode)
                        assert st["variant"][:len(want)].tolist() == want, (depth, k, mode)
        finally:
            bfs.bfs_load_tree(None)


def _write_tree(path, nodes):
    path.write_text(f"bfs-tree 1 {len(nodes)}\n" + "".join(
        f"{n['f']} {n['t']} {n['l']} {n['r']} {n['v']}\n" for n in nodes))


def _stump(f, t, left, right):
    return [{"f": f, "t": t, "l": 1, "r": 2, "v": -1}, {"f": -1, "t": 0, "l": -1, "r": -1, "v": left},
            {"f": -1, "t": 0, "l": -1, "r": -1, "v": right}]


def test_directed_graphs_tree_splits_on_in_degree(tmp_path):
    """Directed R-MAT graphs whose in-degree distributions differ (b != c): a
    tree that splits on the in-degree maximum and on the total-degree upper
    quartile (Section 4.1's in- and total-degree features) sends them down
    different branches; every schedule equals the oracle's walk and every depth
    the oracle's, in the persistent and graph drivers."""
    ga = gg.rmat(12, 16, seed=51, directed=True, b=0.30, c=0.08)  # skewed out-degree, flat in-degree
    gb = gg.rmat(12, 16, seed=52, directed=True, b=0.08, c=0.30)  # flat out-degree, skewed in-degree
    F = oracle.F
    xa = oracle.level_features(ga.off, ga.idx, oracle.bfs(ga.off, ga.idx, 0))[0]
    xb = oracle.level_features(gb.off, gb.idx, oracle.bfs(gb.off, gb.idx, 0))[0]
    assert xa[F["in_deg_max"]] < xb[F["in_deg_max"]]
    t_in = (xa[F["in_deg_max"]] + xb[F["in_deg_max"]]) // 2
    nodes = [{"f": F["in_deg_max"], "t": t_in, "l": 1, "r": 2, "v": -1},
             {"f": F["frontier"], "t": 40, "l": 3, "r": 4, "v": -1},
             {"f": F["tot_deg_q3"], "t": xb[F["tot_deg_q3"]], "l": 5, "r": 6, "v": -1},
             {"f": -1, "t": 0, "l": -1, "r": -1, "v": 0}, {"f": -1, "t": 0, "l": -1, "r": -1, "v": 4},
             {"f": -1, "t": 0, "l": -1, "r": -1, "v": 2}, {"f": -1, "t": 0, "l": -1, "r": -1, "v": 3}]
    p = tmp_path / "io.tree"
    _write_tree(p, nodes)
    bfs.bfs_load_tree(str(p))
    try:
        seen = set()
        for g in (ga, gb):
            with make(g, flags=0) as G:
                for r in gg.sample_roots(g, 3, seed=53):
                    ref = oracle.bfs(g.off, g.idx, int(r))
                    want = oracle.predict_schedule({"nodes": nodes}, oracle.level_features(g.off, g.idx, ref))
                    seen.update(want)
                    for mode in (bfs.MODE_PERSISTENT, bfs.MODE_GRAPH):
                        _, st = assert_parity(g, G, r, mode=mode)
                        assert st["variant"][:len(want)].tolist() == want
        assert {0, 4}.issubset(seen) and seen & {2, 3}  # both sides of the in-degree split ran
    finally:
        bfs.bfs_load_tree(None)


def test_tree_threshold_edges(tmp_path):
    """Split thresholds at the edges of each feature's range: ppm thresholds
    below 0 and at 1e6, thresholds equal to an observed value and one below it
    (the <= boundary, ppm compared without dividing), and trees whose only tests
    are on graph features (decided once per graph, no level test left). Every
    driver's schedule equals the oracle's walk."""
    g = gg.rmat(13, 16, seed=46)
    roots = [int(r) for r in gg.sample_roots(g, 2, seed=9)]
    refs = [(r, oracle.bfs(g.off, g.idx, r)) for r in roots]
    feats = oracle.level_features(g.off, g.idx, refs[0][1])
    mid = feats[len(feats) // 2]
    trees = [_stump(9, -1, 1, 4), _stump(11, -1, 1, 4), _stump(9, 1000000, 1, 4), _stump(11, 999999, 1, 4)]
    for fi in (8, 9, 10, 11, 12, 13):
        trees += [_stump(fi, mid[fi], 0, 4), _stump(fi, mid[fi] - 1, 2, 3)]
    for fi in range(8):  # graph features only
        trees += [_stump(fi, feats[0][fi], 1, 4), _stump(fi, feats[0][fi] - 1, 1, 4)]
    # a graph-feature test above a level-feature test, and below one
    trees.append([{"f": 6, "t": feats[0][6], "l": 1, "r": 2, "v": -1},
                  {"f": 11, "t": mid[11], "l": 3, "r": 4, "v": -1},
                  {"f": -1, "t": 0, "l": -1, "r": -1, "v": 2},
                  {"f": -1, "t": 0, "l": -1, "r": -1, "v": 3},
                  {"f": -1, "t": 0, "l": -1, "r": -1, "v": 4}])
    trees.append([{"f": 8, "t": mid[8], "l": 1, "r": 2, "v": -1},
                  {"f": 0, "t": feats[0][0] - 1, "l": 3, "r": 4, "v": -1},
                  {"f": -1, "t": 0, "l": -1, "r": -1, "v": 1},
                  {"f": -1, "t": 0, "l": -1, "r": -1, "v": 0},
                  {"f": -1, "t": 0, "l": -1, "r": -1, "v": 4}])
    with make(g) as G:
        for k, nodes in enumerate(trees):
            p = tmp_path / f"e{k}.tree"
            _write_tree(p, nodes)
            bfs.bfs_load_tree(str(p))
            try:
                for r, ref in refs:
                    want = oracle.predict_schedule({"nodes": nodes}, oracle.level_features(g.off, g.idx, ref))
                    for mode in (bfs.MODE_PERSISTENT, bfs.MODE_GRAPH, bfs.MODE_HOST_LOOP):
                        _, st = assert_parity(g, G, r, mode=mode)
                        assert st["variant"][:len(want)].tolist() == want, (k, nodes[0], mode)
            finally:
                bfs.bfs_load_tree(None)


def test_profile_levels_features_match_oracle():
    g = gg.rmat(13, 16, seed=51)
    r = int(gg.sample_roots(g, 1, seed=8)[0])
    ref = oracle.bfs(g.off, g.idx, r)
    with make(g) as G:
        feats, ms, tv = bfs.bfs_profile_levels(G.handle, r, reps=3)
        assert feats.shape[0] == ref.num_levels
        assert feats.tolist() == oracle.level_features(g.off, g.idx, ref)
        assert np.all(ms > 0)
        # the harness leaves the graph usable and results unchanged
        assert_parity(g, G, r)


def test_concurrent_streams():
    g = gg.rmat(14, 16, seed=61)
    roots = gg.sample_roots(g, 6, seed=9)
    refs = [oracle.bfs(g.off, g.idx, int(r)).depth for r in roots]
    with make(g) as G:
        streams = [torch.cuda.Stream() for _ in range(3)]
        outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in roots]
        for k in range(2):
            for i, r in enumerate(roots):
                bfs.bfs_run(G.handle, int(r), outs[i], streams[i % 3])
        torch.cuda.synchronize()
        for i in range(len(roots)):
            assert np.array_equal(outs[i].cpu().numpy(), refs[i])
        assert G.info()["num_workspaces"] >= 1


@pytest.mark.parametrize("mode", [bfs.MODE_PERSISTENT, bfs.MODE_GRAPH, bfs.MODE_HOST_LOOP])
def test_many_streams_mixed_graphs(mode):
    """400 traversals over four graphs spread round-robin over 16 streams, all
    enqueued before any finishes: every output equals the run alone."""
    gs = [gg.rmat(14, 16, seed=501), gg.grid(120, 90, 0.1, seed=502), gg.erdos_renyi(30000, 6.0, seed=503),
          gg.rmat(12, 8, seed=504, permute=True)]
    Gs = [make(g) for g in gs]
    try:
        rng = np.random.default_rng(1)
        streams = [torch.cuda.Stream() for _ in range(16)]
        plan = []
        for q in range(400 if mode != bfs.MODE_HOST_LOOP else 64):
            gi = int(rng.integers(0, 4))
            r = int(gg.sample_roots(gs[gi], 1, seed=q)[0])
            plan.append((gi, r, torch.full((gs[gi].n,), -7, dtype=torch.int32, device="cuda")))
        want = {}
        for gi, r, _ in plan:
            if (gi, r) not in want:
                want[(gi, r)] = oracle.bfs(gs[gi].off, gs[gi].idx, r).depth
        torch.cuda.synchronize()
        for q, (gi, r, out) in enumerate(plan):
            bfs.bfs_run_ex(Gs[gi].handle, r, out, streams[q % 16], mode=mode)
        torch.cuda.synchronize()
        bad = [q for q, (gi, r, out) in enumerate(plan) if not np.array_equal(out.cpu().numpy(), want[(gi, r)])]
        detail = []
        for q in bad[:3]:
            gi, r, out = plan[q]
            o, e = out.cpu().numpy(), want[(gi, r)]
            dif = np.nonzero(o != e)[0]
            pairs = sorted(set(zip(e[dif].tolist(), o[dif].tolist())))[:8]
            _, st = run(Gs[gi], r, log=64, mode=mode)
            detail.append(f"q={q} graph={gi} root={r} stream={q % 16}: {len(dif)} depths differ, unreached "
                          f"{int((o == -1).sum())} vs {int((e == -1).sum())}, untouched {int((o == -7).sum())}, "
                          f"(want, got) {pairs}; schedule alone {st['variant'].tolist()}")
        assert not bad, f"{len(bad)} of {len(plan)} traversals wrong: " + " | ".join(detail)
    finally:
        for G in Gs:
            G.close()


def test_batch_equals_single_runs():
    g = gg.rmat(12, 16, seed=71)
    roots = gg.sample_roots(g, 70, seed=10)  # more than one wave of 64
    with make(g) as G:
        out = torch.empty(len(roots) * g.n, dtype=torch.int32, device="cuda")
        edges = bfs.bfs_run_batch(G.handle, roots, out, edges=True)
        torch.cuda.synchronize()
        D, E = oracle.bfs_batch(g.off, g.idx, roots)
        assert np.array_equal(out.cpu().numpy().reshape(len(roots), g.n), D)
        assert np.array_equal(edges, E)


@pytest.mark.parametrize("grid_blocks", [1, 5, 37, 1 << 20])
def test_persistent_grid_blocks(grid_blocks):
    """The persistent driver on any number of blocks (1, odd, fewer than the SMs,
    more than one occupancy wave: clamped) gives the oracle's depths; the other
    drivers reject a block count."""
    for g in (gg.rmat(13, 16, seed=83), gg.grid(45, 61, 0.1, seed=84)):
        with make(g) as G:
            for r in gg.sample_roots(g, 2, seed=13):
                ref = oracle.bfs(g.off, g.idx, int(r))
                d = torch.empty(g.n, dtype=torch.int32, device="cuda")
                st = bfs.bfs_run_ex(G.handle, int(r), d, mode=bfs.MODE_PERSISTENT, grid_blocks=grid_blocks, stats=True)
                assert np.array_equal(d.cpu().numpy(), ref.depth) and st["levels"] == ref.num_levels
            for m in (bfs.MODE_GRAPH, bfs.MODE_HOST_LOOP):
                with pytest.raises(bfs.BFSError) as e:
                    bfs.bfs_run_ex(G.handle, 0, d, mode=m, grid_blocks=grid_blocks)
                assert e.value.code == bfs.BFS_ERR_INVALID_ARG


@pytest.mark.parametrize("which", ["rmat", "grid"])
@pytest.mark.parametrize("push_mode", [0, 1])
@pytest.mark.parametrize("alpha,grid_blocks", [(1, 0), (8, 3), (64, 0), (1 << 20, 0), (8, 1 << 20)])
def test_batch_configs(which, push_mode, alpha, grid_blocks):
    """Multi-source BFS in every configuration (alpha 1: pull from level 1 on;
    huge alpha: push only) equals independent oracle runs, repeated and isolated
    roots included, on a skewed graph and on a high-diameter grid."""
    g = gg.rmat(12, 8, seed=91) if which == "rmat" else gg.grid(70, 60, 0.15, seed=92)
    if which == "grid":  # an isolated vertex for the isolated-root case
        g = gg.Graph(np.concatenate([g.off, [g.m]]).astype(np.int32), g.idx, "grid+isolated")
    iso = int(np.nonzero(g.degrees() == 0)[0][0])
    roots = np.concatenate([gg.sample_roots(g, 40, seed=12), [iso, iso], gg.sample_roots(g, 3, seed=12)])
    D, E = oracle.bfs_batch(g.off, g.idx, roots)
    with make(g) as G:
        bfs.bfs_batch_set_config(G.handle, push_mode, alpha, grid_blocks)
        out = torch.empty(len(roots) * g.n, dtype=torch.int32, device="cuda")
        edges = bfs.bfs_run_batch(G.handle, roots, out, edges=True)
        assert np.array_equal(out.cpu().numpy().reshape(len(roots), g.n), D)
        assert np.array_equal(edges, E)


@pytest.mark.parametrize("alpha", [1, 4, 1 << 20])
def test_batch_depth_history_boundary(alpha):
    """Depths on both sides of the end of the multi-source depth history (the
    frontier masks of depths 0-14 are kept for the final pass; deeper depths
    are written when found): a path of 80 vertices with a 40-vertex clique
    hung on path vertex 16, roots along the path, so that with alpha 4 the
    levels that reach the clique pull (frontier edges x 4 > m) between push
    levels at depths 14-18, and pull-only and push-only as well."""
    P, C = 80, 40
    src, dst = [], []
    for i in range(P - 1):
        src.append(i)
        dst.append(i + 1)
    for a in range(C):
        src.append(16)
        dst.append(P + a)
        for b in range(a + 1, C):
            src.append(P + a)
            dst.append(P + b)
    g = gg.from_edges(P + C, np.array(src, np.int32), np.array(dst, np.int32), name="path+clique")
    roots = np.array([0, 1, 2, 3, 0, 79, 60, 30, P + 5, 15, 14], np.int32)
    D, E = oracle.bfs_batch(g.off, g.idx, roots)
    assert D.max() > 20  # depths well past the history
    with make(g) as G:
        for push_mode in (0, 1):
            bfs.bfs_batch_set_config(G.handle, push_mode, alpha, 0)
            out = torch.full((len(roots) * g.n,), -7, dtype=torch.int32, device="cuda")
            edges = bfs.bfs_run_batch(G.handle, roots, out, edges=True)
            assert np.array_equal(out.cpu().numpy().reshape(len(roots), g.n), D)
            assert np.array_equal(edges, E)


def test_batch_uneven_graphs_concurrently():
    """A batch of uneven R-MAT graphs (scale 8-13, edge factor 8-32), 64 roots
    each in one launch per graph, launches spread over streams and overlapping:
    every depth row equals the oracle's."""
    rng = np.random.default_rng(21)
    specs = [(int(rng.integers(8, 14)), int(rng.choice([8, 16, 32]))) for _ in range(6)]
    gs = [gg.rmat(sc, ef, seed=700 + i) for i, (sc, ef) in enumerate(specs)]
    Gs = [make(g) for g in gs]
    try:
        streams = [torch.cuda.Stream() for _ in range(3)]
        roots = [gg.sample_roots(g, 64, seed=800 + i) for i, g in enumerate(gs)]
        outs = [torch.full((64 * g.n,), -7, dtype=torch.int32, device="cuda") for g in gs]
        torch.cuda.synchronize()
        for i, G in enumerate(Gs):
            bfs.bfs_run_batch(G.handle, roots[i], outs[i], streams[i % 3])
        torch.cuda.synchronize()
        for i, g in enumerate(gs):
            D, _ = oracle.bfs_batch(g.off, g.idx, roots[i])
            assert np.array_equal(outs[i].cpu().numpy().reshape(64, g.n), D), specs[i]
    finally:
        for G in Gs:
            G.close()


def test_batch_directed_and_tuner():
    rng = np.random.default_rng(5)
    n = 5000
    g = gg.from_edges(n, rng.integers(0, n, 20000), rng.integers(0, n, 20000), symmetrize=False)
    roots = gg.sample_roots(g, 64, seed=13)
    D, E = oracle.bfs_batch(g.off, g.idx, roots)
    with make(g, flags=0) as G:
        scratch = torch.empty(64 * n, dtype=torch.int32, device="cuda")
        cfg = bfs.bfs_batch_tune(G.handle, roots, scratch)
        assert cfg["push_mode"] in (0, 1) and cfg["alpha"] >= 1 and cfg["ms"] > 0 and cfg["grid_blocks"] > 0
        out = torch.empty(64 * n, dtype=torch.int32, device="cuda")
        edges = bfs.bfs_run_batch(G.handle, roots, out, edges=True)
        assert np.array_equal(out.cpu().numpy().reshape(64, n), D)
        assert np.array_equal(edges, E)
        # tuned for 8 waves at once: a grid of at most 1/4 of a full wave
        full = bfs.bfs_batch_tune(G.handle, roots, scratch, concurrency=1)
        c8 = bfs.bfs_batch_tune(G.handle, roots, scratch, concurrency=8)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert 1 <= c8["grid_blocks"] <= max(1, 8 * sms // 4)
        out.fill_(-7)
        edges = bfs.bfs_run_batch(G.handle, roots, out, edges=True)
        assert np.array_equal(out.cpu().numpy().reshape(64, n), D)
        assert np.array_equal(edges, E)
        assert full["grid_blocks"] >= c8["grid_blocks"]
        with pytest.raises(bfs.BFSError) as e:
            bfs.bfs_batch_tune(G.handle, roots, scratch, concurrency=0)
        assert e.value.code == bfs.BFS_ERR_INVALID_ARG


# --------------------------------------------------------- full-size workloads

@pytest.mark.slow
def test_rmat_s22_full_size():
    """R-MAT scale 22, edge factor 16 (~128M directed edges), roots in the giant
    component: switched and every fixed variant bit-exact, in the launch
    configuration the benchmark times."""
    g = gg.rmat_s22_ef16()
    roots = gg.sample_roots(g, 2, seed=gg.SEED_ROOTS + 1, giant=True)
    with make(g) as G:
        for i, r in enumerate(roots):
            assert_parity(g, G, r)
            if i == 0:
                for v in range(V):
                    assert_parity(g, G, r, v)


@pytest.mark.slow
def test_grid_4096_full_size():
    """4096 x 4096 permuted grid with 10% of edges dropped: thousands of levels."""
    g = gg.grid_4096_permuted()
    r = int(gg.sample_roots(g, 1, seed=gg.SEED_ROOTS + 2, giant=True)[0])
    with make(g) as G:
        ref, st = assert_parity(g, G, r)
        assert ref.num_levels > 1000


@pytest.mark.parametrize("policy", list(range(len(bfs.WARP_WIDTHS))))
def test_warp_width_policies_exact(policy):
    """Every virtual-warp width policy (the mean-degree rule, doubled, halved,
    fixed 4/8/16/32) gives the oracle's depths with push_warp forced and with
    the tree, in the persistent and graph drivers, on a skewed, a
    high-diameter and a directed graph."""
    cases = ((gg.rmat(12, 16, seed=811), bfs.BFS_SYMMETRIC), (gg.grid(40, 30, 0.1, seed=812), bfs.BFS_SYMMETRIC),
             (gg.rmat(11, 8, seed=813, directed=True), 0))
    for g, flags in cases:
        with make(g, flags) as G:
            bfs.bfs_set_warp_width(G.handle, policy)
            assert bfs.bfs_get_warp_width(G.handle) == policy
            for r in gg.sample_roots(g, 2, seed=814):
                ref = oracle.bfs(g.off, g.idx, int(r))
                for mode in (bfs.MODE_PERSISTENT, bfs.MODE_GRAPH):
                    for v in (bfs.VARIANTS.index("push_warp"), bfs.VARIANT_TREE):
                        d = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
                        st = bfs.bfs_run_ex(G.handle, int(r), d, forced_variant=v, mode=mode, stats=True)
                        assert np.array_equal(d.cpu().numpy(), ref.depth), (policy, mode, v)
                        assert st["edges_reached"] == ref.edges_reached


def test_warp_width_tuner_sets_the_fastest():
    g = gg.grid(120, 90, 0.1, seed=815)
    roots = gg.sample_roots(g, 3, seed=816)
    with make(g) as G:
        res = bfs.bfs_tune_warp_width(G.handle, roots)
        assert 0 <= res["policy"] < len(bfs.WARP_WIDTHS)
        assert res["ms"][res["name"]] == min(res["ms"].values()) and min(res["ms"].values()) > 0
        assert bfs.bfs_get_warp_width(G.handle) == res["policy"]
        with pytest.raises(bfs.BFSError) as e:
            bfs.bfs_set_warp_width(G.handle, len(bfs.WARP_WIDTHS))
        assert e.value.code == bfs.BFS_ERR_INVALID_ARG
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for r in roots:  # exact under the tuned policy
            bfs.bfs_run(G.handle, int(r), d)
            assert np.array_equal(d.cpu().numpy(), oracle.bfs(g.off, g.idx, int(r)).depth)
