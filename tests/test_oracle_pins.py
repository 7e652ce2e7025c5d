"""Pins for the CPU oracle: each check ties it to something other than itself
(brute force, closed forms, library routines, invariants, hand-derived
fixtures). CPU only."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import graphs_closed_form as cf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def check_invariants(off, idx, root, depth, symmetric=True):
    """Properties every BFS depth vector has (Section 2.2 shortest distances)."""
    n = off.shape[0] - 1
    assert depth[root] == 0
    src = np.repeat(np.arange(n), np.diff(off))
    du, dv = depth[src], depth[idx]
    both = (du >= 0) & (dv >= 0)
    # an edge u->v with u reached gives v a depth of at most depth(u) + 1
    assert np.all(dv[du >= 0] >= 0)
    assert np.all(dv[both] <= du[both] + 1)
    if symmetric:
        assert np.all(np.abs(du[both] - dv[both]) <= 1)
    # every reached v != root has an in-neighbour one level closer
    has_parent = np.zeros(n, dtype=bool)
    ok = both & (du == dv - 1)
    has_parent[idx[ok]] = True
    reached = depth >= 0
    reached[root] = False
    assert np.all(has_parent[reached])
    # the level histogram is contiguous from 0
    levels = np.unique(depth[depth >= 0])
    assert np.array_equal(levels, np.arange(levels.shape[0]))


# ----------------------------------------------------------------- brute force

def test_exhaustive_undirected_up_to_5_vertices():
    """Every undirected graph on n <= 5 vertices, every root, vs dense brute force."""
    for n in range(1, 6):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            adj = np.zeros((n, n), dtype=bool)
            for b, (u, v) in enumerate(pairs):
                if mask >> b & 1:
                    adj[u, v] = adj[v, u] = True
            g = cf.csr_from_adj(adj)
            for r in range(n):
                res = oracle.bfs(g.off, g.idx, r)
                assert np.array_equal(res.depth, cf.brute_force_depth(adj, r)), (n, mask, r)


def test_random_directed_vs_brute_force():
    rng = np.random.default_rng(11)
    for trial in range(300):
        n = int(rng.integers(1, 13))
        p = float(rng.uniform(0.05, 0.6))
        adj = rng.random((n, n)) < p
        np.fill_diagonal(adj, rng.random(n) < 0.2)  # self-loops must not change anything
        g = cf.csr_from_adj(adj)
        for r in range(n):
            res = oracle.bfs(g.off, g.idx, r)
            assert np.array_equal(res.depth, cf.brute_force_depth(adj, r)), (trial, r)
            check_invariants(g.off, g.idx, r, res.depth, symmetric=False)


def test_duplicate_edges_do_not_change_depths():
    rng = np.random.default_rng(5)
    for _ in range(50):
        n = int(rng.integers(2, 12))
        adj = rng.random((n, n)) < 0.3
        g = cf.csr_from_adj(adj)
        # duplicate every entry of the CSR
        deg = np.diff(g.off)
        off2 = np.concatenate([[0], np.cumsum(2 * deg)]).astype(np.int32)
        idx2 = np.repeat(g.idx, 2).astype(np.int32)
        for r in range(n):
            a = oracle.bfs(g.off, g.idx, r)
            b = oracle.bfs(off2, idx2, r)
            assert np.array_equal(a.depth, b.depth)
            assert b.edges_reached == 2 * a.edges_reached


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("name", sorted(cf.ALL))
def test_closed_forms(name):
    g, fn = cf.ALL[name]()
    for r in range(g.n):
        res = oracle.bfs(g.off, g.idx, r)
        assert np.array_equal(res.depth, fn(r)), (name, r)
        check_invariants(g.off, g.idx, r, res.depth)


def test_pure_python_definition_agrees_on_tiny():
    rng = np.random.default_rng(3)
    for _ in range(40):
        n = int(rng.integers(1, 30))
        adj = rng.random((n, n)) < 0.15
        g = cf.csr_from_adj(adj)
        for r in range(n):
            assert oracle.bfs(g.off, g.idx, r).depth.tolist() == oracle.bfs_python(g.off.tolist(), g.idx.tolist(), r)


# --------------------------------------------------------------- library routines

@pytest.mark.parametrize("which", ["rmat12", "grid48", "er3000"])
def test_scipy_shortest_path(which):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    if which == "rmat12":
        g = gg.rmat(12, 16, seed=77)
    elif which == "grid48":
        g = gg.grid(48, 48, 0.1, seed=78)
    else:
        g = gg.erdos_renyi(3000, 3.0, seed=79)
    A = sp.csr_matrix((np.ones(g.m), g.idx, g.off), shape=(g.n, g.n))
    roots = gg.sample_roots(g, 6, seed=1)
    D = csgraph.shortest_path(A, unweighted=True, indices=roots)
    for i, r in enumerate(roots):
        exp = np.where(np.isinf(D[i]), -1, D[i]).astype(np.int32)
        res = oracle.bfs(g.off, g.idx, int(r))
        assert np.array_equal(res.depth, exp)
        check_invariants(g.off, g.idx, int(r), res.depth)


def test_networkx_directed():
    nx = pytest.importorskip("networkx")
    G = nx.gnp_random_graph(400, 0.01, seed=5, directed=True)
    n = 400
    off = np.zeros(n + 1, dtype=np.int32)
    idx = []
    for u in range(n):
        nb = sorted(G.successors(u))
        idx += nb
        off[u + 1] = len(idx)
    idx = np.asarray(idx, dtype=np.int32)
    for r in (0, 17, 399):
        exp = np.full(n, -1, dtype=np.int32)
        for v, d in nx.single_source_shortest_path_length(G, r).items():
            exp[v] = d
        assert np.array_equal(oracle.bfs(off, idx, r).depth, exp)


# ---------------------------------------------------------- counts and edge sums

def test_edges_reached_and_level_counts():
    g = gg.rmat(13, 8, seed=91)
    deg = g.degrees()
    comp, _, _ = gg.components(g)
    for r in gg.sample_roots(g, 8, seed=3):
        res = oracle.bfs(g.off, g.idx, int(r))
        # symmetric graph: reached set = r's connected component; edges = sum of its degrees
        in_comp = comp == comp[r]
        assert np.array_equal(res.depth >= 0, in_comp)
        assert res.edges_reached == int(deg[in_comp].sum())
        d = res.depth[res.depth >= 0]
        assert np.array_equal(res.level_count, np.bincount(d))
        assert np.array_equal(res.level_edges, np.bincount(d, weights=deg[res.depth >= 0]).astype(np.int64))
        assert int(res.level_count.sum()) == int(in_comp.sum())


def test_connected_graph_reaches_all_edges():
    g, _ = cf.hypercube(7)
    assert oracle.bfs(g.off, g.idx, 5).edges_reached == g.m


def test_golden_directed_fixture():
    fx = json.load(open(os.path.join(GOLDEN, "directed6.json")))
    s, t = zip(*fx["edges"])
    g = gg.from_edges(fx["n"], s, t, symmetrize=False)
    for c in fx["cases"]:
        res = oracle.bfs(g.off, g.idx, c["root"])
        assert res.depth.tolist() == c["depth"]
        assert res.edges_reached == c["edges_reached"]
        assert res.level_count.tolist() == c["level_count"]


def test_batch_is_independent_runs():
    g = gg.rmat(10, 8, seed=4)
    roots = gg.sample_roots(g, 5, seed=9)
    D, E = oracle.bfs_batch(g.off, g.idx, roots)
    for i, r in enumerate(roots):
        res = oracle.bfs(g.off, g.idx, int(r))
        assert np.array_equal(D[i], res.depth)
        assert E[i] == res.edges_reached


# ----------------------------------------------------------------- validation

def test_validate_csr():
    g, _ = cf.path(6)
    assert oracle.validate_csr(g.off, g.idx) == 0
    bad = g.off.copy(); bad[0] = 1
    assert oracle.validate_csr(bad, g.idx) == oracle.ORACLE_ERR_BAD_GRAPH
    bad = g.off.copy(); bad[2], bad[3] = bad[3], bad[2]
    assert oracle.validate_csr(bad, g.idx) == oracle.ORACLE_ERR_BAD_GRAPH
    bad = g.idx.copy(); bad[0] = 6
    assert oracle.validate_csr(g.off, bad) == oracle.ORACLE_ERR_BAD_GRAPH
    bad = g.idx.copy(); bad[1] = -1
    assert oracle.validate_csr(g.off, bad) == oracle.ORACLE_ERR_BAD_GRAPH
    assert oracle.validate_csr(g.off, g.idx[:-1]) == oracle.ORACLE_ERR_BAD_GRAPH
    with pytest.raises(ValueError):
        oracle.bfs(g.off, g.idx, 6)
    with pytest.raises(ValueError):
        oracle.bfs(g.off, g.idx, -1)


# ------------------------------------------------------------------ features

def test_degree_stats_vs_numpy():
    for g in (gg.rmat(12, 16, seed=8), gg.grid(30, 41, 0.1, seed=2), gg.erdos_renyi(999, 5.0, seed=1),
              cf.star(10)[0], cf.path(2)[0]):
        deg = g.degrees()
        st = oracle.degree_stats(g.off)
        q = [int(np.percentile(deg, 25 * k, method="lower")) for k in range(5)]
        assert st[:5] == q
        assert st[0] == deg.min() and st[4] == deg.max()
        sd = 256.0 * float(np.std(deg))
        assert abs(st[5] - math.floor(sd)) <= 1 and st[5] <= sd + 1e-6


def test_degree_sd_exact_cases():
    # degrees {0, 2}: sigma = 1 exactly -> 256; regular graph: sigma = 0
    g = gg.from_edges(4, [0], [1])  # degrees 1,1,0,0 -> mean 1/2, sigma 1/2 -> 128
    assert oracle.degree_stats(g.off)[5] == 128
    g, _ = cf.cycle(9)
    assert oracle.degree_stats(g.off) == [2, 2, 2, 2, 2, 0]


def test_level_features_layout():
    g, _ = cf.star(9)
    res = oracle.bfs(g.off, g.idx, 3)
    feats = oracle.level_features(g.off, g.idx, res)
    assert len(feats) == 3
    F = oracle.F
    assert [x[F["frontier"]] for x in feats] == [1, 1, 7]
    assert [x[F["discovered"]] for x in feats] == [1, 2, 9]
    assert [x[F["frontier_edges"]] for x in feats] == [1, 8, 7]
    assert [x[F["discovered_ppm"]] for x in feats] == [111111, 222222, 1000000]
    assert all(x[F["n"]] == 9 and x[F["m"]] == 16 for x in feats)
    assert [x[F["level"]] for x in feats] == [0, 1, 2]


# ---------------------------------------------------------------- tree walk

def _export_sklearn(clf):
    """Integer tree from a fitted sklearn classifier: x <= t with t = floor(threshold)."""
    t = clf.tree_
    nodes = []
    for i in range(t.node_count):
        if t.children_left[i] < 0:
            nodes.append({"f": -1, "t": 0, "l": -1, "r": -1, "v": int(np.argmax(t.value[i][0]))})
        else:
            nodes.append({"f": int(t.feature[i]), "t": int(math.floor(t.threshold[i])),
                          "l": int(t.children_left[i]), "r": int(t.children_right[i]), "v": -1})
    return {"nodes": nodes}


def test_tree_walk_matches_sklearn_predict():
    tree_mod = pytest.importorskip("sklearn.tree")
    rng = np.random.default_rng(0)
    X = rng.integers(0, 1000, size=(3000, 14))
    y = ((X[:, 8] > 500).astype(int) * 2 + (X[:, 11] % 7 > 3).astype(int) + (X[:, 2] > 900)) % 5
    clf = tree_mod.DecisionTreeClassifier(max_depth=8, random_state=0).fit(X, y)
    tree = _export_sklearn(clf)
    Xt = rng.integers(0, 1000, size=(2000, 14))
    pred = clf.predict(Xt)
    walk = np.array([oracle.tree_walk(tree, x) for x in Xt])
    assert np.array_equal(walk, pred)


def test_unknown_prediction_rule_golden():
    fx = json.load(open(os.path.join(GOLDEN, "unknown_rule.json")))
    feats = []
    for L, f in enumerate(fx["frontier"]):
        x = [0] * len(oracle.FEATURES)
        x[oracle.F["frontier"]] = f
        x[oracle.F["level"]] = L
        feats.append(x)
    assert oracle.predict_schedule(fx["tree"], feats) == fx["schedule"]
    assert oracle.VARIANTS == tuple(fx["classes"])


def test_in_and_total_degree_features_directed_fixture():
    """Section 4.1's in- and total-degree summaries on the hand-derived directed
    fixture (tests/golden/directed6.json)."""
    import json
    fx = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "directed6.json")))
    src, dst = zip(*fx["edges"])
    g = gg.from_edges(fx["n"], list(src), list(dst), symmetrize=False)
    want = fx["degree_features"]
    res = oracle.bfs(g.off, g.idx, 0)
    feats = oracle.level_features(g.off, g.idx, res)
    F = oracle.F
    for x in feats:
        assert [x[F[k]] for k in ("deg_min", "deg_q1", "deg_med", "deg_q3", "deg_max", "deg_sd256")] == want["out"]
        assert [x[F[k]] for k in ("in_deg_min", "in_deg_q1", "in_deg_med", "in_deg_q3", "in_deg_max",
                                  "in_deg_sd256")] == want["in"]
        assert [x[F[k]] for k in ("tot_deg_min", "tot_deg_q1", "tot_deg_med", "tot_deg_q3", "tot_deg_max",
                                  "tot_deg_sd256")] == want["total"]


def test_in_degree_summary_is_the_transpose_out_degree_summary():
    """The in-degree summary equals the out-degree summary of the transposed
    graph (built by scipy); total degree against numpy's lower percentile; on a
    symmetric graph in = out and total = out + in."""
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(17)
    n = 700
    g = gg.from_edges(n, rng.integers(0, n, 4000), rng.integers(0, n - 50, 4000), symmetrize=False)
    a = sp.csr_matrix((np.ones(g.m), g.idx, g.off), shape=(n, n)).T.tocsr()
    res = oracle.bfs(g.off, g.idx, int(gg.sample_roots(g, 1, seed=3)[0]))
    x = oracle.level_features(g.off, g.idx, res)[0]
    F = oracle.F
    ins = [x[F[k]] for k in ("in_deg_min", "in_deg_q1", "in_deg_med", "in_deg_q3", "in_deg_max", "in_deg_sd256")]
    assert ins == oracle.degree_stats(a.indptr.astype(np.int32))
    tot = np.diff(g.off.astype(np.int64)) + np.diff(a.indptr.astype(np.int64))
    q = [int(np.percentile(tot, 25 * k, method="lower")) for k in range(5)]
    assert [x[F[k]] for k in ("tot_deg_min", "tot_deg_q1", "tot_deg_med", "tot_deg_q3", "tot_deg_max")] == q
    sd = 256.0 * float(np.std(tot))
    assert abs(x[F["tot_deg_sd256"]] - math.floor(sd)) <= 1
    s = gg.rmat(9, 8, seed=5)
    xs = oracle.level_features(s.off, s.idx, oracle.bfs(s.off, s.idx, 1))[0]
    assert xs[F["in_deg_min"]:F["in_deg_sd256"] + 1] == xs[F["deg_min"]:F["deg_sd256"] + 1]
    assert xs[F["tot_deg_max"]] == 2 * xs[F["deg_max"]] and xs[F["tot_deg_min"]] == 2 * xs[F["deg_min"]]
