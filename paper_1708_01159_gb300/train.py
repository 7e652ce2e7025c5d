"""Training the per-level decision tree (Section 4.1, Section 4.2).

  collect  -- on a GPU: run the per-level timing harness (bfs_profile_levels)
              over a set of generated graphs and roots and write one CSV row
              per (graph, root, level): the 26 integer features and the median
              time of every variant expanding that level from the same state.
  train    -- label every level with its fastest variant, fit a CART tree
              (Gini impurity, scikit-learn) and export it in the integer text
              format bfs_load_tree reads: thresholds become floor(t) (the
              features are integers, so x <= t and x <= floor(t) agree), and a
              leaf whose two largest class weights tie is marked unknown (-1),
              the case Section 4.1 resolves by repeating the previous level's
              choice.
  evaluate -- per traversal, the time of the tree's schedule (unknown rule
              applied), of the best fixed variant and of every variant, each
              relative to the per-level optimum (the shape of Table 2).
  cv       -- k-fold cross-validation by graph over feature sets, weightings
              and depths.
  holdout  -- each generator family (R-MAT, directed R-MAT, grid, ER) held out
              in turn: trained on the others, evaluated on it (Section 4.4).
  level-split -- the paper's random 70/30 split over levels: held-out
              per-level accuracy, for comparison with its reported accuracy.

The benchmark's own graph (R-MAT scale 22, seed 1001) is never in the
training set. Graphs are split into train and test sets by graph, since the
levels of one traversal are correlated.

  python -m paper_1708_01159_gb300.train collect --out levels.csv
  python -m paper_1708_01159_gb300.train train --csv levels.csv --out trees/default.tree
  python -m paper_1708_01159_gb300.train evaluate --csv levels.csv --tree trees/default.tree
  python -m paper_1708_01159_gb300.train level-split --csv levels.csv
  python -m paper_1708_01159_gb300.train holdout --csv levels.csv
"""
from __future__ import annotations

import argparse
import csv
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_1708_01159_gb300 import FEATURES, NUM_FEATURES, NUM_VARIANTS, VARIANTS  # noqa: E402

LEVEL0_DEFAULT = 3  # Section 4.1: unknown at the first level -> edge list (edge-centric push)

# Feature sets (indices into FEATURES):
#   paper -- Section 4.2's best model: graph size, % of vertices discovered,
#            out-degree distribution, vertices in the frontier
#   m1    -- every feature Section 4.1 lists (frontier and discovered both
#            absolute and as a share of the vertices)
#   ext   -- m1 plus the frontier's edge count and the level index
#   *_io  -- the same plus the in-degree and total-degree summaries (Section
#            4.1 names the distribution of in-, out- or total degree), which
#            tell directed graphs apart
FEATURE_SETS = {
    "paper": [0, 1, 2, 3, 4, 5, 6, 7, 8, 11],
    "paper_io": [0, 1, 2, 3, 4, 5, 6, 7, 8, 11] + list(range(14, 26)),
    "m1": list(range(12)),
    "ext": list(range(14)),
    "ext_io": list(range(26)),
}

# Training graphs: (name, generator kwargs). Seeds start at 3000; the
# benchmark graph uses seed 1001 and is excluded by construction.
TRAIN_GRAPHS = [
    ("rmat", dict(scale=16, edge_factor=16, seed=3001)),
    ("rmat", dict(scale=18, edge_factor=8, seed=3002)),
    ("rmat", dict(scale=18, edge_factor=32, seed=3003)),
    ("rmat", dict(scale=20, edge_factor=16, seed=3004)),
    ("rmat", dict(scale=20, edge_factor=4, seed=3005)),
    ("rmat", dict(scale=21, edge_factor=16, seed=3006, permute=True)),
    ("rmat", dict(scale=22, edge_factor=16, seed=3007)),
    ("rmat", dict(scale=22, edge_factor=8, seed=3008)),
    ("rmat", dict(scale=19, edge_factor=16, seed=3009, a=0.45, b=0.15, c=0.15)),
    ("rmat", dict(scale=21, edge_factor=24, seed=3010, a=0.50, b=0.20, c=0.20)),
    ("grid", dict(rows=512, cols=512, drop=0.1, seed=3011)),
    ("grid", dict(rows=1024, cols=1024, drop=0.1, seed=3012)),
    ("grid", dict(rows=2048, cols=2048, drop=0.2, seed=3013)),
    ("grid", dict(rows=1500, cols=3000, drop=0.05, seed=3014)),
    ("er", dict(n=1 << 20, avg_degree=4.0, seed=3015)),
    ("er", dict(n=1 << 21, avg_degree=8.0, seed=3016)),
    ("er", dict(n=1 << 22, avg_degree=16.0, seed=3017)),
    ("er", dict(n=1 << 18, avg_degree=32.0, seed=3018)),
    # the workloads' own sizes, other seeds: 16.8M-vertex grids, 2^23 ER, scale 23 R-MAT
    ("grid", dict(rows=4096, cols=4096, drop=0.1, seed=3019)),
    ("grid", dict(rows=3000, cols=3000, drop=0.15, seed=3020)),
    ("er", dict(n=1 << 23, avg_degree=8.0, seed=3021)),
    ("rmat", dict(scale=23, edge_factor=16, seed=3022)),
    ("rmat", dict(scale=17, edge_factor=16, seed=3023, permute=True)),
    # directed R-MAT (not symmetrised): with b != c the in- and out-degree
    # distributions differ, and pull scans the transpose
    ("rmat", dict(scale=18, edge_factor=16, seed=3024, directed=True, b=0.30, c=0.08)),
    ("rmat", dict(scale=20, edge_factor=8, seed=3025, directed=True, b=0.08, c=0.30)),
    ("rmat", dict(scale=21, edge_factor=16, seed=3026, directed=True)),
    ("rmat", dict(scale=22, edge_factor=8, seed=3027, directed=True, b=0.25, c=0.13)),
]


def family(name: str) -> str:
    """Generator family of a training graph's name: rmat, rmat-dir, grid or er."""
    if name.startswith("rmat"):
        return "rmat-dir" if name.endswith("-dir") else "rmat"
    return name.split("-")[0]


def make_graph(kind, kw):
    import graphgen as gg
    if kind == "rmat":
        kw = dict(kw)
        return gg.rmat(kw.pop("scale"), kw.pop("edge_factor"), **kw)
    if kind == "grid":
        return gg.grid(kw["rows"], kw["cols"], kw["drop"], seed=kw["seed"], permute=True)
    if kind == "er":
        return gg.erdos_renyi(kw["n"], kw["avg_degree"], seed=kw["seed"])
    raise ValueError(kind)


def collect(out: str, roots_per_graph: int = 4, reps: int = 3, max_levels: int = 16384, graphs=None):
    import graphgen as gg
    import torch
    import paper_1708_01159_gb300 as bfs
    bfs.build()
    torch.cuda.set_device(0)
    graphs = graphs or TRAIN_GRAPHS
    cols = ["graph", "root", "level"] + list(FEATURES) + [f"ms_{v}" for v in VARIANTS] + ["tree_variant"]
    with open(out, "w", newline="") as fh:
        w = csv.writer(fh)
        w.writerow(cols)
        for kind, kw in graphs:
            t0 = time.time()
            g = make_graph(kind, kw)
            name = g.name
            roots = gg.sample_roots(g, roots_per_graph, seed=kw["seed"] + 500, giant=True)
            flags = 0 if kw.get("directed") else bfs.BFS_SYMMETRIC
            with bfs.Graph(g.off, g.idx, flags) as G:
                for r in roots:
                    feats, ms, tv = bfs.bfs_profile_levels(G.handle, int(r), reps=reps, capacity=max_levels)
                    for L in range(feats.shape[0]):
                        w.writerow([name, int(r), L] + [int(x) for x in feats[L]] + [f"{x:.5f}" for x in ms[L]]
                                   + [int(tv[L])])
            fh.flush()
            print(f"{name}: {len(roots)} roots in {time.time() - t0:.1f}s", file=sys.stderr, flush=True)


def load(csv_path: str):
    import gzip
    fh = gzip.open(csv_path, "rt") if csv_path.endswith(".gz") else open(csv_path)
    rows = list(csv.DictReader(fh))
    graph = np.array([r["graph"] for r in rows])
    root = np.array([int(r["root"]) for r in rows])
    level = np.array([int(r["level"]) for r in rows])
    X = np.array([[int(r[f]) for f in FEATURES] for r in rows], dtype=np.int64).reshape(-1, NUM_FEATURES)
    T = np.array([[float(r[f"ms_{v}"]) for v in VARIANTS] for r in rows]).reshape(-1, NUM_VARIANTS)
    return graph, root, level, X, T


def split_by_graph(graph, test_frac=0.3, seed=0):
    names = sorted(set(graph.tolist()))
    rng = np.random.default_rng(seed)
    rng.shuffle(names)
    k = max(1, int(round(test_frac * len(names))))
    test = set(names[:k])
    return np.array([g not in test for g in graph]), sorted(test)


def level_weights(T, trav, weighting):
    """Sample weights. 'uniform': the paper's plain classification. 'regret':
    a level weighs its spread of times (slowest minus fastest), so splits go
    where a wrong choice costs most. 'relregret': that spread divided by the
    traversal's per-level-optimal time, the level's share of the traversal
    slowdown that Table 2 averages."""
    if weighting == "uniform":
        return np.ones(len(T))
    spread = T.max(axis=1) - T.min(axis=1) + 1e-5
    if weighting == "regret":
        return spread
    opt = T.min(axis=1)
    tot = {}
    for k, t in zip(trav, opt):
        tot[k] = tot.get(k, 0.0) + t
    return spread / np.array([tot[k] for k in trav])


# The library evaluates trees of up to 64 leaves in their bit-parallel form,
# held in shared memory (larger ones are walked node by node in global
# memory, about 1 us per level); the exporter keeps to that.
MAX_LEAVES = 64


def fit(X, T, feature_idx, max_depth=8, min_samples_leaf=8, weighting="regret", trav=None, max_leaves=MAX_LEAVES):
    """CART with Gini impurity (Section 2.1); labels: the fastest variant per level."""
    from sklearn.tree import DecisionTreeClassifier
    y = T.argmin(axis=1)
    w = level_weights(T, trav if trav is not None else np.zeros(len(T)), weighting)
    clf = DecisionTreeClassifier(criterion="gini", max_depth=max_depth, min_samples_leaf=min_samples_leaf,
                                 max_leaf_nodes=max_leaves, random_state=0)
    clf.fit(X[:, feature_idx], y, sample_weight=w)
    return clf


def export(clf, feature_idx, path, meta=""):
    """Integer tree text: 'feature threshold left right value' per node."""
    t = clf.tree_
    lines = []
    for i in range(t.node_count):
        if t.children_left[i] < 0:
            v = t.value[i][0]
            order = np.argsort(v)[::-1]
            cls = clf.classes_
            top = int(cls[order[0]])
            tie = len(order) > 1 and math.isclose(float(v[order[0]]), float(v[order[1]]), rel_tol=1e-9)
            lines.append(f"-1 0 -1 -1 {-1 if tie else top}")
        else:
            f = int(feature_idx[t.feature[i]])
            lines.append(f"{f} {int(math.floor(t.threshold[i]))} {t.children_left[i]} {t.children_right[i]} -1")
    with open(path, "w") as fh:
        fh.write("# Decision tree trained on per-level GB300 timings (CART, Gini).\n")
        for m in meta.splitlines():
            fh.write(f"# {m}\n")
        fh.write("# Features: " + ", ".join(f"{i} {f}" for i, f in enumerate(FEATURES)) + "\n")
        fh.write("# Classes: " + ", ".join(f"{i} {v}" for i, v in enumerate(VARIANTS)) + "\n")
        fh.write(f"bfs-tree 1 {t.node_count}\n")
        fh.write("\n".join(lines) + "\n")


def read_tree(path):
    from paper_1708_01159_gb300.buildlib import parse_tree_text
    rows = parse_tree_text(open(path).read())
    return [{"f": f, "t": t, "l": l, "r": r, "v": v} for f, t, l, r, v in rows]


def walk(nodes, x):
    i = 0
    while nodes[i]["f"] >= 0:
        i = nodes[i]["l"] if x[nodes[i]["f"]] <= nodes[i]["t"] else nodes[i]["r"]
    return nodes[i]["v"]


def schedule_time(nodes, X, T, level):
    """Per-level choice with the unknown rule; returns the chosen variants."""
    out = np.empty(len(X), dtype=np.int64)
    for i in range(len(X)):
        v = walk(nodes, X[i])
        if v < 0:
            v = out[i - 1] if level[i] > 0 else LEVEL0_DEFAULT
        out[i] = v
    return out


def evaluate(graph, root, level, X, T, nodes, mask=None):
    """Table-2-shaped summary over traversals: slowdown vs the per-level optimum."""
    if mask is None:
        mask = np.ones(len(X), bool)
    keys = sorted(set(zip(graph[mask].tolist(), root[mask].tolist())))
    pred = schedule_time(nodes, X, T, level)
    rows = {"predicted": [], "best_fixed": []}
    for v in VARIANTS:
        rows[v] = []
    fixed_by_graph = {}
    for gname in set(graph[mask].tolist()):
        sel = mask & (graph == gname)
        fixed_by_graph[gname] = int(T[sel].sum(axis=0).argmin())
    acc_hits = 0
    for gname, r in keys:
        sel = np.nonzero(mask & (graph == gname) & (root == r))[0]
        opt = T[sel].min(axis=1).sum()
        rows["predicted"].append(T[sel, pred[sel]].sum() / opt)
        rows["best_fixed"].append(T[sel, fixed_by_graph[gname]].sum() / opt)
        for k, v in enumerate(VARIANTS):
            rows[v].append(T[sel, k].sum() / opt)
        acc_hits += int((pred[sel] == T[sel].argmin(axis=1)).sum())
    summary = {}
    for k, vals in rows.items():
        a = np.array(vals)
        summary[k] = {"optimal": float((a < 1.0 + 1e-9).mean()), "1-2x": float(((a >= 1) & (a <= 2)).mean()),
                      ">5x": float((a > 5).mean()), ">20x": float((a > 20).mean()), "average": float(a.mean()),
                      "worst": float(a.max())}
    summary["level_accuracy"] = acc_hits / int(mask.sum())
    summary["traversals"] = len(keys)
    return summary


def cross_validate(graph, root, level, X, T, folds=6, depths=(6, 8, 10), feature_sets=None,
                   weightings=("uniform", "regret", "relregret")):
    """Mean held-out slowdown vs the per-level optimum, k folds split by graph."""
    import tempfile
    names = sorted(set(graph.tolist()))
    rng = np.random.default_rng(1)
    rng.shuffle(names)
    fold_of = {nm: i % folds for i, nm in enumerate(names)}
    fold = np.array([fold_of[g] for g in graph])
    trav = np.array([f"{g}/{r}" for g, r in zip(graph, root)])
    for fs in sorted(feature_sets or FEATURE_SETS):
        for wt in weightings:
            for depth in depths:
                slow, worst, best_fixed = [], 0.0, []
                for k in range(folds):
                    tr, te = fold != k, fold == k
                    fidx = np.array(FEATURE_SETS[fs])
                    clf = fit(X[tr], T[tr], fidx, depth, 8, wt, trav[tr])
                    with tempfile.NamedTemporaryFile("w", suffix=".tree", delete=False) as fh:
                        path = fh.name
                    export(clf, fidx, path)
                    s = evaluate(graph, root, level, X, T, read_tree(path), te)
                    os.unlink(path)
                    slow.append(s["predicted"]["average"] * s["traversals"])
                    best_fixed.append(s["best_fixed"]["average"] * s["traversals"])
                    worst = max(worst, s["predicted"]["worst"])
                n = len(set(trav.tolist()))
                print(f"features={fs:5s} weighting={wt:9s} depth={depth:2d}: held-out mean {sum(slow) / n:.3f}x "
                      f"worst {worst:.2f}x (best fixed {sum(best_fixed) / n:.3f}x)", flush=True)


def level_split(graph, root, level, X, T, test_frac=0.3, seed=0, depths=(6, 8, 10)):
    """The paper's protocol (Section 2.1, Section 4.4): a random 70/30 split over
    levels, pooled across graphs, scored by held-out per-level accuracy (the
    predicted variant is the fastest one). Levels of one traversal are
    correlated, so this flatters a tree compared with the split by graph; it is
    reported for comparability. Also the share of held-out levels whose
    prediction is within 10 % of the fastest time."""
    rng = np.random.default_rng(seed)
    te = np.zeros(len(X), bool)
    te[rng.permutation(len(X))[: int(round(test_frac * len(X)))]] = True
    tr = ~te
    trav = np.array([f"{g}/{r}" for g, r in zip(graph, root)])
    y = T.argmin(axis=1)
    rows = np.nonzero(te)[0]
    for fs in sorted(FEATURE_SETS):
        fidx = np.array(FEATURE_SETS[fs])
        for wt in ("uniform", "relregret"):
            for depth in depths:
                clf = fit(X[tr], T[tr], fidx, depth, 8, wt, trav[tr])
                pred = clf.predict(X[te][:, fidx])
                acc = float((pred == y[te]).mean())
                near = float((T[rows, pred] <= 1.1 * T[rows].min(axis=1)).mean())
                print(f"features={fs:5s} weighting={wt:9s} depth={depth:2d}: held-out level accuracy {acc:.3f}, "
                      f"within 10 % of the fastest {near:.3f} ({int(te.sum())} of {len(X)} levels)", flush=True)


def holdout_families(graph, root, level, X, T, features="ext_io", weighting="relregret", depth=8, min_leaf=8):
    """Section 4.4's generality question on generated families: for each
    family (R-MAT, directed R-MAT, grid, Erdos-Renyi) in turn, train on the
    other families only and evaluate on this one; per family, the tree's and
    the best fixed variant's traversal time relative to the per-level optimum."""
    import tempfile
    fam = np.array([family(g) for g in graph])
    trav = np.array([f"{g}/{r}" for g, r in zip(graph, root)])
    fidx = np.array(FEATURE_SETS[features])
    print(f"held-out family (features={features} weighting={weighting} depth={depth}):")
    print(f"{'family':10s} {'traversals':>10s} {'tree/opt':>9s} {'worst':>7s} {'best fixed/opt':>15s} "
          f"{'tree <= best fixed':>19s}")
    out = {}
    for f in sorted(set(fam.tolist())):
        tr, te = fam != f, fam == f
        clf = fit(X[tr], T[tr], fidx, depth, min_leaf, weighting, trav[tr])
        with tempfile.NamedTemporaryFile("w", suffix=".tree", delete=False) as fh:
            path = fh.name
        export(clf, fidx, path)
        nodes = read_tree(path)
        os.unlink(path)
        pred = schedule_time(nodes, X, T, level)
        keys = sorted(set(zip(graph[te].tolist(), root[te].tolist())))
        fixed = {g: int(T[te & (graph == g)].sum(axis=0).argmin()) for g in set(graph[te].tolist())}
        rt, rb, wins = [], [], 0
        for g, r in keys:
            sel = np.nonzero(te & (graph == g) & (root == r))[0]
            opt = T[sel].min(axis=1).sum()
            t_tree = T[sel, pred[sel]].sum()
            t_fix = T[sel, fixed[g]].sum()
            rt.append(t_tree / opt)
            rb.append(t_fix / opt)
            wins += int(t_tree <= t_fix * 1.0001)
        out[f] = {"traversals": len(keys), "tree_over_opt": float(np.mean(rt)), "worst": float(np.max(rt)),
                  "best_fixed_over_opt": float(np.mean(rb)), "tree_le_best_fixed": wins / len(keys)}
        print(f"{f:10s} {len(keys):10d} {np.mean(rt):8.3f}x {np.max(rt):6.2f}x {np.mean(rb):14.3f}x "
              f"{wins / len(keys):18.0%}", flush=True)
    return out


def print_table(summary, file=sys.stdout):
    print(f"traversals: {summary['traversals']}, per-level accuracy: {summary['level_accuracy']:.3f}", file=file)
    print(f"{'algorithm':14s} {'optimal':>8s} {'1-2x':>7s} {'>5x':>6s} {'>20x':>6s} {'average':>8s} {'worst':>8s}",
          file=file)
    for k in ["predicted", "best_fixed"] + list(VARIANTS):
        s = summary[k]
        print(f"{k:14s} {s['optimal']:8.2%} {s['1-2x']:7.2%} {s['>5x']:6.2%} {s['>20x']:6.2%} "
              f"{s['average']:7.2f}x {s['worst']:7.2f}x", file=file)


def main():
    p = argparse.ArgumentParser()
    sub = p.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--out", required=True)
    c.add_argument("--roots", type=int, default=4)
    c.add_argument("--reps", type=int, default=3)
    t = sub.add_parser("train")
    t.add_argument("--csv", required=True)
    t.add_argument("--out", required=True)
    t.add_argument("--features", default="ext", choices=sorted(FEATURE_SETS))
    t.add_argument("--max-depth", type=int, default=8)
    t.add_argument("--min-leaf", type=int, default=8)
    t.add_argument("--weighting", default="relregret", choices=["regret", "uniform", "relregret"])
    t.add_argument("--all-graphs", action="store_true", help="train on every graph (no held-out split)")
    v = sub.add_parser("cv", help="k-fold cross-validation by graph over feature sets and weightings")
    v.add_argument("--csv", required=True)
    v.add_argument("--folds", type=int, default=6)
    v.add_argument("--features", nargs="*", default=None, choices=sorted(FEATURE_SETS))
    v.add_argument("--weightings", nargs="*", default=["uniform", "regret", "relregret"])
    ls = sub.add_parser("level-split", help="the paper's random 70/30 split over levels: held-out accuracy")
    ls.add_argument("--csv", required=True)
    h = sub.add_parser("holdout", help="leave each graph family out in turn (Section 4.4 generality)")
    h.add_argument("--csv", required=True)
    h.add_argument("--features", default="ext_io", choices=sorted(FEATURE_SETS))
    h.add_argument("--weighting", default="relregret", choices=["regret", "uniform", "relregret"])
    h.add_argument("--max-depth", type=int, default=8)
    e = sub.add_parser("evaluate")
    e.add_argument("--csv", required=True)
    e.add_argument("--tree", required=True)
    a = p.parse_args()
    if a.cmd == "collect":
        collect(a.out, a.roots, a.reps)
        return
    graph, root, level, X, T = load(a.csv)
    if a.cmd == "train":
        fidx = np.array(FEATURE_SETS[a.features])
        train_mask, test_graphs = split_by_graph(graph)
        if a.all_graphs:
            train_mask = np.ones(len(graph), bool)
        trav = np.array([f"{g}/{r}" for g, r in zip(graph, root)])
        clf = fit(X[train_mask], T[train_mask], fidx, a.max_depth, a.min_leaf, a.weighting, trav[train_mask])
        meta = (f"features={a.features} max_depth={a.max_depth} min_samples_leaf={a.min_leaf} "
                f"weighting={a.weighting}\nlevels={int(train_mask.sum())} "
                f"held-out graphs={'none' if a.all_graphs else ','.join(test_graphs)}")
        export(clf, fidx, a.out, meta)
        nodes = read_tree(a.out)
        print("train:")
        print_table(evaluate(graph, root, level, X, T, nodes, train_mask))
        if not a.all_graphs:
            print("held-out graphs:", ", ".join(test_graphs))
            print_table(evaluate(graph, root, level, X, T, nodes, ~train_mask))
    elif a.cmd == "cv":
        cross_validate(graph, root, level, X, T, a.folds, feature_sets=a.features, weightings=a.weightings)
    elif a.cmd == "level-split":
        level_split(graph, root, level, X, T)
    elif a.cmd == "holdout":
        holdout_families(graph, root, level, X, T, a.features, a.weighting, a.max_depth)
    else:
        print_table(evaluate(graph, root, level, X, T, read_tree(a.tree)))


if __name__ == "__main__":
    main()
