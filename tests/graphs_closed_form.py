"""Small graphs whose BFS distances have closed forms, for pinning the oracle
and for GPU parity edge cases. Each returns (Graph, expected_depth_fn(root))."""
from __future__ import annotations

import itertools

import numpy as np

import graphgen as gg


def csr_from_adj(adj: np.ndarray) -> gg.Graph:
    """CSR of a dense boolean adjacency matrix (row u lists the out-neighbours of u)."""
    n = adj.shape[0]
    off = np.zeros(n + 1, dtype=np.int32)
    idx = []
    for u in range(n):
        nb = np.nonzero(adj[u])[0]
        idx.extend(int(v) for v in nb)
        off[u + 1] = len(idx)
    return gg.Graph(off, np.asarray(idx, dtype=np.int32), "dense")


def brute_force_depth(adj: np.ndarray, root: int) -> np.ndarray:
    """d(v) = min k such that a walk of length k leads from root to v, by dense
    boolean row-vector / matrix products (w_k = w_{k-1} A), -1 if none within n
    steps. A different algorithm from the FIFO oracle: no queue, no visited set."""
    n = adj.shape[0]
    A = adj.astype(np.int64)
    w = np.zeros(n, dtype=np.int64)
    w[root] = 1
    d = np.full(n, -1, dtype=np.int64)
    for k in range(n + 1):
        newly = (w > 0) & (d < 0)
        d[newly] = k
        w = (w @ A > 0).astype(np.int64)
    return d.astype(np.int32)


def path(n):
    g = gg.from_edges(n, np.arange(n - 1), np.arange(1, n), name=f"path{n}")
    return g, lambda r: np.abs(np.arange(n) - r).astype(np.int32)


def cycle(n):
    g = gg.from_edges(n, np.arange(n), (np.arange(n) + 1) % n, name=f"cycle{n}")

    def f(r):
        a = np.abs(np.arange(n) - r)
        return np.minimum(a, n - a).astype(np.int32)
    return g, f


def star(n):
    g = gg.from_edges(n, np.zeros(n - 1, dtype=np.int32), np.arange(1, n), name=f"star{n}")

    def f(r):
        if r == 0:
            d = np.ones(n, dtype=np.int32)
        else:
            d = np.full(n, 2, dtype=np.int32)
            d[0] = 1
        d[r] = 0
        return d
    return g, f


def complete(n):
    s, t = zip(*itertools.combinations(range(n), 2))
    g = gg.from_edges(n, s, t, name=f"K{n}")

    def f(r):
        d = np.ones(n, dtype=np.int32)
        d[r] = 0
        return d
    return g, f


def binary_tree(levels):
    n = (1 << levels) - 1
    child = np.arange(1, n)
    parent = (child - 1) // 2
    g = gg.from_edges(n, parent, child, name=f"bintree{levels}")

    def f(r):
        # distance in a tree = depth(u) + depth(v) - 2 depth(lca)
        out = np.empty(n, dtype=np.int32)
        for v in range(n):
            a, b = r + 1, v + 1  # heap numbering from 1
            da, db = a.bit_length(), b.bit_length()
            x, y = a, b
            while x.bit_length() > y.bit_length():
                x >>= 1
            while y.bit_length() > x.bit_length():
                y >>= 1
            while x != y:
                x >>= 1
                y >>= 1
            dl = x.bit_length()
            out[v] = (da - dl) + (db - dl)
        return out
    return g, f


def hypercube(dim):
    n = 1 << dim
    s, t = [], []
    for v in range(n):
        for b in range(dim):
            w = v ^ (1 << b)
            if v < w:
                s.append(v)
                t.append(w)
    g = gg.from_edges(n, s, t, name=f"Q{dim}")

    def f(r):
        return np.array([bin(v ^ r).count("1") for v in range(n)], dtype=np.int32)
    return g, f


def full_grid_permuted(rows, cols, seed=7):
    """Undamaged lattice under a random relabelling: distance = Manhattan distance."""
    n = rows * cols
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n).astype(np.int32)  # old id -> new id
    s, t = [], []
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            if c + 1 < cols:
                s.append(v)
                t.append(v + 1)
            if r + 1 < rows:
                s.append(v)
                t.append(v + cols)
    s = perm[np.asarray(s)]
    t = perm[np.asarray(t)]
    g = gg.from_edges(n, s, t, name=f"grid{rows}x{cols}-perm")
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)

    def f(r):
        old = inv[r]
        rr, rc = divmod(int(old), cols)
        olds = inv  # new id -> old id
        orow, ocol = olds // cols, olds % cols
        return (np.abs(orow - rr) + np.abs(ocol - rc)).astype(np.int32)
    return g, f


def disjoint_union(parts):
    """Union of closed-form graphs: vertices outside the root's part are unreached."""
    offs, idxs, fns, sizes = [], [], [], []
    base = 0
    eoff = 0
    for g, fn in parts:
        offs.append(g.off[:-1].astype(np.int64) + eoff)
        idxs.append(g.idx.astype(np.int64) + base)
        fns.append(fn)
        sizes.append(g.n)
        base += g.n
        eoff += g.m
    n = base
    idx = np.concatenate(idxs).astype(np.int32)
    off = np.concatenate(offs + [np.array([idx.shape[0]])]).astype(np.int32)
    g = gg.Graph(off, idx, "union")
    starts = np.cumsum([0] + sizes)

    def f(r):
        d = np.full(n, -1, dtype=np.int32)
        p = int(np.searchsorted(starts, r, side="right") - 1)
        d[starts[p]:starts[p + 1]] = fns[p](r - starts[p])
        return d
    return g, f


def isolated_root(n=10):
    """Vertex 0 has no edges; the rest form a path."""
    g = gg.from_edges(n, np.arange(1, n - 1), np.arange(2, n), name="isolated0")

    def f(r):
        d = np.full(n, -1, dtype=np.int32)
        if r == 0:
            d[0] = 0
        else:
            d[1:] = np.abs(np.arange(1, n) - r)
        return d
    return g, f


ALL = {
    "path17": lambda: path(17),
    "cycle16": lambda: cycle(16),
    "cycle15": lambda: cycle(15),
    "star9": lambda: star(9),
    "K7": lambda: complete(7),
    "bintree5": lambda: binary_tree(5),
    "Q6": lambda: hypercube(6),
    "grid7x9": lambda: full_grid_permuted(7, 9),
    "union": lambda: disjoint_union([cycle(6), path(5), star(4)]),
    "isolated": lambda: isolated_root(10),
}
