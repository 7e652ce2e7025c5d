"""Seeded synthetic graph generators (input preparation only).

The generators build the int32 CSR graphs that both the CPU oracle and the GPU
library consume: R-MAT (Chakrabarti et al., SDM 2004), permuted 2D grids with
edge drops, and Erdos-Renyi G(n, p) by geometric skipping (Batagelj and
Brandes 2005). Every graph is symmetrised, stripped of self-loops and
duplicates, with each adjacency list sorted ascending. Randomness is SplitMix64
in counter mode, so the output does not depend on the thread count.

This module holds none of the BFS arithmetic; it only prepares inputs and root
samples, and it imports neither the oracle nor the GPU package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

# Seed conventions for the standard workloads: graph = 1000 + workload index
# (+ graph index within a set), roots = 2000 + ..., permutation derived inside.
SEED_GRAPH = 1000
SEED_ROOTS = 2000


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to this file (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CSR(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("m", ctypes.c_int64),
        ("off", ctypes.POINTER(ctypes.c_int32)),
        ("idx", ctypes.POINTER(ctypes.c_int32)),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER(_CSR)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.gg_rmat.restype = P
        lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_uint64, ctypes.c_int]
        lib.gg_grid.restype = P
        lib.gg_grid.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
        lib.gg_er.restype = P
        lib.gg_er.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64]
        lib.gg_from_pairs.restype = P
        lib.gg_from_pairs.argtypes = [ctypes.c_int64, ctypes.c_int64, i32p, i32p, ctypes.c_int]
        lib.gg_free.restype = None
        lib.gg_free.argtypes = [P]
        lib.gg_components.restype = ctypes.c_int64
        lib.gg_components.argtypes = [ctypes.c_int64, i32p, i32p, i32p, i32p]
        lib.gg_sample_roots.restype = ctypes.c_int32
        lib.gg_sample_roots.argtypes = [ctypes.c_int64, i32p, i32p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int,
                                        i32p]
        lib.gg_splitmix64_at.restype = ctypes.c_uint64
        lib.gg_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        _lib = lib
        return lib


class Graph:
    """A symmetric int32 CSR graph held in host memory (numpy)."""

    def __init__(self, off: np.ndarray, idx: np.ndarray, name: str = ""):
        self.off = np.ascontiguousarray(off, dtype=np.int32)
        self.idx = np.ascontiguousarray(idx, dtype=np.int32)
        self.name = name

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.idx.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.off.astype(np.int64))

    def __repr__(self) -> str:
        return f"Graph({self.name!r}, n={self.n}, m={self.m})"


def _i32p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _take(ptr, name: str) -> Graph:
    lib = _load()
    if not ptr:
        raise MemoryError(f"graph generation failed for {name}")
    c = ptr.contents
    n, m = int(c.n), int(c.m)
    off = np.ctypeslib.as_array(c.off, shape=(n + 1,)).copy()
    idx = np.ctypeslib.as_array(c.idx, shape=(max(m, 1),))[:m].copy()
    lib.gg_free(ptr)
    return Graph(off, idx, name)


def splitmix64_at(state: int, k: int) -> int:
    """Draw k (0-based) of the SplitMix64 stream starting at `state`."""
    return int(_load().gg_splitmix64_at(ctypes.c_uint64(state), ctypes.c_uint64(k)))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = SEED_GRAPH, permute: bool = False, directed: bool = False) -> Graph:
    """R-MAT graph with 2^scale vertices and edge_factor * 2^scale generated edges
    (directed: each generated edge kept in its direction, not symmetrised)."""
    ptr = _load().gg_rmat(scale, edge_factor, a, b, c, seed, int(permute) | (int(directed) << 1))
    return _take(ptr, f"rmat-s{scale}-ef{edge_factor}-seed{seed}{'-perm' if permute else ''}"
                      f"{'-dir' if directed else ''}")


def grid(rows: int, cols: int, drop: float = 0.1, seed: int = SEED_GRAPH, permute: bool = True) -> Graph:
    """rows x cols 4-neighbour lattice, undirected edges dropped with probability `drop`."""
    ptr = _load().gg_grid(rows, cols, drop, seed, int(permute))
    return _take(ptr, f"grid-{rows}x{cols}-drop{drop}-seed{seed}{'-perm' if permute else ''}")


def erdos_renyi(n: int, avg_degree: float, seed: int = SEED_GRAPH) -> Graph:
    """G(n, p) with p = avg_degree / (n - 1)."""
    ptr = _load().gg_er(n, avg_degree, seed)
    return _take(ptr, f"er-n{n}-d{avg_degree}-seed{seed}")


def from_edges(n: int, src, dst, symmetrize: bool = True, name: str = "edges") -> Graph:
    """CSR from an explicit edge list (self-loops and duplicates removed)."""
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    d = np.ascontiguousarray(np.asarray(dst, dtype=np.int32))
    if s.shape != d.shape:
        raise ValueError("src and dst must have the same length")
    ptr = _load().gg_from_pairs(n, s.shape[0], _i32p(s), _i32p(d), int(symmetrize))
    return _take(ptr, name)


def components(g: Graph):
    """(labels, giant_size, giant_label) of the undirected connected components."""
    comp = np.empty(max(g.n, 1), dtype=np.int32)
    lab = np.zeros(1, dtype=np.int32)
    sz = _load().gg_components(g.n, _i32p(g.off), _i32p(g.idx), _i32p(comp), _i32p(lab))
    if sz < 0:
        raise MemoryError("components: allocation failed")
    return comp[: g.n], int(sz), int(lab[0])


def sample_roots(g: Graph, k: int, seed: int = SEED_ROOTS, giant: bool = False) -> np.ndarray:
    """k distinct seeded roots of nonzero degree (optionally inside the giant component)."""
    out = np.empty(max(k, 1), dtype=np.int32)
    got = _load().gg_sample_roots(g.n, _i32p(g.off), _i32p(g.idx), k, seed, int(giant), _i32p(out))
    if got < 0:
        raise MemoryError("sample_roots: allocation failed")
    return out[:got].copy()


# Standard workloads, by what they are.
def rmat_s14_ef16(seed: int = SEED_GRAPH + 0) -> Graph:
    """R-MAT scale 14 (16,384 vertices), edge factor 16, a/b/c/d = .57/.19/.19/.05."""
    return rmat(14, 16, seed=seed)


def rmat_s22_ef16(seed: int = SEED_GRAPH + 1) -> Graph:
    """R-MAT scale 22 (4,194,304 vertices), edge factor 16, a/b/c/d = .57/.19/.19/.05."""
    return rmat(22, 16, seed=seed)


def grid_4096_permuted(seed: int = SEED_GRAPH + 2) -> Graph:
    """4096 x 4096 lattice, 10% of undirected edges dropped, vertex ids permuted."""
    return grid(4096, 4096, 0.1, seed=seed, permute=True)


def er_2p22_d8(seed: int = SEED_GRAPH + 3) -> Graph:
    """Erdos-Renyi with 2^22 vertices and average degree 8."""
    return erdos_renyi(1 << 22, 8.0, seed=seed)


def rmat_batch_specs(count: int = 32, seed: int = 6000):
    """The batch of uneven R-MAT graphs: `count` (scale, edge factor, graph
    seed, root seed) tuples, scale drawn from 12-20 and edge factor from
    {8, 16, 32} with a seeded generator; graph i is rmat(scale, ef,
    seed=seed + i) with 64 giant-component roots drawn with seed + 100 + i."""
    rng = np.random.default_rng(seed)
    specs = [(int(rng.integers(12, 21)), int(rng.choice([8, 16, 32]))) for _ in range(count)]
    return [(sc, ef, seed + i, seed + 100 + i) for i, (sc, ef) in enumerate(specs)]


def serve_graph_specs():
    """The eight graphs the query server holds resident: (name, maker) pairs.
    R-MAT scale 16/18/20/22/24 at edge factor 16, 2048^2 and 4096^2 permuted
    grids with 10% of edges dropped, Erdos-Renyi 2^21 with average degree 16."""
    return [("rmat16", lambda: rmat(16, 16, seed=5016)), ("rmat18", lambda: rmat(18, 16, seed=5018)),
            ("rmat20", lambda: rmat(20, 16, seed=5020)), ("rmat22", lambda: rmat(22, 16, seed=5022)),
            ("rmat24", lambda: rmat(24, 16, seed=5024)), ("grid2048", lambda: grid(2048, 2048, 0.1, seed=5025)),
            ("grid4096", lambda: grid(4096, 4096, 0.1, seed=5026)),
            ("er21", lambda: erdos_renyi(1 << 21, 16.0, seed=5027))]
