"""CPU oracle for per-level, model-switched BFS.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package; the GPU library never does, and this
package imports nothing from it. It shares no code with the GPU path: the two
agree only on the CSR format and on the numbering of the tree features and
variants, which both restate from the paper in their own code.

Contents (each function cites the passage it follows):
  bfs / bfs_batch    -- plain FIFO-queue BFS (Section 2.2, Section 3.1), in C
  validate_csr       -- CSR well-formedness (Section 4.3 names CSR as the
                        vertex-centric representation)
  degree_stats       -- 5-number summary and standard deviation of out-degrees
                        (Section 4.1, "Degree distribution")
  level_features     -- per-level feature vectors (Section 4.1, Section 4.2)
  tree_walk          -- decision-tree prediction walk (Section 2.1)
  predict_schedule   -- per-level prediction with the unknown-prediction rule
                        (Section 4.1)

Parity status: bfs, bfs_batch, validate_csr, degree_stats and tree_walk are
pinned by tests against brute force, closed forms, library routines and
invariants. predict_schedule is pinned through its parts (features from the
pinned BFS counts, the pinned walk, and hand-built trees that exercise the
unknown-prediction rule).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libbfs_oracle.so")
_lock = threading.Lock()
_lib = None

ORACLE_OK = 0
ORACLE_ERR_INVALID_ARG = 1
ORACLE_ERR_BAD_GRAPH = 2
ORACLE_ERR_OOM = 3


def build(force: bool = False, src: str | None = None, out: str | None = None) -> str:
    """Compile the oracle with gcc -O2 (no OpenMP: it is the plain definition)."""
    src = src or _SRC
    out = out or _LIB_PATH
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", src, "-o", tmp], check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_validate_csr.restype = ctypes.c_int
    lib.oracle_validate_csr.argtypes = [ctypes.c_int64, ctypes.c_int64, i32p, i32p]
    lib.oracle_bfs.restype = ctypes.c_int64
    lib.oracle_bfs.argtypes = [ctypes.c_int64, i32p, i32p, ctypes.c_int32, i32p, i64p, i64p, ctypes.c_int64, i64p]
    lib.oracle_bfs_batch.restype = ctypes.c_int
    lib.oracle_bfs_batch.argtypes = [ctypes.c_int64, i32p, i32p, i32p, ctypes.c_int64, i32p, i64p]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def load_variant(path: str):
    """Load another build of the oracle source (used by tests that plant a mistake)."""
    return _bind(ctypes.CDLL(path))


def _i32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _i64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def validate_csr(off: np.ndarray, idx: np.ndarray) -> int:
    """0 if off/idx form a well-formed CSR over n = len(off) - 1 vertices, else an error code."""
    off = np.ascontiguousarray(off, dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    if off.shape[0] < 1:
        return ORACLE_ERR_INVALID_ARG
    return int(_load().oracle_validate_csr(off.shape[0] - 1, idx.shape[0], _i32(off), _i32(idx)))


class BFSResult:
    """depth (int32, -1 = unreached), edges_reached, and per-level counts."""

    def __init__(self, depth, edges_reached, level_count, level_edges):
        self.depth = depth
        self.edges_reached = int(edges_reached)
        self.level_count = level_count  # vertices at depth L
        self.level_edges = level_edges  # sum of out-degrees of vertices at depth L

    @property
    def num_levels(self) -> int:
        return int(self.level_count.shape[0])


def bfs(off: np.ndarray, idx: np.ndarray, root: int, lib=None) -> BFSResult:
    """Single-source BFS from `root` (Section 2.2 problem, Section 3.1 init/termination)."""
    off = np.ascontiguousarray(off, dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    lib = lib or _load()
    n = off.shape[0] - 1
    depth = np.empty(max(n, 1), dtype=np.int32)
    cap = max(n, 1)
    cnt = np.zeros(cap, dtype=np.int64)
    edg = np.zeros(cap, dtype=np.int64)
    nl = np.zeros(1, dtype=np.int64)
    r = lib.oracle_bfs(n, _i32(off), _i32(idx if idx.size else np.zeros(1, np.int32)), int(root), _i32(depth),
                       _i64(cnt), _i64(edg), cap, _i64(nl))
    if r < 0:
        raise ValueError(f"oracle_bfs error {-r}")
    L = int(nl[0])
    return BFSResult(depth[:n], r, cnt[:L].copy(), edg[:L].copy())


def bfs_batch(off: np.ndarray, idx: np.ndarray, roots: Sequence[int]):
    """k independent runs (the oracle of multi-source BFS): (depth[k, n], edges[k])."""
    off = np.ascontiguousarray(off, dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    roots = np.ascontiguousarray(np.asarray(roots, dtype=np.int32))
    n = off.shape[0] - 1
    k = roots.shape[0]
    depth = np.empty((k, n), dtype=np.int32)
    edges = np.zeros(k, dtype=np.int64)
    rc = _load().oracle_bfs_batch(n, _i32(off), _i32(idx if idx.size else np.zeros(1, np.int32)), _i32(roots), k,
                                  _i32(depth), _i64(edges))
    if rc != 0:
        raise ValueError(f"oracle_bfs_batch error {rc}")
    return depth, edges


# ---------------------------------------------------------------------------
# Features (Section 4.1) and the decision tree (Section 2.1)
# ---------------------------------------------------------------------------

# Feature numbering. Section 4.1 lists graph size (vertices and edges), the
# frontier size and the discovered count (absolute or as a share of the
# vertices) and the degree distribution (5-number summary and standard
# deviation) of in-, out- or total degree; the level index and the frontier's
# edge count are kept alongside for the extended feature sets. The out-degree
# summary comes first, the in-degree and total-degree summaries last.
FEATURES = (
    "n", "m", "deg_min", "deg_q1", "deg_med", "deg_q3", "deg_max", "deg_sd256",
    "frontier", "frontier_ppm", "discovered", "discovered_ppm", "frontier_edges", "level",
    "in_deg_min", "in_deg_q1", "in_deg_med", "in_deg_q3", "in_deg_max", "in_deg_sd256",
    "tot_deg_min", "tot_deg_q1", "tot_deg_med", "tot_deg_q3", "tot_deg_max", "tot_deg_sd256",
)
F = {name: i for i, name in enumerate(FEATURES)}

# Variant numbering (the classes the tree predicts).
VARIANTS = ("push_thread", "push_warp", "push_cta", "push_edge", "pull")
V = {name: i for i, name in enumerate(VARIANTS)}
# Section 4.1: an unknown prediction at the first level defaults to the edge
# list implementation; the edge-centric push is that implementation here.
LEVEL0_DEFAULT = V["push_edge"]


def degree_summary(deg) -> list:
    """5-number summary and floor(256 * population std) of a degree sequence (Section 4.1).

    Quantile rule (the paper does not fix one): nearest rank on the sorted
    degrees, q_k = sorted[floor(k (n - 1) / 4)] for k = 0..4. The standard
    deviation is exact: floor(256 sigma) = isqrt(65536 (n S2 - S1^2)) // n with
    S1, S2 the sums of degrees and squared degrees.
    """
    deg = np.asarray(deg, dtype=np.int64)
    n = int(deg.shape[0])
    s = np.sort(deg)
    q = [int(s[(k * (n - 1)) // 4]) for k in range(5)]
    s1 = int(deg.sum())
    s2 = int((deg * deg).sum())
    sd256 = math.isqrt(65536 * (n * s2 - s1 * s1)) // n
    return q + [sd256]


def degree_stats(off: np.ndarray):
    """Out-degree summary: degree_summary of the row lengths."""
    return degree_summary(np.diff(np.asarray(off, dtype=np.int64)))


def in_degrees(off: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """In-degree of every vertex: how many adjacency entries name it."""
    n = int(np.asarray(off).shape[0] - 1)
    return np.bincount(np.asarray(idx, dtype=np.int64), minlength=n)[:n].astype(np.int64)


def level_features(off: np.ndarray, idx: np.ndarray, res: BFSResult):
    """One feature vector per BFS level L, describing the frontier being expanded.

    Section 4.1 features: graph size, frontier size, discovered count (absolute
    and in parts per million of the vertices, floor(1e6 * count / n)), the
    out-, in- and total-degree summaries. "Discovered" at level L counts every
    vertex of depth <= L, i.e. including the frontier itself.
    """
    off = np.asarray(off, dtype=np.int64)
    n = int(off.shape[0] - 1)
    m = int(off[-1])
    out_deg = np.diff(off)
    in_deg = in_degrees(off, idx)
    ds = degree_summary(out_deg)
    ins = degree_summary(in_deg)
    tot = degree_summary(out_deg + in_deg)
    rows = []
    disc = 0
    for L in range(res.num_levels):
        f = int(res.level_count[L])
        disc += f
        rows.append([n, m] + ds + [f, (1_000_000 * f) // n, disc, (1_000_000 * disc) // n,
                                   int(res.level_edges[L]), L] + ins + tot)
    return rows


def tree_walk(tree: dict, x: Sequence[int]) -> int:
    """Prediction walk (Section 2.1): from the root, compare the node's feature
    with its threshold and descend, until a leaf; return the leaf's class, or
    -1 for an unknown prediction. Split rule: x[f] <= t goes left.
    """
    nodes = tree["nodes"]
    i = 0
    while nodes[i]["f"] >= 0:
        nd = nodes[i]
        i = nd["l"] if int(x[nd["f"]]) <= int(nd["t"]) else nd["r"]
    return int(nodes[i]["v"])


def predict_schedule(tree: dict, feats) -> list:
    """Per-level variant choice with the unknown-prediction rule (Section 4.1):
    an unknown prediction at level L repeats level L-1's choice; at the first
    level it falls back to the edge list implementation.
    """
    out = []
    for L, x in enumerate(feats):
        v = tree_walk(tree, x)
        if v < 0:
            v = out[L - 1] if L > 0 else LEVEL0_DEFAULT
        out.append(v)
    return out


def bfs_python(off, idx, root):
    """Pure-Python FIFO BFS for tiny graphs (same definition as the C oracle)."""
    n = len(off) - 1
    depth = [-1] * n
    depth[root] = 0
    q = [root]
    h = 0
    while h < len(q):
        u = q[h]
        h += 1
        for e in range(off[u], off[u + 1]):
            v = idx[e]
            if depth[v] == -1:
                depth[v] = depth[u] + 1
                q.append(v)
    return depth
