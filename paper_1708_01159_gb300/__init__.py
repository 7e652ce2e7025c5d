"""GB300-native level-synchronous BFS with per-level kernel switching.

Implements the hot path of "Using Graph Properties to Speed-up GPU-based Graph
Traversal: A Model-driven Approach" (Verstraaten, Varbanescu, de Laat): BFS
over an int32 CSR graph where, at every level, a binary decision tree over
graph and frontier properties (Section 4.1) picks the kernel that expands the
level (Section 3.1 variants), evaluated on the device.

This module is a thin ctypes binding of libbfs.so (C ABI in include/bfs.h):
it marshals arguments (numpy host arrays, torch tensors, CUDA stream handles)
and calls the library under the same names. Every step of the traversal runs
in the library's CUDA kernels; there is no CPU fallback. If libbfs.so has not
been built, importing the functions raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbfs.so")
DEFAULT_TREE = os.path.join(_HERE, "trees", "default.tree")

BFS_OK = 0
BFS_ERR_INVALID_ARG = 1
BFS_ERR_BAD_GRAPH = 2
BFS_ERR_OOM = 3
BFS_ERR_CUDA = 4
BFS_ERR_TIMEOUT = 5
BFS_ERR_BUSY = 6
BFS_ERR_CANCELLED = 7
BFS_ERR_NOT_FOUND = 8

BFS_SYMMETRIC = 1
BFS_INPUT_ON_DEVICE = 2
BFS_VALIDATE = 4

MODE_DEFAULT = 0
MODE_PERSISTENT = 1
MODE_GRAPH = 2
MODE_HOST_LOOP = 3
MODES = {"default": MODE_DEFAULT, "persistent": MODE_PERSISTENT, "graph": MODE_GRAPH, "host_loop": MODE_HOST_LOOP}

VARIANT_TREE = -1
VARIANTS = ("push_thread", "push_warp", "push_cta", "push_edge", "pull")  # the tree's classes
NUM_VARIANTS = len(VARIANTS)
VARIANT_EDGE_LIST = 5
VARIANT_REVERSE_EDGE_LIST = 6
# every variant a run can be forced to: the tree's classes plus the whole-edge-list kernels
FORCED_VARIANTS = VARIANTS + ("edge_list", "reverse_edge_list")
NUM_FORCED_VARIANTS = len(FORCED_VARIANTS)
# bfs_options.count_mode: how vertex push appends reached vertices (Section 3.1.4 comparison)
COUNT_MODES = {"block": 0, "warp": 1, "atomic": 2}
FEATURES = ("n", "m", "deg_min", "deg_q1", "deg_med", "deg_q3", "deg_max", "deg_sd256",
            "frontier", "frontier_ppm", "discovered", "discovered_ppm", "frontier_edges", "level",
            "in_deg_min", "in_deg_q1", "in_deg_med", "in_deg_q3", "in_deg_max", "in_deg_sd256",
            "tot_deg_min", "tot_deg_q1", "tot_deg_med", "tot_deg_q3", "tot_deg_max", "tot_deg_sd256")
NUM_FEATURES = len(FEATURES)


class BFSError(RuntimeError):
    """A non-zero status from the library; .code is the bfs_status value."""

    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {status_string(code)} ({code}): {detail}")
        self.code = code


class _GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("deg_summary", ctypes.c_int64 * 5),
                ("deg_sd256", ctypes.c_int64), ("in_deg_summary", ctypes.c_int64 * 5), ("in_deg_sd256", ctypes.c_int64),
                ("tot_deg_summary", ctypes.c_int64 * 5), ("tot_deg_sd256", ctypes.c_int64),
                ("bytes_resident", ctypes.c_int64), ("symmetric", ctypes.c_int32), ("num_workspaces", ctypes.c_int32)]


class _Options(ctypes.Structure):
    _fields_ = [("forced_variant", ctypes.c_int32), ("depth_on_host", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("count_mode", ctypes.c_int32), ("host_async", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class _Stats(ctypes.Structure):
    _fields_ = [("edges_reached", ctypes.c_int64), ("vertices_reached", ctypes.c_int64), ("levels", ctypes.c_int32),
                ("status", ctypes.c_int32), ("log_capacity", ctypes.c_int32),
                ("log_variant", ctypes.POINTER(ctypes.c_int32)), ("log_frontier", ctypes.POINTER(ctypes.c_int64)),
                ("log_frontier_edges", ctypes.POINTER(ctypes.c_int64)), ("log_time_ns", ctypes.POINTER(ctypes.c_int64)),
                ("start_ns", ctypes.c_int64)]


class _ServeConfig(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("num_streams", ctypes.c_int32), ("queue_capacity", ctypes.c_int32), ("merge_batch", ctypes.c_int32),
                ("merge_policy", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("failed", ctypes.c_int64), ("peak_bytes_inflight", ctypes.c_int64),
                ("merged_waves", ctypes.c_int32), ("queued", ctypes.c_int32), ("qps", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("gteps", ctypes.c_double), ("wait_p50_ms", ctypes.c_double), ("wait_p99_ms", ctypes.c_double)]


class _BatchConfig(ctypes.Structure):
    _fields_ = [("push_mode", ctypes.c_int32), ("alpha", ctypes.c_int32), ("ms", ctypes.c_float),
                ("grid_blocks", ctypes.c_int32)]


# virtual-warp width policies of the push_warp variant (enum bfs_warp_width)
WARP_WIDTHS = ("rule", "rule_x2", "rule_half", "w4", "w8", "w16", "w32")


class _WarpTune(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_int32), ("reserved", ctypes.c_int32), ("ms", ctypes.c_float * len(WARP_WIDTHS))]


class _LevelProfile(ctypes.Structure):
    _fields_ = [("features", ctypes.c_int64 * NUM_FEATURES), ("ms", ctypes.c_float * NUM_VARIANTS),
                ("tree_variant", ctypes.c_int32), ("pad", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile libbfs.so in-tree (nvcc, sm_103a)."""
    from .buildlib import build as _build
    return _build(force=force)


def lib():
    """The loaded libbfs.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built (run paper_1708_01159_gb300.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        c_i32, c_i64, c_u32, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p
        sig = {
            "bfs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "bfs_last_error_detail": (ctypes.c_char_p, []),
            "bfs_version": (ctypes.c_int, []),
            "bfs_graph_create": (ctypes.c_int, [vp, vp, c_i64, c_i64, c_u32, ctypes.POINTER(vp)]),
            "bfs_graph_destroy": (ctypes.c_int, [vp]),
            "bfs_graph_info": (ctypes.c_int, [vp, ctypes.POINTER(_GraphInfo)]),
            "bfs_load_tree": (ctypes.c_int, [ctypes.c_char_p]),
            "bfs_run": (ctypes.c_int, [vp, c_i32, vp, vp]),
            "bfs_run_ex": (ctypes.c_int, [vp, c_i32, vp, vp, ctypes.POINTER(_Options), ctypes.POINTER(_Stats)]),
            "bfs_run_batch": (ctypes.c_int, [vp, vp, c_i32, vp, vp, vp]),
            "bfs_profile_levels": (ctypes.c_int, [vp, c_i32, c_i32, c_i32, vp, ctypes.POINTER(_LevelProfile), c_i32,
                                                  ctypes.POINTER(c_i32)]),
            "bfs_debug_fail_alloc_after": (ctypes.c_int, [ctypes.c_int]),
            "bfs_debug_stall_next_launch": (ctypes.c_int, [ctypes.c_int]),
            "bfs_run_static": (ctypes.c_int, [vp, vp, c_i64, c_i64, c_i32, vp, vp]),
            "bfs_set_warp_width": (ctypes.c_int, [vp, c_i32]),
            "bfs_get_warp_width": (ctypes.c_int, [vp, ctypes.POINTER(c_i32)]),
            "bfs_tune_warp_width": (ctypes.c_int, [vp, vp, c_i32, vp, ctypes.POINTER(_WarpTune)]),
            "bfs_batch_set_config": (ctypes.c_int, [vp, ctypes.POINTER(_BatchConfig)]),
            "bfs_batch_tune": (ctypes.c_int, [vp, vp, c_i32, vp, vp, ctypes.POINTER(_BatchConfig)]),
            "bfs_batch_tune_ex": (ctypes.c_int, [vp, vp, c_i32, vp, vp, c_i32, ctypes.POINTER(_BatchConfig)]),
            "bfs_serve_create": (ctypes.c_int, [ctypes.POINTER(_ServeConfig), ctypes.POINTER(vp)]),
            "bfs_serve_add_graph": (ctypes.c_int, [vp, vp, ctypes.POINTER(c_i32)]),
            "bfs_serve_graph_shape": (ctypes.c_int, [vp, c_i32, ctypes.POINTER(c_i32), ctypes.POINTER(c_i32)]),
            "bfs_serve_query_bytes": (ctypes.c_int, [vp, c_i32, c_i32, ctypes.POINTER(c_i64)]),
            "bfs_serve_reset_stats": (ctypes.c_int, [vp]),
            "bfs_serve_cancel_queued": (ctypes.c_int, [vp, ctypes.POINTER(c_i64)]),
            "bfs_serve_submit": (ctypes.c_int, [vp, c_i32, c_i32, vp, ctypes.POINTER(ctypes.c_uint64)]),
            "bfs_serve_poll": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
            "bfs_serve_wait": (ctypes.c_int, [vp, ctypes.c_uint64, c_i64]),
            "bfs_serve_stats": (ctypes.c_int, [vp, ctypes.POINTER(_ServeStats)]),
            "bfs_serve_destroy": (ctypes.c_int, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def status_string(code: int) -> str:
    """The library's text for a status code (the number itself if the library is not built)."""
    try:
        return lib().bfs_status_string(code).decode()
    except Exception:  # library unavailable
        return str(code)


def _check(code: int, where: str):
    if code != BFS_OK:
        raise BFSError(code, where, lib().bfs_last_error_detail().decode())


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype=np.int32, what="array"):
    """(pointer, on_device, numel) of a contiguous int32 numpy array or torch tensor."""
    if x is None:
        return None, False, 0
    if _is_torch(x):
        import torch
        want = {np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise ValueError(f"{what} must be a contiguous {want} tensor")
        return x.data_ptr(), x.is_cuda, x.numel()
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{what} must be a C-contiguous {np.dtype(dtype).name} array")
    return a.ctypes.data, False, a.size


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if _is_torch(stream):
        return stream.cuda_stream
    return int(stream)


def bfs_graph_create(row_offsets, col_indices, flags: int = BFS_SYMMETRIC) -> int:
    """Create a graph from a CSR (numpy host arrays or CUDA int32 tensors). Returns the handle."""
    po, dev_o, no = _ptr(row_offsets, what="row_offsets")
    pi, dev_i, ni = _ptr(col_indices, what="col_indices")
    if dev_o != dev_i:
        raise ValueError("row_offsets and col_indices must both be host or both be device memory")
    if dev_o:
        flags |= BFS_INPUT_ON_DEVICE
    out = ctypes.c_void_p()
    _check(lib().bfs_graph_create(po, pi, no - 1, ni, flags, ctypes.byref(out)), "bfs_graph_create")
    return out.value


def bfs_graph_destroy(g: int) -> None:
    """Free a graph and its workspaces once its runs have finished."""
    _check(lib().bfs_graph_destroy(g), "bfs_graph_destroy")


def bfs_graph_info(g: int) -> dict:
    """Sizes, out-degree 5-number summary and floor(256 sd), resident bytes, symmetry, workspace count."""
    info = _GraphInfo()
    _check(lib().bfs_graph_info(g, ctypes.byref(info)), "bfs_graph_info")
    return {"n": info.n, "m": info.m, "deg_summary": list(info.deg_summary), "deg_sd256": info.deg_sd256,
            "in_deg_summary": list(info.in_deg_summary), "in_deg_sd256": info.in_deg_sd256,
            "tot_deg_summary": list(info.tot_deg_summary), "tot_deg_sd256": info.tot_deg_sd256,
            "bytes_resident": info.bytes_resident, "symmetric": bool(info.symmetric),
            "num_workspaces": info.num_workspaces}


def bfs_load_tree(path: Optional[str] = None) -> None:
    """Load the process-wide decision tree from a tree file (None: the built-in tree)."""
    _check(lib().bfs_load_tree(path.encode() if path else None), "bfs_load_tree")


def bfs_run(g: int, root: int, depth_out, stream=None) -> None:
    """Asynchronous BFS from `root` into depth_out (CUDA int32 tensor of n entries)."""
    p, dev, _ = _ptr(depth_out, what="depth_out")
    if not dev:
        raise ValueError("bfs_run writes device memory; use bfs_run_ex(depth_on_host=True) for host output")
    _check(lib().bfs_run(g, int(root), p, _stream(stream)), "bfs_run")


def bfs_run_ex(g: int, root: int, depth_out, stream=None, forced_variant: int = VARIANT_TREE,
               depth_on_host: Optional[bool] = None, stats: bool = False, log_capacity: int = 0,
               mode: int = MODE_DEFAULT, grid_blocks: int = 0, count_mode: int = 0, host_async: bool = False):
    """BFS with options. Returns a stats dict when stats=True (then the stream is synchronised).
    grid_blocks: persistent driver only, blocks of the cooperative grid (0: a full occupancy wave).
    count_mode: host-loop driver only, how vertex push appends to the next queue (COUNT_MODES).
    host_async: with host output (pinned) and no stats, return once the copy is enqueued on the
    stream; synchronise the stream before reading depth_out."""
    p, dev, _ = _ptr(depth_out, what="depth_out")
    host = (not dev) if depth_on_host is None else bool(depth_on_host)
    opts = _Options(forced_variant=int(forced_variant), depth_on_host=int(host), mode=int(mode),
                    grid_blocks=int(grid_blocks), count_mode=int(count_mode), host_async=int(bool(host_async)))
    st = None
    logs = None
    if stats:
        st = _Stats()
        if log_capacity > 0:
            logs = (np.zeros(log_capacity, np.int32), np.zeros(log_capacity, np.int64),
                    np.zeros(log_capacity, np.int64), np.zeros(log_capacity + 1, np.int64))
            st.log_capacity = log_capacity
            st.log_variant = logs[0].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            st.log_frontier = logs[1].ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
            st.log_frontier_edges = logs[2].ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
            st.log_time_ns = logs[3].ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    _check(lib().bfs_run_ex(g, int(root), p, _stream(stream), ctypes.byref(opts),
                            ctypes.byref(st) if st is not None else None), "bfs_run_ex")
    if st is None:
        return None
    out = {"edges_reached": st.edges_reached, "vertices_reached": st.vertices_reached, "levels": st.levels,
           "status": st.status}
    if logs is not None:
        k = min(st.levels, log_capacity)
        out["variant"] = logs[0][:k].copy()
        out["frontier"] = logs[1][:k].copy()
        out["frontier_edges"] = logs[2][:k].copy()
        # per-level device time (ns) from the start stamps (graph and persistent drivers)
        if st.levels < log_capacity + 1 and mode != MODE_HOST_LOOP:
            out["level_ns"] = np.diff(logs[3][: st.levels + 1])
            # from the first kernel's start to level 0 (depth init, first barrier), and to the end
            out["init_ns"] = int(logs[3][0] - st.start_ns)
            out["device_ns"] = int(logs[3][st.levels] - st.start_ns)
    return out


def bfs_run_batch(g: int, roots, depth_out, stream=None, edges: bool = False):
    """k traversals (host roots) into depth_out (CUDA int32 tensor of k * n, row-major)."""
    r = np.ascontiguousarray(np.asarray(roots, dtype=np.int32))
    p, dev, _ = _ptr(depth_out, what="depth_out")
    if not dev:
        raise ValueError("depth_out must be device memory")
    e = np.zeros(max(r.size, 1), np.int64) if edges else None
    _check(lib().bfs_run_batch(g, r.ctypes.data, r.size, p, _stream(stream),
                               e.ctypes.data if e is not None else None), "bfs_run_batch")
    return e[: r.size] if e is not None else None


def bfs_set_warp_width(g: int, policy) -> None:
    """Set a graph's virtual-warp width policy (an index or a name of WARP_WIDTHS)."""
    p = WARP_WIDTHS.index(policy) if isinstance(policy, str) else int(policy)
    _check(lib().bfs_set_warp_width(g, p), "bfs_set_warp_width")


def bfs_get_warp_width(g: int) -> int:
    """A graph's virtual-warp width policy (index into WARP_WIDTHS)."""
    p = ctypes.c_int32(0)
    _check(lib().bfs_get_warp_width(g, ctypes.byref(p)), "bfs_get_warp_width")
    return p.value


def bfs_tune_warp_width(g: int, roots, stream=None) -> dict:
    """Autotune the width policy on these roots (synchronous): the fastest is set
    on the graph; returns it and every policy's device time in ms."""
    r = np.ascontiguousarray(np.asarray(roots, dtype=np.int32))
    out = _WarpTune()
    _check(lib().bfs_tune_warp_width(g, r.ctypes.data, int(r.size), _stream(stream), ctypes.byref(out)),
           "bfs_tune_warp_width")
    return {"policy": out.policy, "name": WARP_WIDTHS[out.policy],
            "ms": {WARP_WIDTHS[i]: float(out.ms[i]) for i in range(len(WARP_WIDTHS))}}


def warp_width_cache_key(device_name: str, info: dict) -> str:
    """Key of a graph in the width-tuning cache: the GPU's name and the graph's
    class (size and out-degree summary)."""
    deg = ",".join(str(int(x)) for x in info["deg_summary"])
    return f"{device_name}|n={info['n']}|m={info['m']}|deg={deg}"


def tune_warp_width_cached(g: int, roots, cache_path: str, device_name: str, info: dict, stream=None) -> dict:
    """The width policy from a JSON cache (keyed by warp_width_cache_key), or
    tuned on `roots` and added to the cache; the policy is set on the graph."""
    import json
    key = warp_width_cache_key(device_name, info)
    cache = {}
    if os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
    if key in cache:
        bfs_set_warp_width(g, cache[key]["policy"])
        return dict(cache[key], cached=True)
    res = bfs_tune_warp_width(g, roots, stream)
    cache[key] = res
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return dict(res, cached=False)


def bfs_batch_set_config(g: int, push_mode: int, alpha: int, grid_blocks: int = 0) -> None:
    """Fix the multi-source launch shape of a graph: push_mode 0 (thread per vertex,
    block for hubs) or 1 (warp per vertex), pull when frontier edges x alpha > m,
    grid_blocks (0: a grid sized to the graph, one block per 4096 vertices within [SMs / 4, a full wave])."""
    c = _BatchConfig(push_mode=push_mode, alpha=alpha, grid_blocks=grid_blocks)
    _check(lib().bfs_batch_set_config(g, ctypes.byref(c)), "bfs_batch_set_config")


def bfs_batch_tune(g: int, roots, depth_scratch, stream=None, concurrency: int = 1) -> dict:
    """Autotune the multi-source kernel on up to 64 roots; returns the chosen
    configuration. concurrency > 1: for waves of that many graphs running at
    once (grids up to a full wave / concurrency)."""
    r = np.ascontiguousarray(np.asarray(roots, dtype=np.int32))
    p, dev, _ = _ptr(depth_scratch, what="depth_scratch")
    if not dev:
        raise ValueError("depth_scratch must be device memory")
    c = _BatchConfig()
    _check(lib().bfs_batch_tune_ex(g, r.ctypes.data, r.size, p, _stream(stream), int(concurrency), ctypes.byref(c)),
           "bfs_batch_tune")
    return {"push_mode": c.push_mode, "alpha": c.alpha, "ms": c.ms, "grid_blocks": c.grid_blocks}


def bfs_profile_levels(g: int, root: int, reps: int = 5, advance_variant: int = VARIANT_TREE, stream=None,
                       capacity: int = 4096):
    """Per-level timing harness: for every level, time each variant from the same
    state (median of `reps`). Returns (features[L, F], ms[L, V], tree_variant[L])."""
    buf = (_LevelProfile * capacity)()
    nl = ctypes.c_int32(0)
    _check(lib().bfs_profile_levels(g, int(root), int(reps), int(advance_variant), _stream(stream), buf, capacity,
                                    ctypes.byref(nl)), "bfs_profile_levels")
    k = min(nl.value, capacity)
    feats = np.array([list(buf[i].features) for i in range(k)], dtype=np.int64).reshape(k, NUM_FEATURES)
    ms = np.array([list(buf[i].ms) for i in range(k)], dtype=np.float64).reshape(k, NUM_VARIANTS)
    tv = np.array([buf[i].tree_variant for i in range(k)], dtype=np.int32)
    return feats, ms, tv


def bfs_debug_stall_next_launch(mode: int) -> None:
    """Test hook: the next persistent traversal or multi-source wave lets one
    bounded device wait run out (1 first grid barrier, 2 first level barrier,
    3 first staged copy of the CTA push; 0 clears), so the run reports
    BFS_ERR_TIMEOUT after about 2 s instead of finishing."""
    _check(lib().bfs_debug_stall_next_launch(int(mode)), "bfs_debug_stall_next_launch")


def bfs_run_static(row_offsets, col_indices, root: int, depth_out, stream=None) -> None:
    """BFS that allocates nothing, for callers that cannot allocate device memory
    while they run. All three arrays are CUDA int32 tensors the caller owns; the
    library's scratch is a fixed array inside libbfs.so, so n is limited to
    1,048,576 vertices and calls must not overlap on the GPU. Synchronous."""
    po, do, no = _ptr(row_offsets, what="row_offsets")
    pi, di, ni = _ptr(col_indices, what="col_indices")
    pd, dd, nd = _ptr(depth_out, what="depth_out")
    if not (do and di and dd):
        raise ValueError("bfs_run_static takes device arrays only")
    if nd != no - 1:
        raise ValueError("depth_out must have n = len(row_offsets) - 1 entries")
    _check(lib().bfs_run_static(po, pi, no - 1, ni, int(root), pd, _stream(stream)), "bfs_run_static")


def bfs_serve_create(mem_budget_bytes: int = 0, max_inflight: int = 16, num_streams: int = 8,
                     queue_capacity: int = 1 << 16, merge_batch: int = 0, merge_policy: int = 0) -> int:
    """Start a query server (its dispatcher thread owns the device side); returns its handle.
    mem_budget_bytes: admission budget (0: none); max_inflight: units on the device at once;
    merge_batch: most roots per merged multi-source wave (0 or 1: no merging); merge_policy:
    0 merges where the registration probe found waves cheaper, 1 merges always."""
    c = _ServeConfig(mem_budget_bytes=mem_budget_bytes, max_inflight=max_inflight, num_streams=num_streams,
                     queue_capacity=queue_capacity, merge_batch=merge_batch, merge_policy=merge_policy)
    out = ctypes.c_void_p()
    _check(lib().bfs_serve_create(ctypes.byref(c), ctypes.byref(out)), "bfs_serve_create")
    return out.value


def bfs_serve_add_graph(s: int, g: int) -> int:
    """Register a resident graph with the server (probes its query shape); returns its graph id."""
    gid = ctypes.c_int32()
    _check(lib().bfs_serve_add_graph(s, g, ctypes.byref(gid)), "bfs_serve_add_graph")
    return gid.value


def bfs_serve_graph_shape(s: int, graph_id: int) -> dict:
    """Launch shape registration chose for a graph: query blocks and whether its queries merge."""
    b, m = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib().bfs_serve_graph_shape(s, int(graph_id), ctypes.byref(b), ctypes.byref(m)), "bfs_serve_graph_shape")
    return {"query_blocks": b.value, "merges": bool(m.value)}


def bfs_serve_query_bytes(s: int, graph_id: int, with_output: bool = False) -> int:
    """Device bytes one query of the graph is charged against the memory budget."""
    b = ctypes.c_int64()
    _check(lib().bfs_serve_query_bytes(s, int(graph_id), int(bool(with_output)), ctypes.byref(b)),
           "bfs_serve_query_bytes")
    return int(b.value)


def bfs_serve_submit(s: int, graph_id: int, root: int, depth_out=None) -> int:
    """Queue one query; returns its ticket. Raises BFSError(BFS_ERR_BUSY) when the queue is full."""
    p = None
    if depth_out is not None:
        p, dev, _ = _ptr(depth_out, what="depth_out")
        if not dev:
            raise ValueError("depth_out must be device memory")
    t = ctypes.c_uint64()
    _check(lib().bfs_serve_submit(s, int(graph_id), int(root), p, ctypes.byref(t)), "bfs_serve_submit")
    return t.value


def bfs_serve_poll(s: int, ticket: int):
    """(state, status): state 0 done, 1 queued, 2 running."""
    st = ctypes.c_int()
    rc = lib().bfs_serve_poll(s, ticket, ctypes.byref(st))
    if rc == BFS_ERR_NOT_FOUND:
        _check(rc, "bfs_serve_poll")
    return st.value, rc


def bfs_serve_wait(s: int, ticket: int, timeout_us: int = -1) -> int:
    """The query's status once done; BFS_ERR_TIMEOUT if still pending after timeout_us."""
    return int(lib().bfs_serve_wait(s, ticket, int(timeout_us)))


def bfs_serve_stats(s: int) -> dict:
    """Counters, queries/s, GTEPS, latency and queue-wait percentiles since creation or the last reset."""
    st = _ServeStats()
    _check(lib().bfs_serve_stats(s, ctypes.byref(st)), "bfs_serve_stats")
    return {f: getattr(st, f) for f, _ in _ServeStats._fields_}


def bfs_serve_reset_stats(s: int) -> None:
    """Start a new statistics window."""
    _check(lib().bfs_serve_reset_stats(s), "bfs_serve_reset_stats")


def bfs_serve_cancel_queued(s: int) -> int:
    """Cancel every query not yet admitted; returns how many."""
    k = ctypes.c_int64(0)
    _check(lib().bfs_serve_cancel_queued(s, ctypes.byref(k)), "bfs_serve_cancel_queued")
    return k.value


def bfs_serve_destroy(s: int) -> None:
    """Stop the server: queued queries are cancelled, running ones finish."""
    _check(lib().bfs_serve_destroy(s), "bfs_serve_destroy")


class Graph:
    """Owning wrapper of a bfs_graph_t handle."""

    def __init__(self, row_offsets, col_indices, flags: int = BFS_SYMMETRIC):
        self.handle = bfs_graph_create(row_offsets, col_indices, flags)
        info = bfs_graph_info(self.handle)
        self.n, self.m = info["n"], info["m"]

    def info(self) -> dict:
        return bfs_graph_info(self.handle)

    def run(self, root: int, depth_out, stream=None) -> None:
        bfs_run(self.handle, root, depth_out, stream)

    def close(self) -> None:
        if self.handle:
            bfs_graph_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
