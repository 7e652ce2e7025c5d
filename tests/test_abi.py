"""The C ABI library builds, loads and exports every symbol include/bfs.h
declares; host-side argument checks and tree parsing work without a GPU."""
import ctypes
import os
import re

import pytest

import paper_1708_01159_gb300 as bfs
from paper_1708_01159_gb300 import buildlib as bfs_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bfs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(bfs_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    bfs.build()
    return bfs.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("bfs_graph_create", "bfs_graph_destroy", "bfs_graph_info", "bfs_load_tree", "bfs_run",
                 "bfs_run_ex", "bfs_run_batch", "bfs_profile_levels", "bfs_status_string"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_status_strings(lib):
    assert bfs.status_string(bfs.BFS_OK) == "ok"
    assert bfs.status_string(bfs.BFS_ERR_TIMEOUT) == "timed out"
    assert lib.bfs_version() >= 100


def test_host_side_argument_checks(lib):
    import numpy as np
    off = np.array([0, 1, 2], np.int32)
    idx = np.array([1, 0], np.int32)
    out = ctypes.c_void_p()
    # n < 1, unknown flags and null output are rejected before any CUDA call
    assert lib.bfs_graph_create(off.ctypes.data, idx.ctypes.data, 0, 2, 1, ctypes.byref(out)) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_graph_create(off.ctypes.data, idx.ctypes.data, 2, 2, 1 << 7, ctypes.byref(out)) == \
        bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_graph_create(off.ctypes.data, idx.ctypes.data, 2, 2, 1, None) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_graph_create(None, idx.ctypes.data, 2, 2, 1, ctypes.byref(out)) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_run(None, 0, None, None) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_graph_destroy(None) == bfs.BFS_OK


def test_tree_files(lib, tmp_path):
    # the built-in tree file parses on both sides
    rows = bfs_build.parse_tree_text(open(bfs.DEFAULT_TREE).read())
    assert rows and all(len(r) == 5 for r in rows)
    bfs.bfs_load_tree(bfs.DEFAULT_TREE)
    bfs.bfs_load_tree(None)
    with pytest.raises(bfs.BFSError) as e:
        bfs.bfs_load_tree(str(tmp_path / "missing.tree"))
    assert e.value.code == bfs.BFS_ERR_NOT_FOUND
    bad = tmp_path / "bad.tree"
    # a cycle (child index not greater than its parent) must be rejected
    bad.write_text("bfs-tree 1 2\n8 5 0 1 -1\n-1 0 -1 -1 3\n")
    with pytest.raises(bfs.BFSError) as e:
        bfs.bfs_load_tree(str(bad))
    assert e.value.code == bfs.BFS_ERR_INVALID_ARG
    bad.write_text("bfs-tree 1 1\n-1 0 -1 -1 9\n")  # class out of range
    with pytest.raises(bfs.BFSError):
        bfs.bfs_load_tree(str(bad))
    bad.write_text("bfs-tree 1 3\n99 5 1 2 -1\n-1 0 -1 -1 3\n-1 0 -1 -1 4\n")  # feature out of range
    with pytest.raises(bfs.BFSError):
        bfs.bfs_load_tree(str(bad))
    good_leaves = "-1 0 -1 -1 3\n-1 0 -1 -1 4\n"
    for text in (
        "bfs-tree 1 3\n4294967304 5 1 2 -1\n" + good_leaves,  # feature 2^32 + 8 must not wrap to 8
        "bfs-tree 1 3\n8 5 4294967297 2 -1\n" + good_leaves,  # child 2^32 + 1 must not wrap to 1
        "bfs-tree 1 1\n-1 0 -1 -1 4294967297\n",              # class 2^32 + 1 must not wrap to 1
        "bfs-tree 1 3\n8 5 1 3 -1\n" + good_leaves,            # child past the last node
        "bfs-tree 2 3\n8 5 1 2 -1\n" + good_leaves,            # unknown format version
        "bfs-tree 1 0\n",                                       # no nodes
        "bfs-tree 1 4\n8 5 1 2 -1\n" + good_leaves,            # fewer nodes than declared
        "bfs-tree 1 3\n8 five 1 2 -1\n" + good_leaves,         # not a number
        "8 5 1 2 -1\n" + good_leaves,                            # no header
    ):
        bad.write_text(text)
        with pytest.raises(bfs.BFSError) as e:
            bfs.bfs_load_tree(str(bad))
        assert e.value.code == bfs.BFS_ERR_INVALID_ARG, text
    # a subtree shared by two parents is a valid tree file (every walk ends);
    # it is walked node by node instead of bit-parallel
    ok = tmp_path / "dag.tree"
    ok.write_text("bfs-tree 1 4\n8 5 1 2 -1\n10 7 3 3 -1\n12 9 3 3 -1\n-1 0 -1 -1 1\n")
    bfs.bfs_load_tree(str(ok))
    bfs.bfs_load_tree(None)


def test_serve_and_batch_argument_checks(lib):
    """Server configurations out of range and null handles are rejected before
    any CUDA call (these run on a machine without a GPU)."""
    good = dict(mem_budget_bytes=0, max_inflight=16, num_streams=8, queue_capacity=1024, merge_batch=0,
                merge_policy=0, reserved=0)
    out = ctypes.c_void_p()
    for field, value in (("max_inflight", 0), ("max_inflight", 1025), ("num_streams", 0), ("num_streams", 1025),
                         ("queue_capacity", 0), ("merge_batch", -1), ("merge_batch", 65),
                         ("mem_budget_bytes", -1), ("merge_policy", 2), ("reserved", 1)):
        cfg = bfs._ServeConfig(**dict(good, **{field: value}))
        assert lib.bfs_serve_create(ctypes.byref(cfg), ctypes.byref(out)) == bfs.BFS_ERR_INVALID_ARG, field
    cfg = bfs._ServeConfig(**good)
    assert lib.bfs_serve_create(None, ctypes.byref(out)) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_serve_create(ctypes.byref(cfg), None) == bfs.BFS_ERR_INVALID_ARG
    i32, u64, i64 = ctypes.c_int32(), ctypes.c_uint64(), ctypes.c_int64()
    st = ctypes.c_int()
    stats = bfs._ServeStats()
    assert lib.bfs_serve_add_graph(None, None, ctypes.byref(i32)) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_serve_graph_shape(None, 0, ctypes.byref(i32), ctypes.byref(i32)) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_serve_submit(None, 0, 0, None, ctypes.byref(u64)) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_serve_poll(None, 1, ctypes.byref(st)) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_serve_wait(None, 1, 0) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_serve_stats(None, ctypes.byref(stats)) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_serve_reset_stats(None) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_serve_cancel_queued(None, ctypes.byref(i64)) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_serve_destroy(None) == bfs.BFS_OK
    bc = bfs._BatchConfig(push_mode=2, alpha=8, grid_blocks=0)
    assert lib.bfs_batch_set_config(None, ctypes.byref(bc)) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_run_batch(None, None, 1, None, None, None) == bfs.BFS_ERR_INVALID_ARG


def test_no_cpu_fallback_without_the_library(tmp_path, monkeypatch):
    """Without libbfs.so the binding raises on first use: nothing on the path
    falls back to a CPU implementation."""
    import numpy as np
    monkeypatch.setattr(bfs, "LIB_PATH", str(tmp_path / "absent" / "libbfs.so"))
    monkeypatch.setattr(bfs, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        bfs.lib()
    off = np.array([0, 1, 2], np.int32)
    idx = np.array([1, 0], np.int32)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        bfs.bfs_graph_create(off, idx)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        bfs.bfs_run_ex(1, 0, np.zeros(2, np.int32), depth_on_host=True)


def test_stall_hook_modes_checked_on_the_host(lib):
    assert lib.bfs_debug_stall_next_launch(4) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_debug_stall_next_launch(-1) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_debug_stall_next_launch(0) == bfs.BFS_OK


def test_warp_width_calls_checked_on_the_host(lib):
    p = ctypes.c_int32(0)
    assert lib.bfs_set_warp_width(None, 0) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_get_warp_width(None, ctypes.byref(p)) == bfs.BFS_ERR_INVALID_ARG
    assert lib.bfs_tune_warp_width(None, None, 1, None, None) == bfs.BFS_ERR_INVALID_ARG
    assert len(bfs.WARP_WIDTHS) == 7
