"""Build libbfs.so in-tree with nvcc for sm_103a.

The built-in decision tree (trees/default.tree, the text format bfs_load_tree
reads) is turned into a C array include first. Translation units compile in
parallel, then link into one shared library with the static CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbfs.so")
TREE = os.path.join(HERE, "trees", "default.tree")
TREE_INC = os.path.join(BUILD, "default_tree.inc")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
SOURCES = ["bfs_kernels.cu", "bfs_api.cu", "bfs_static.cu", "bfs_msbfs.cu", "bfs_serve.cu"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def parse_tree_text(text: str):
    """(feature, threshold, left, right, value) rows of a tree file."""
    rows, count = [], None
    for line in text.splitlines():
        s = line.strip()
        if not s or s.startswith("#"):
            continue
        parts = s.split()
        if count is None:
            if parts[0] != "bfs-tree" or parts[1] != "1":
                raise ValueError(f"bad tree header: {s}")
            count = int(parts[2])
            continue
        rows.append(tuple(int(x) for x in parts[:5]))
    if count is None or len(rows) != count:
        raise ValueError("tree node count mismatch")
    return rows


def write_tree_inc() -> None:
    rows = parse_tree_text(open(TREE).read())
    lines = ["// generated from trees/default.tree by build.py; fields: t, f, l, r, v"]
    for f, t, l, r, v in rows:
        lines.append(f"{{{t}LL, {f}, {l}, {r}, {v}}},")
    text = "\n".join(lines) + "\n"
    if not os.path.exists(TREE_INC) or open(TREE_INC).read() != text:
        with open(TREE_INC, "w") as fh:
            fh.write(text)


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    write_tree_inc()
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers += [os.path.join(INCLUDE, "bfs.h"), TREE_INC]
    cc = nvcc()
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [cc, *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-I", CSRC, "-I", BUILD, "-c", s, "-o", o]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return r

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-lpthread", "-ldl"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
