#!/usr/bin/env python3
"""Benchmark of the per-level switched BFS on GB300.

Workload: R-MAT scale 22, edge factor 16 (a/b/c/d = .57/.19/.19/.05),
symmetrised and deduplicated (4,194,304 vertices, ~128M directed edges), 64
seeded roots in the giant component. One step = one switched BFS from each
root (the whole hot path: init, per-level tree decision on the device, level
kernels). Reported value: GTEPS, harmonic mean over the roots, GTEPS_i =
(edges_reached_i / 2) / t_i / 1e9 with t_i the device time of run i (CUDA
events on the launching stream, depth init included, graph upload excluded).

Also reported on the same line: every fixed variant on the same roots, the
end-to-end number through the C ABI with host output buffers, the roofline of
the dominant kernel, the CPU oracle baseline and the SM clocks seen while
timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BFS GTEPS (harmonic mean, 16 roots) vs best fixed kernel; serve p50/p99 ms"
UNIT = "GTEPS"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--roots", type=int, default=64)
    p.add_argument("--scale", type=int, default=22)
    p.add_argument("--edge-factor", type=int, default=16)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fixed", action="store_true")
    p.add_argument("--no-roofline", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-grid", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--serve-only", action="store_true",
                   help="only the serving section, one JSON object (the main run starts it as a child process)")
    p.add_argument("--serve-rates", default="1000,4000,16000,50000", help="offered loads (queries/s)")
    p.add_argument("--serve-seconds", type=float, default=2.0)
    p.add_argument("--mode", default="default", choices=["default", "persistent", "graph", "host_loop"],
                   help="level-loop driver of the timed switched runs (host_loop: every kernel visible to profilers)")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def make_workload(args, rank):
    import graphgen as gg
    g = gg.rmat(args.scale, args.edge_factor, seed=gg.SEED_GRAPH + 1)
    roots = gg.sample_roots(g, args.roots, seed=gg.SEED_ROOTS + 1 + 100 * rank, giant=True)
    return g, roots


def workload_name(args, g):
    return (f"R-MAT scale {args.scale} edge factor {args.edge_factor} (a/b/c/d .57/.19/.19/.05, symmetrised, "
            f"deduplicated): {g.n:,} vertices, {g.m:,} directed edges; {args.roots} roots in the giant component")


def aggregate_ranks(total_s, edges_local, device):
    """Whole-job GTEPS of independent replicas (one per rank, no data-path
    collective): the edges all ranks traversed (edges_reached / 2, summed) over
    the slowest rank's timed seconds. Returns (GTEPS, max seconds)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_s)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(edges_local)], dtype=torch.float64, device=device)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(e.item()) / float(t.item()) / 1e9, float(t.item())


def per_root_summary(times_s, edges, steps):
    """Per-root view of the timed steps (times step-major, one per root per
    step): the harmonic-mean GTEPS of each root's median and of its mean time,
    and the spread of the per-root GTEPS over the roots."""
    t = np.asarray(times_s, dtype=np.float64).reshape(steps, len(edges))
    med, mean = np.median(t, axis=0), t.mean(axis=0)
    g = np.asarray(edges, dtype=np.float64) / 2.0 / med / 1e9
    return {"harmonic_gteps_of_medians": harmonic_gteps(med, edges),
            "harmonic_gteps_of_means": harmonic_gteps(mean, edges),
            "min_gteps": float(g.min()), "max_gteps": float(g.max()), "runs_per_root": int(steps)}


def harmonic_gteps(times_s, edges):
    """k / sum(1 / GTEPS_i), GTEPS_i = (edges_i / 2) / t_i / 1e9."""
    inv = [t / (e / 2.0 / 1e9) for t, e in zip(times_s, edges)]
    return len(inv) / sum(inv)


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    """The CPU oracle, as it stands, timed on the host: each step is one root."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    g, roots = make_workload(args, 0)
    times, edges = [], []
    for step in range(args.warmup + args.steps):
        r = int(roots[step % len(roots)])
        t0 = time.perf_counter()
        res = oracle.bfs(g.off, g.idx, r)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            edges.append(res.edges_reached)
    value = harmonic_gteps(times, edges)
    sample = f"{args.steps} single-root traversals (one per step) of the {args.roots}-root workload"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_name(args, g), "roots_per_step": 1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

HINT_SCAN = 64  # in-list entries the library examines when it chooses a vertex's pull hint


def pull_hints(g):
    """The pull variant's first test per vertex, as the library defines it:
    among the first HINT_SCAN entries of the vertex's in-list (the CSR itself
    for a symmetric graph), the in-neighbour of largest out-degree, the first
    such on ties; -1 without in-edges."""
    off = g.off.astype(np.int64)
    deg = np.diff(off)
    n = g.n
    cap = np.minimum(deg, HINT_SCAN)
    rows = np.repeat(np.arange(n, dtype=np.int64), cap)
    starts = np.repeat(off[:-1], cap)
    k = np.arange(int(cap.sum()), dtype=np.int64) - np.repeat(np.cumsum(cap) - cap, cap)  # position in the row
    nbr = g.idx[starts + k].astype(np.int64)
    # largest out-degree first, then the earliest position
    score = (deg[nbr] << 8) | (255 - k)
    hint = np.full(n, -1, dtype=np.int64)
    if rows.size:
        seg = np.nonzero(cap > 0)[0]
        best = np.maximum.reduceat(score, (np.cumsum(cap) - cap)[seg])
        kbest = 255 - (best & 255)
        hint[seg] = g.idx[off[:-1][seg] + kbest]
    return hint


def algorithmic_bytes(g, depth, feats, L, variant, hint=None):
    """Bytes level L must move for the variant that expanded it (HBM traffic the
    method needs; the visited bitmaps, n/8 bytes, stay in L2 and are not counted)."""
    n = g.n
    F_FRONTIER, F_DISC, F_FE = 8, 10, 12
    f = int(feats[L][F_FRONTIER])
    nxt = int(feats[L + 1][F_FRONTIER]) if L + 1 < len(feats) else 0
    if variant != 4:  # push: queue read, row extents, adjacency, depth + queue writes, degree of new vertices
        e = int(feats[L][F_FE])
        return 4 * f + 8 * f + 4 * e + 4 * nxt + 4 * nxt + 8 * nxt
    # pull: bitmap words read/written, the row extent and the hint of every
    # unvisited vertex that has in-edges (the others start visited), the
    # adjacency entries scanned up to the first frontier neighbour by the
    # vertices whose hint is not in the frontier, writes
    if hint is None:
        hint = pull_hints(g)
    words = (n + 31) // 32
    deg = np.diff(g.off.astype(np.int64))
    unvis = ((depth < 0) | (depth > L)) & (deg > 0)
    hint_hit = unvis & (hint >= 0) & (depth[np.maximum(hint, 0)] == L)
    hit = depth[g.idx] == L
    pos = np.arange(g.m, dtype=np.int64)
    cand = np.where(hit, pos, np.int64(g.m + 1))
    rows = np.nonzero(unvis & ~hint_hit)[0]
    first = np.minimum.reduceat(cand, g.off[:-1].astype(np.int64)[rows]) if rows.size else np.zeros(0, np.int64)
    # reduceat over the selected starts spans to the next selected start; clip to the row end
    ends = g.off[1:].astype(np.int64)[rows]
    starts = g.off[:-1].astype(np.int64)[rows]
    scanned = np.where(first < ends, first - starts + 1, ends - starts)
    return 8 * words + 8 * int(unvis.sum()) + 4 * int(scanned.sum()) + 8 * nxt


def traffic_for(kernel_key):
    """Per-launch DRAM bytes from a committed ncu summary, if it still matches the kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        import hashlib
        d = json.load(open(path))
        src = os.path.join(ROOT, "paper_1708_01159_gb300", "csrc", "bfs_kernels.cu")
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if d.get("kernels_sha") != h:
            return None
        return d.get("per_launch_bytes", {}).get(kernel_key)
    except Exception:
        return None


def progress(msg):
    """Synchronise the device (so an asynchronous error is charged to the section
    that caused it) and note the section on stderr."""
    import torch
    torch.cuda.synchronize()
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def bench_count_modes(bfs, torch, G, g, roots, edges, stream):
    """Vertex push (push_thread forced) with each frontier-count mode, host-loop
    driver (a host round trip per level, the same for every mode), on the
    benchmark graph and on R-MAT scale 14 (16 roots)."""
    import graphgen as gg
    out = {"note": "push_thread forced, host-loop driver; harmonic-mean GTEPS"}

    def measure(Gh, n, rs, es):
        d = torch.empty(n, dtype=torch.int32, device="cuda")
        res = {}
        for name, cm in bfs.COUNT_MODES.items():
            bfs.bfs_run_ex(Gh.handle, int(rs[0]), d, stream, forced_variant=0, mode=bfs.MODE_HOST_LOOP, count_mode=cm)
            torch.cuda.synchronize()
            ts = []
            for r in rs:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                bfs.bfs_run_ex(Gh.handle, int(r), d, stream, forced_variant=0, mode=bfs.MODE_HOST_LOOP, count_mode=cm)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            res[name] = harmonic_gteps(ts, es)
        return res

    out["rmat22"] = measure(G, g.n, roots, edges)
    g14 = gg.rmat_s14_ef16()
    r14 = gg.sample_roots(g14, 16, seed=gg.SEED_ROOTS)
    with bfs.Graph(g14.off, g14.idx) as G14:
        d = torch.empty(g14.n, dtype=torch.int32, device="cuda")
        e14 = [bfs.bfs_run_ex(G14.handle, int(r), d, stream, stats=True)["edges_reached"] for r in r14]
        out["rmat14"] = measure(G14, g14.n, r14, e14)
    return out


def bench_c1(bfs, torch, stream, reps=5):
    """R-MAT scale 14, edge factor 16, 16 seeded roots of nonzero degree, every
    level run by one fixed top-down push kernel: the one-thread-per-vertex push
    (the paper's vertex push) in the persistent driver (one launch per
    traversal) and the graph driver, and each of the other push kernels in the
    persistent driver, beside the switched traversal. CUDA events per
    traversal, harmonic-mean GTEPS over the roots (median of `reps` runs per
    root). The graph is about 2 MB, L2-resident: latency bound."""
    import graphgen as gg
    g = gg.rmat_s14_ef16()
    roots = gg.sample_roots(g, 16, seed=gg.SEED_ROOTS)
    out = {"workload": f"R-MAT scale 14 edge factor 16 ({g.n:,} vertices, {g.m:,} directed edges), 16 roots, "
                       "push_thread forced (and each push kernel in the persistent driver)"}
    with bfs.Graph(g.off, g.idx) as G:
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        sts = [bfs.bfs_run_ex(G.handle, int(r), d, stream, forced_variant=0, stats=True, log_capacity=256)
               for r in roots]
        edges = [st["edges_reached"] for st in sts]

        def measure(variant, mode):
            bfs.bfs_run_ex(G.handle, int(roots[0]), d, stream, forced_variant=variant, mode=mode)
            torch.cuda.synchronize()
            med = []
            for r in roots:
                ts = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    bfs.bfs_run_ex(G.handle, int(r), d, stream, forced_variant=variant, mode=mode)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1) / 1e3)
                med.append(float(np.median(ts)))
            return {"gteps": harmonic_gteps(med, edges), "us_per_traversal": 1e6 * float(np.mean(med))}

        for name, mode in (("persistent", bfs.MODE_PERSISTENT), ("graph", bfs.MODE_GRAPH)):
            out[name] = measure(0, mode)
        out["push_kernels_persistent"] = {bfs.VARIANTS[v]: measure(v, bfs.MODE_PERSISTENT) for v in range(4)}
        out["switched_persistent"] = measure(bfs.VARIANT_TREE, bfs.MODE_PERSISTENT)
        out["levels"] = [st["levels"] for st in sts]
        out["device_us"] = float(np.mean([st.get("device_ns", 0) for st in sts]) / 1e3)
    return out


def bench_batch(bfs, torch, stream):
    """Multi-source BFS: ER 2^22, average degree 8, 64 roots in one launch (tuned), against
    the same 64 roots as single-source switched traversals."""
    import graphgen as gg
    g = gg.er_2p22_d8()
    roots = gg.sample_roots(g, 64, seed=gg.SEED_ROOTS + 3, giant=True)
    out = {"workload": f"Erdos-Renyi 2^22 vertices, average degree 8 ({g.m:,} directed edges), 64 roots per launch"}
    with bfs.Graph(g.off, g.idx) as G:
        depth = torch.empty(64 * g.n, dtype=torch.int32, device="cuda")
        cfg = bfs.bfs_batch_tune(G.handle, roots, depth, stream)
        edges = bfs.bfs_run_batch(G.handle, roots, depth, stream, edges=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            bfs.bfs_run_batch(G.handle, roots, depth, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        single = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for r in roots[:4]:
            bfs.bfs_run(G.handle, int(r), single, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for r in roots:
            bfs.bfs_run(G.handle, int(r), single, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ts = e0.elapsed_time(e1) / 1e3
        out.update({"gteps": float(edges.sum()) / 2 / t / 1e9, "ms_per_launch": t * 1e3,
                    "single_source_gteps": float(edges.sum()) / 2 / ts / 1e9, "speedup_vs_single": ts / t,
                    "tuned": {"push_mode": ["thread+block", "warp"][cfg["push_mode"]], "alpha": cfg["alpha"],
                              "grid_blocks": cfg["grid_blocks"]},
                    "note": "depth output k x n int32 written inside the timed region (1.07 GB per launch)"})
    return out


def bench_batch_graphs(bfs, torch):
    """Multi-source BFS over a batch of 32 uneven R-MAT graphs (scale 12-20, edge
    factor 8-32, seeded): each graph's 64 roots in one launch, the 32 launches
    spread over 8 streams (graphs of scale 16 and up tuned for 8 waves at once,
    the others on the default grid sized to the graph); against the same 2048
    roots as single-source runs."""
    import graphgen as gg
    specs = gg.rmat_batch_specs()
    streams = [torch.cuda.Stream() for _ in range(8)]
    main = torch.cuda.current_stream()
    Gs, roots, outs, tuned = [], [], [], 0
    edges_total = 0
    try:
        for sc, ef, gseed, rseed in specs:
            g = gg.rmat(sc, ef, seed=gseed)
            G = bfs.Graph(g.off, g.idx)
            Gs.append(G)
            r = gg.sample_roots(g, 64, seed=rseed, giant=True)
            roots.append(r)
            out = torch.empty(64 * g.n, dtype=torch.int32, device="cuda")
            outs.append(out)
            if sc >= 16:  # smaller graphs keep the default configuration
                # tuned for waves that run 8 at a time (one per stream)
                bfs.bfs_batch_tune(G.handle, r, out, concurrency=len(streams))
                tuned += 1
            edges_total += int(bfs.bfs_run_batch(G.handle, r, out, edges=True).sum())
        single = [torch.empty(G.n, dtype=torch.int32, device="cuda") for G in Gs]

        def run(batch):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(main)
            for st in streams:
                st.wait_event(e0)
            for i, G in enumerate(Gs):
                st = streams[i % len(streams)]
                if batch:
                    bfs.bfs_run_batch(G.handle, roots[i], outs[i], st)
                else:
                    for r in roots[i]:
                        bfs.bfs_run(G.handle, int(r), single[i], st)
            for st in streams:
                ev = torch.cuda.Event()
                ev.record(st)
                main.wait_event(ev)
            e1.record(main)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / 1e3

        run(True)
        t = min(run(True) for _ in range(3))
        run(False)
        ts = min(run(False) for _ in range(2))
    finally:
        for G in Gs:
            G.close()
    return {"workload": "32 R-MAT graphs (a/b/c/d .57/.19/.19/.05), scale 12-20 and edge factor 8-32 drawn with "
                        "seed 6000, 64 giant-component roots each; one multi-source launch per graph, 8 streams",
            "scales": [sp[0] for sp in specs], "edge_factors": [sp[1] for sp in specs],
            "gteps": edges_total / 2 / t / 1e9, "ms_per_batch": t * 1e3,
            "single_source_gteps": edges_total / 2 / ts / 1e9, "speedup_vs_single": ts / t,
            "tuned_graphs": tuned}


def bench_grid(bfs, torch, stream):
    """High diameter: 4096 x 4096 permuted grid, 10% edges dropped, 16 roots in the
    giant component; the switched traversal under both drivers, and every fixed
    variant (persistent driver): the tree's classes on all 16 roots, the
    whole-edge-list kernels on the first 4."""
    import graphgen as gg
    g = gg.grid_4096_permuted()
    roots = [int(r) for r in gg.sample_roots(g, 16, seed=gg.SEED_ROOTS + 2, giant=True)]
    out = {"workload": f"4096x4096 grid, 10% of edges dropped, ids permuted ({g.m:,} directed edges), "
                       f"{len(roots)} roots in the giant component"}
    with bfs.Graph(g.off, g.idx) as G:
        depth = torch.empty(g.n, dtype=torch.int32, device="cuda")
        stats = [bfs.bfs_run_ex(G.handle, r, depth, stream, stats=True) for r in roots]
        edges = [st["edges_reached"] for st in stats]
        levels = [st["levels"] for st in stats]
        out["levels"] = {"min": min(levels), "max": max(levels), "mean": float(np.mean(levels))}

        def timed(rs, **kw):
            bfs.bfs_run_ex(G.handle, rs[0], depth, stream, **kw)
            torch.cuda.synchronize()
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(rs) + 1)]
            evs[0].record(stream)
            for i, r in enumerate(rs):
                bfs.bfs_run_ex(G.handle, r, depth, stream, **kw)
                evs[i + 1].record(stream)
            torch.cuda.synchronize()
            return [evs[i].elapsed_time(evs[i + 1]) / 1e3 for i in range(len(rs))]

        for name, mode in (("persistent", bfs.MODE_PERSISTENT), ("graph", bfs.MODE_GRAPH)):
            ts = timed(roots, mode=mode)
            out[name] = {"gteps": harmonic_gteps(ts, edges), "ms_per_traversal": 1e3 * float(np.mean(ts)),
                         "us_per_level": 1e6 * sum(ts) / sum(levels)}
        # the tree's five classes on every root; the two whole-edge-list kernels
        # (a scan of all m edges per level, over 100x slower here) on 4
        fixed, fixed_roots = {}, {}
        for v, vname in enumerate(bfs.FORCED_VARIANTS):
            k = len(roots) if v < bfs.NUM_VARIANTS else 4
            fixed[vname] = harmonic_gteps(timed(roots[:k], mode=bfs.MODE_PERSISTENT, forced_variant=v), edges[:k])
            fixed_roots[vname] = k
        switched = harmonic_gteps(timed(roots, mode=bfs.MODE_PERSISTENT), edges)
        best = max(fixed, key=fixed.get)
        out["fixed_variants_gteps"] = fixed
        out["fixed_variants_roots"] = fixed_roots
        out["best_fixed"] = {"variant": best, "gteps": fixed[best], "roots": fixed_roots[best],
                             "switched_gteps": switched, "switched_over_best_fixed": switched / fixed[best],
                             "note": "switched re-timed on the same roots right after the fixed variants"}
        out["warp_width_tuning"] = warp_width_tuning(bfs, G, roots[:4])
    return out


def warp_width_tuning(bfs, G, roots):
    """The virtual-warp width autotuner on these roots (device time of the
    switched traversals under each policy); the graph goes back to the
    default policy (the mean-degree rule), which every other number uses."""
    res = bfs.bfs_tune_warp_width(G.handle, roots)
    bfs.bfs_set_warp_width(G.handle, 0)
    return {"roots": len(roots), "fastest": res["name"], "ms": res["ms"],
            "rule_over_fastest": res["ms"]["rule"] / res["ms"][res["name"]]}


def bench_serve(bfs, torch, args):
    """Serving: 8 resident graphs, Poisson arrivals of single-root queries (graph
    uniform, root uniform over vertices of nonzero degree), continuous batching."""
    import graphgen as gg
    specs = gg.serve_graph_specs()
    Gs, cand = [], []
    for name, mk in specs:
        g = mk()
        Gs.append(bfs.Graph(g.off, g.idx))
        cand.append(np.nonzero(np.diff(g.off) > 0)[0].astype(np.int32))
        del g
        progress(f"serve graph {name} resident")
    rng = np.random.default_rng(5000)
    out = {"graphs": [n for n, _ in specs], "loads": [],
           "warmup": "one server for every load: graphs registered (probed) once, then 1000 queries submitted at "
                     "once before the measured loads (fills the workspace and depth-buffer pools; not reported); "
                     "each load starts a new statistics window and ends by cancelling what is still queued after "
                     "the drain"}
    budget = 40 << 30
    out["mem_budget_bytes"] = budget
    out["cuda_device_max_connections"] = os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8 (default)")
    s = bfs.bfs_serve_create(mem_budget_bytes=budget, max_inflight=256, num_streams=256, queue_capacity=1 << 17,
                             merge_batch=64)
    try:
        ids = [bfs.bfs_serve_add_graph(s, G.handle) for G in Gs]
        out["shapes"] = {name: bfs.bfs_serve_graph_shape(s, i) for (name, _), i in zip(specs, ids)}

        def drain(tickets, seconds):
            deadline = time.perf_counter() + seconds
            for t in tickets:
                left_us = int((deadline - time.perf_counter()) * 1e6)
                if left_us <= 0 or bfs.bfs_serve_wait(s, t, left_us) == bfs.BFS_ERR_TIMEOUT:
                    return False
            return True

        gsel = rng.integers(0, len(Gs), 1000)
        warm = [bfs.bfs_serve_submit(s, ids[k], int(cand[k][rng.integers(0, len(cand[k]))])) for k in gsel]
        drain(warm, 30.0)
        progress("serve warm-up done")
        for rate in [float(x) for x in args.serve_rates.split(",")]:
            nq = int(rate * args.serve_seconds)
            arrivals = np.cumsum(rng.exponential(1.0 / rate, nq))
            gsel = rng.integers(0, len(Gs), nq)
            roots = [int(cand[k][rng.integers(0, len(cand[k]))]) for k in gsel]
            bfs.bfs_serve_reset_stats(s)
            tickets = []
            t0 = time.perf_counter()
            for q in range(nq):
                while time.perf_counter() - t0 < arrivals[q]:
                    pass
                try:
                    tickets.append(bfs.bfs_serve_submit(s, ids[gsel[q]], roots[q]))
                except bfs.BFSError:
                    pass  # counted by the server as rejected
            drain(tickets, 10.0)  # what is still queued after 10 s is not finished
            st = bfs.bfs_serve_stats(s)
            out["loads"].append({"offered_qps": rate, "achieved_qps": st["qps"], "p50_ms": st["p50_ms"],
                                 "p99_ms": st["p99_ms"], "wait_p50_ms": st["wait_p50_ms"],
                                 "wait_p99_ms": st["wait_p99_ms"], "gteps": st["gteps"], "submitted": st["submitted"],
                                 "completed": st["completed"], "not_finished": st["submitted"] - st["completed"],
                                 "rejected": st["rejected"], "failed": st["failed"],
                                 "merged_waves": st["merged_waves"], "peak_bytes_inflight": st["peak_bytes_inflight"]})
            bfs.bfs_serve_cancel_queued(s)
            drain(tickets, 60.0)  # the admitted ones finish before the next load
    finally:
        bfs.bfs_serve_destroy(s)
        for G in Gs:
            G.close()
    return out


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1708_01159_gb300 as bfs

    g, roots = make_workload(args, rank)
    R = len(roots)
    G = bfs.Graph(g.off, g.idx)
    dev = torch.device("cuda", torch.cuda.current_device())
    depth = [torch.empty(g.n, dtype=torch.int32, device=dev) for _ in range(2)]
    stream = torch.cuda.current_stream()

    # per-root edges and levels (one stats run each, untimed)
    edges, launches = [], 0
    for r in roots:
        st = bfs.bfs_run_ex(G.handle, int(r), depth[0], stats=True, log_capacity=4096)
        edges.append(st["edges_reached"])
        if args.mode in ("default", "persistent"):
            launches += 1  # one cooperative persistent kernel per traversal
        else:  # init, (graph: loop start), per level decide + the variant's kernels, final decide
            kern = {0: 1, 1: 1, 2: 1, 3: 4, 4: 1}
            launches += 2 + (args.mode == "graph") + sum(1 + kern[int(v)] for v in st["variant"])
    edges = np.array(edges, dtype=np.int64)

    def step(forced=-1, mode=bfs.MODE_DEFAULT):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(R + 1)]
        # hold the stream while the host enqueues the whole step, so host-side
        # launch overhead never shows up inside a timed interval
        torch.cuda._sleep(20_000_000)
        evs[0].record(stream)
        for i, r in enumerate(roots):
            if forced < 0 and mode == bfs.MODE_DEFAULT:
                bfs.bfs_run(G.handle, int(r), depth[i & 1], stream)
            else:
                bfs.bfs_run_ex(G.handle, int(r), depth[i & 1], stream, forced_variant=forced, mode=mode)
            evs[i + 1].record(stream)
        return evs

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    main_mode = bfs.MODES[args.mode]
    for _ in range(args.warmup):
        step(-1, main_mode)
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    all_evs = [step(-1, main_mode) for _ in range(args.steps)]
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    times = []
    for evs in all_evs:
        times += [evs[i].elapsed_time(evs[i + 1]) * 1e-3 for i in range(R)]
    total_s = sum(times)
    value_local = harmonic_gteps(times, np.tile(edges, args.steps))
    total_edges_local = float(edges.sum()) * args.steps / 2.0
    if world > 1:
        value, total_s = aggregate_ranks(total_s, total_edges_local, dev)
    else:
        value = value_local

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_name(args, g), "roots": R,
                   "switching": "decision tree evaluated on the device every level",
                   "mode": {"default": "persistent cooperative kernel per traversal (grid barrier between levels)",
                            "persistent": "persistent cooperative kernel per traversal (grid barrier between levels)",
                            "graph": "CUDA graph with WHILE and SWITCH conditional nodes",
                            "host_loop": "host-driven level loop (one launch per kernel)"}[args.mode],
                   "l2": "inputs larger than L2 (CSR %.0f MB vs 129 MB L2)" % ((g.off.nbytes + g.idx.nbytes) / 1e6),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
        "per_root": per_root_summary(times, edges, args.steps),
    }

    # every fixed variant on the same roots (the "best fixed kernel" comparison)
    if not args.no_fixed:
        fixed = {}
        for v, name in enumerate(bfs.FORCED_VARIANTS):
            step(v)
            torch.cuda.synchronize()
            evs = step(v)
            torch.cuda.synchronize()
            ts = [evs[i].elapsed_time(evs[i + 1]) * 1e-3 for i in range(R)]
            fixed[name] = harmonic_gteps(ts, edges)
        best = max(fixed, key=fixed.get)
        line["fixed_variants_gteps"] = fixed
        line["best_fixed"] = {"variant": best, "gteps": fixed[best], "switched_over_best_fixed": value_local / fixed[best]}
        # the same switched traversal driven by the CUDA graph (WHILE + SWITCH nodes)
        step(-1, bfs.MODE_GRAPH)
        torch.cuda.synchronize()
        evs = step(-1, bfs.MODE_GRAPH)
        torch.cuda.synchronize()
        ts = [evs[i].elapsed_time(evs[i + 1]) * 1e-3 for i in range(R)]
        line["modes_gteps"] = {"persistent (timed above)": value_local, "graph": harmonic_gteps(ts, edges)}

    # end to end through the C ABI with host output buffers (pinned), copies
    # timed: the roots alternate between two streams, each with its own pinned
    # host buffer (reused in stream order: a root's copy lands before the next
    # root of that stream overwrites it), and each call returns once its copy
    # is enqueued, so that one root's copy overlaps the next root's traversal
    e2e_streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pinned = [torch.empty(g.n, dtype=torch.int32).pin_memory() for _ in e2e_streams]
    for rep in range(2):  # warm-up: each stream's workspace, host stage and buffer pages
        for j in range(min(2, R)):
            bfs.bfs_run_ex(G.handle, int(roots[j]), pinned[j], e2e_streams[j], depth_on_host=True, host_async=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, r in enumerate(roots):
        bfs.bfs_run_ex(G.handle, int(r), pinned[i & 1], e2e_streams[i & 1], depth_on_host=True, host_async=True)
    for st in e2e_streams:
        st.synchronize()
    e2e_s = time.perf_counter() - t0
    line["e2e"] = {"value": float(edges.sum()) / 2.0 / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": 4 * R,
                   "d2h_bytes_per_step": 4 * g.n * R,
                   "note": "one step: every root's depths copied to pinned host memory inside the timed region; "
                           "roots alternate between two streams (a pinned buffer each), each copy overlapping the "
                           "next traversal, and each traversal queued before the previous one ends (so this can "
                           "exceed `value`, whose per-root intervals include the gap between launches on one stream)"}
    del pinned

    # roofline of the dominant kernel: per-level launches timed with CUDA events
    # on the launching stream (per-level harness, same state for every variant)
    if not args.no_roofline:
        hbm, src = peaks()
        # The timed region runs one kernel per traversal, k_bfs_persistent, so
        # that launch is the dominant kernel. Its
        # algorithmic bytes are the schedule-exact bytes of the traversal (every
        # level's bytes for the variant the tree ran there), replayed on the host
        # for a sample of roots; its duration is the CUDA-event time of the same
        # roots in the timed steps above (mean over steps).
        per_root_s = np.array(times, dtype=np.float64).reshape(args.steps, R).mean(axis=0)
        sample = list(range(min(4, R)))
        hint = pull_hints(g)
        b_sched, b_td, t_sum = [], [], 0.0
        for i in sample:
            r = int(roots[i])
            st = bfs.bfs_run_ex(G.handle, r, depth[0], stream, stats=True, log_capacity=4096)
            dep = depth[0].cpu().numpy()
            nl = st["levels"]
            feats = np.zeros((nl, 13), dtype=np.int64)
            feats[:, 8] = st["frontier"][:nl]
            feats[:, 12] = st["frontier_edges"][:nl]
            # depth init (4 n) plus every level's bytes for the variant that ran it
            b_sched.append(4 * g.n + sum(algorithmic_bytes(g, dep, feats, L, int(st["variant"][L]), hint)
                                         for L in range(nl)))
            n_r = st["vertices_reached"]
            b_td.append(4 * st["edges_reached"] + 8 * n_r + 4 * g.n + 4 * n_r + 8 * n_r)
            t_sum += float(per_root_s[i])
        achieved = sum(b_sched) / t_sum / 1e9
        r0 = int(roots[0])
        line["roofline"] = {
            "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic_for(f"persistent_root_{r0}"), "peak_source": src,
            "kernel": "k_bfs_persistent (one launch = one switched traversal; the timed region's only level kernel)",
            "algorithmic_bytes": int(b_sched[0]), "launch_ms": 1e3 * float(per_root_s[0]),
            "sample": f"roots {[int(roots[i]) for i in sample]}; algorithmic_bytes, launch_ms and traffic "
                      f"are those of root {r0}",
            "top_down_bytes": int(b_td[0]), "frac_top_down": sum(b_td) / t_sum / 1e9 / hbm}
        # the dominant level, kernel by kernel: the timing harness runs every
        # variant from the same snapshot of every level (CUDA events per launch)
        feats, ms, tv = bfs.bfs_profile_levels(G.handle, r0, reps=5, stream=stream)
        chosen = np.array([ms[L, tv[L]] for L in range(len(tv))])
        L = int(np.argmax(chosen))
        v = int(tv[L])
        bfs.bfs_run(G.handle, r0, depth[0], stream)
        torch.cuda.synchronize()
        dep = depth[0].cpu().numpy()
        nbytes = algorithmic_bytes(g, dep, feats, L, v, hint)
        t = float(chosen[L]) * 1e-3
        line["roofline"]["dominant_level"] = {
            "kernel": f"{bfs.VARIANTS[v]} at level {L} of root {r0}", "algorithmic_bytes": int(nbytes),
            "launch_ms": float(chosen[L]), "achieved": nbytes / t / 1e9, "frac": nbytes / t / 1e9 / hbm,
            "traffic": traffic_for(bfs.VARIANTS[v]), "share_of_traversal": float(chosen[L] / chosen.sum()),
            "per_level_ms_chosen": [round(float(x), 4) for x in chosen],
            "per_level_optimal_ms": float(ms.min(axis=1).sum()), "per_level_tree_ms": float(chosen.sum())}
        # the same traversal inside the real drivers: device timestamps per level
        for name, mode in (("persistent", bfs.MODE_PERSISTENT), ("graph", bfs.MODE_GRAPH)):
            st = bfs.bfs_run_ex(G.handle, r0, depth[0], stream, stats=True, log_capacity=64, mode=mode)
            if "level_ns" in st:
                line["roofline"]["dominant_level"][f"per_level_ms_in_{name}"] = \
                    [round(float(x) / 1e6, 4) for x in st["level_ns"]]
        # tree schedule against the per-level optimal schedule over 16 roots
        tree_ms = opt_ms = 0.0
        fixed_ms = np.zeros(bfs.NUM_VARIANTS)
        k16 = min(16, R)
        for r in roots[:k16]:
            _, ms_r, tv_r = bfs.bfs_profile_levels(G.handle, int(r), reps=3, stream=stream)
            tree_ms += float(sum(ms_r[L, tv_r[L]] for L in range(len(tv_r))))
            opt_ms += float(ms_r.min(axis=1).sum())
            fixed_ms += ms_r.sum(axis=0)
        line["schedule_vs_optimal"] = {
            "roots": k16, "tree_level_ms": tree_ms, "optimal_level_ms": opt_ms, "tree_over_optimal": tree_ms / opt_ms,
            "best_fixed_over_optimal": float(fixed_ms.min()) / opt_ms,
            "note": "sums of per-level kernel times from the timing harness (each variant from the same snapshot); "
                    "init and driver overheads excluded"}
        line["warp_width_tuning"] = warp_width_tuning(bfs, G, roots[:16])

    # Section 3.1.4's frontier-count alternatives in the vertex push (host-loop
    # driver, push_thread forced): block-staged appends (the kernels' own),
    # one atomic per warp, one atomic per vertex
    if not args.no_fixed:
        line["count_modes"] = bench_count_modes(bfs, torch, G, g, roots[:8], edges[:8], stream)

    G.close()
    del depth
    progress("switched, fixed, e2e and roofline done")
    line["c1"] = bench_c1(bfs, torch, stream)
    progress("C1 done")
    if not args.no_batch:
        line["batch"] = bench_batch(bfs, torch, stream)
        progress("batch (ER) done")
        line["batch_graphs"] = bench_batch_graphs(bfs, torch)
        progress("batch done")
    if not args.no_grid:
        line["high_diameter"] = bench_grid(bfs, torch, stream)
        progress("high-diameter done")
    if not args.no_serve:
        line["serve"] = serve_in_child(args, local)
        progress("serve done")

    # the oracle on the host, bounded sample (rank 0, one GPU)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        ts, es = [], []
        t_start = time.perf_counter()
        for r in roots:
            t0 = time.perf_counter()
            res = oracle.bfs(g.off, g.idx, int(r))
            ts.append(time.perf_counter() - t0)
            es.append(res.edges_reached)
            if time.perf_counter() - t_start > 10.0 or len(ts) >= 8:
                break
        line["cpu_baseline"] = {"value": harmonic_gteps(ts, es), "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{len(ts)} of the {R} roots, single-threaded FIFO BFS on the same graph"}
        # throughput mode: independent roots at once, one oracle call per host core
        # (the C oracle runs outside the GIL)
        from concurrent.futures import ThreadPoolExecutor
        cores = os.cpu_count() or 1
        sample = [int(r) for r in roots[:min(R, 2 * cores)]]
        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=cores) as ex:
            done = list(ex.map(lambda r: oracle.bfs(g.off, g.idx, r).edges_reached, sample))
        wall = time.perf_counter() - t0
        line["cpu_baseline_throughput"] = {
            "value": float(sum(done)) / 2 / wall / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(sample)} of the {R} roots, {cores} concurrent single-threaded oracle runs; "
                      "aggregate edges/2 over wall time"}

    G.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def serve_in_child(args, local):
    """The serving section in a child process on the same GPU, started with 32
    hardware work queues instead of CUDA's default 8 (the setting is read when
    a process creates its CUDA context): with 8, the query server's short
    queries wait behind long ones (a 4096^2 grid query runs about 90 ms) of
    other streams that share their hardware queue. The other sections keep the
    default, which the graph driver's conditional graphs run faster under."""
    env = dict(os.environ, CUDA_DEVICE_MAX_CONNECTIONS="32", BENCH_SERVE_DEVICE=str(local))
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "LOCAL_WORLD_SIZE", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    cmd = [sys.executable, os.path.abspath(__file__), "--serve-only", "--serve-rates", args.serve_rates,
           "--serve-seconds", str(args.serve_seconds)]
    r = subprocess.run(cmd, env=env, stdout=subprocess.PIPE, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"serving section failed (exit {r.returncode})")
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    return json.loads(lines[-1])


def run_serve_only(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("BENCH_SERVE_DEVICE", "0")))
    import __graft_entry__
    __graft_entry__.build()
    import paper_1708_01159_gb300 as bfs
    print(json.dumps(bench_serve(bfs, torch, args)), flush=True)


def main():
    args = parse_args()
    if args.serve_only:
        run_serve_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
