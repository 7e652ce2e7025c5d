"""Small fixed BFS workload for profiler captures.

Builds one R-MAT graph (default scale 22, edge factor 16, seed 1001: the
benchmark's graph), then runs the switched traversal (or one forced variant)
from a few giant-component roots. Small and deterministic, so a profiler can
capture a handful of kernel launches of interest.

  python -m paper_1708_01159_gb300.profile_case [--scale 22] [--roots 2] [--variant -1]

With --batch: the multi-source case instead, Erdos-Renyi 2^22 vertices of
average degree 8 (seed 1003), 64 giant-component roots in one launch, with a
fixed multi-source configuration (the autotuner's usual choice for this
graph: warp push, alpha 32, 912 blocks), run twice: the first launch on the
graph's new buffer set also zeroes that set, the second is the timed one
(capture it with ncu -s 1 -c 1).
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--scale", type=int, default=22)
    p.add_argument("--edge-factor", type=int, default=16)
    p.add_argument("--seed", type=int, default=1001)
    p.add_argument("--roots", type=int, default=2)
    p.add_argument("--variant", type=int, default=-1)
    p.add_argument("--mode", default="host_loop", choices=["default", "persistent", "graph", "host_loop"],
                   help="host_loop launches every level kernel on its own, which profilers can capture")
    p.add_argument("--batch", action="store_true", help="multi-source case (one 64-root launch)")
    p.add_argument("--push-mode", type=int, default=1, help="--batch: 0 thread+block, 1 warp")
    p.add_argument("--alpha", type=int, default=32, help="--batch: pull when frontier edges x alpha > m")
    p.add_argument("--grid-blocks", type=int, default=912, help="--batch: blocks of the launch")
    a = p.parse_args()
    import torch

    import graphgen as gg
    import paper_1708_01159_gb300 as bfs
    bfs.build()
    if a.batch:
        g = gg.er_2p22_d8()
        roots = gg.sample_roots(g, 64, seed=gg.SEED_ROOTS + 3, giant=True)
        with bfs.Graph(g.off, g.idx) as G:
            depth = torch.empty(64 * g.n, dtype=torch.int32, device="cuda")
            bfs.bfs_batch_set_config(G.handle, a.push_mode, a.alpha, a.grid_blocks)
            bfs.bfs_run_batch(G.handle, roots, depth)  # zeroes the new buffer set
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            edges = bfs.bfs_run_batch(G.handle, roots, depth, edges=True)
            e1.record()
            torch.cuda.synchronize()
            print(f"batch of {len(roots)} roots: {e0.elapsed_time(e1):.3f} ms (second launch), "
                  f"edges {int(edges.sum())}")
        return
    g = gg.rmat(a.scale, a.edge_factor, seed=a.seed)
    roots = gg.sample_roots(g, a.roots, seed=gg.SEED_ROOTS + 1, giant=True)
    with bfs.Graph(g.off, g.idx) as G:
        depth = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for r in roots:
            st = bfs.bfs_run_ex(G.handle, int(r), depth, forced_variant=a.variant, stats=True, log_capacity=64,
                                mode=bfs.MODES[a.mode])
            names = [bfs.VARIANTS[v] for v in st["variant"]]
            print(f"root {int(r)}: levels {st['levels']} edges {st['edges_reached']} schedule {names}")


if __name__ == "__main__":
    main()
