"""Multi-process host logic of the replicas-only multi-GPU mode, on CPU with
gloo at world size 2: each rank traverses its own roots of the same graph
(weak scaling, no data-path collective), and the whole-job value is the edges
of all ranks over the slowest rank's time."""
import argparse
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, edges, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        assert bench.dist_env() == (rank, world, rank)
        value, t = bench.aggregate_ranks(times[rank], edges[rank], "cpu")
        args = argparse.Namespace(scale=10, edge_factor=8, roots=6)
        g, roots = bench.make_workload(args, rank)
        # the reference arm runs on rank 0 only; the other ranks return at once
        ref_args = argparse.Namespace(steps=1, warmup=0, roots=6, scale=10, edge_factor=8)
        ref_ret = bench.run_reference(ref_args) if rank == 1 else None
        q.put((rank, value, t, [int(r) for r in roots], int(g.m), ref_ret))
    finally:
        dist.destroy_process_group()


def test_replicas_aggregate_and_shard_roots():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [1.5, 2.0]
    edges = [3.0e9, 5.0e9]
    ps = [ctx.Process(target=_worker, args=(r, 2, port, times, edges, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = {}
    for _ in ps:
        rank, value, t, roots, m, ref_ret = q.get(timeout=180)
        out[rank] = (value, t, roots, m, ref_ret)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(2):
        value, t, _, _, _ = out[rank]
        assert t == max(times)
        assert value == pytest.approx(sum(edges) / max(times) / 1e9)
    assert out[0][3] == out[1][3]          # the same graph on every rank
    assert set(out[0][2]) != set(out[1][2])  # each rank its own roots
    assert out[1][4] is None
