"""Host-side arithmetic of bench.py, on CPU: the per-level algorithmic bytes
behind the reported roofline (checked against a plain vertex-by-vertex count),
the harmonic-mean GTEPS, the per-root summary, the traffic lookup's staleness
rule, and the reference arm end to end at a small scale."""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bench
import graphgen as gg
import oracle


def _hint_plain(g, v):
    """The pull hint of v, plainly: among the first 64 entries of its list, the
    neighbour of largest degree, the first such on ties; -1 without edges."""
    best, best_deg = -1, -1
    for e in range(int(g.off[v]), min(int(g.off[v + 1]), int(g.off[v]) + 64)):
        u = int(g.idx[e])
        d = int(g.off[u + 1] - g.off[u])
        if d > best_deg:
            best, best_deg = u, d
    return best


def _pull_bytes_plain(g, depth, L, nxt):
    """Pull at level L, counted vertex by vertex: every bitmap word read and
    written (8 B), the row extent and the hint of each vertex not visited by
    level L that has in-edges (4 + 4 B); unless its hint is at depth L, the
    adjacency entries it scans in order up to and including its first
    in-neighbour at depth L, or all of them (4 B each); and the depth and queue
    writes plus degree read of each new vertex (8 B)."""
    words = (g.n + 31) // 32
    U = S = 0
    for v in range(g.n):
        lo, hi = int(g.off[v]), int(g.off[v + 1])
        if hi == lo or 0 <= depth[v] <= L:
            continue
        U += 1
        h = _hint_plain(g, v)
        if h >= 0 and depth[h] == L:
            continue
        k = 0
        for e in range(lo, hi):
            k += 1
            if depth[g.idx[e]] == L:
                break
        S += k
    return 8 * words + 8 * U + 4 * S + 8 * nxt


def test_pull_hints_match_a_plain_choice():
    for g in (gg.rmat(10, 8, seed=75), gg.rmat(9, 16, seed=76, permute=True), gg.grid(12, 9, 0.3, seed=77)):
        hint = bench.pull_hints(g)
        assert [int(x) for x in hint] == [_hint_plain(g, v) for v in range(g.n)]


@pytest.mark.parametrize("make", [lambda: gg.rmat(10, 8, seed=71), lambda: gg.grid(30, 20, 0.2, seed=72),
                                  lambda: gg.erdos_renyi(3000, 3.0, seed=73)])
def test_algorithmic_bytes_matches_plain_count(make):
    g = make()
    for r in gg.sample_roots(g, 2, seed=74):
        res = oracle.bfs(g.off, g.idx, int(r))
        feats = oracle.level_features(g.off, g.idx, res)
        for L in range(res.num_levels):
            f = int(res.level_count[L])
            e = int(res.level_edges[L])
            nxt = int(res.level_count[L + 1]) if L + 1 < res.num_levels else 0
            for v in range(4):  # every push variant moves the same bytes
                assert bench.algorithmic_bytes(g, res.depth, feats, L, v) == 12 * f + 4 * e + 16 * nxt
            assert bench.algorithmic_bytes(g, res.depth, feats, L, 4) == _pull_bytes_plain(g, res.depth, L, nxt)


def test_harmonic_gteps():
    # GTEPS_i = (e_i / 2) / t_i / 1e9; harmonic mean k / sum(1 / GTEPS_i)
    times = [1.0, 2.0, 4.0]
    edges = [2e9, 2e9, 2e9]  # 1, 0.5, 0.25 GTEPS
    assert bench.harmonic_gteps(times, edges) == pytest.approx(3 / (1 + 2 + 4))
    assert bench.harmonic_gteps([0.5], [4e9]) == pytest.approx(4.0)


def test_traffic_lookup_requires_current_kernel_source(tmp_path, monkeypatch):
    root = tmp_path
    src_dir = root / "paper_1708_01159_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (src_dir / "bfs_kernels.cu").write_text("// kernels v1\n")
    (root / "profiles").mkdir()
    sha = hashlib.sha256(b"// kernels v1\n").hexdigest()[:16]
    (root / "profiles" / "traffic.json").write_text(json.dumps(
        {"kernels_sha": sha, "per_launch_bytes": {"pull": 123}}))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.traffic_for("pull") == 123
    assert bench.traffic_for("absent") is None
    (src_dir / "bfs_kernels.cu").write_text("// kernels v2\n")  # the kernel changed: the capture is stale
    assert bench.traffic_for("pull") is None


def test_per_root_summary():
    # two roots, three steps: root 0 takes 1, 1, 4 s; root 1 takes 2, 2, 2 s
    times = [1.0, 2.0, 1.0, 2.0, 4.0, 2.0]
    edges = [2e9, 4e9]  # 1e9 and 2e9 traversed edges
    s = bench.per_root_summary(times, edges, 3)
    # medians 1 s and 2 s: 1 GTEPS each; means 2 s and 2 s: 0.5 and 1 GTEPS
    assert s["harmonic_gteps_of_medians"] == pytest.approx(1.0)
    assert s["harmonic_gteps_of_means"] == pytest.approx(2 / (1 / 0.5 + 1 / 1.0))
    assert s["min_gteps"] == pytest.approx(1.0) and s["max_gteps"] == pytest.approx(1.0)
    assert s["runs_per_root"] == 3


def test_reference_arm_runs_and_prints_one_line():
    """`bench.py --impl reference` (the oracle timed on the host) at a small
    scale: one JSON line with the contract's keys."""
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--scale", "10", "--edge-factor", "8", "--roots", "4"],
                       capture_output=True, text=True, timeout=300, cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GTEPS"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
