"""Planted-mistake check for the oracle's pins.

Each case copies the oracle's C source to a temporary directory, plants one
plausible mistake (a wrong increment, a dropped neighbour, a stack instead of a
queue, a wrong root depth, a dropped degree term, a miscounted level), builds
it, and runs the pin battery against it. Every mutant must be caught. The
committed oracle is never modified. CPU only.
"""
import json
import os
import shutil

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import graphs_closed_form as cf

SRC = os.path.join(os.path.dirname(oracle.__file__), "bfs_oracle.c")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

MUTANTS = {
    "increment": ("depth[v] = depth[u] + 1;", "depth[v] = depth[u] + 2;"),
    "drop_last_neighbour": ("e < off[u + 1]; ++e)", "e < off[u + 1] - 1; ++e)"),
    "stack_not_queue": ("while (head < tail) {\n    int32_t u = queue[head++];",
                        "while (tail > 0) {\n    int32_t u = queue[--tail];"),
    "root_depth": ("depth[root] = 0;", "depth[root] = 1;"),
    "edges_term": ("edges_reached += deg;", "edges_reached += deg - (deg > 0);"),
    "level_count": ("if (level_count) level_count[d] += 1;", "if (level_count) level_count[d] += (d > 1) ? 2 : 1;"),
}


def pin_battery(lib):
    """Runs a subset of the oracle pins against `lib`; returns the names that failed."""
    failed = set()
    rng = np.random.default_rng(1)
    for trial in range(60):
        n = int(rng.integers(2, 11))
        adj = rng.random((n, n)) < 0.35
        g = cf.csr_from_adj(adj)
        for r in range(n):
            if not np.array_equal(oracle.bfs(g.off, g.idx, r, lib=lib).depth, cf.brute_force_depth(adj, r)):
                failed.add("brute_force")
    for name in ("path17", "cycle16", "bintree5", "Q6", "grid7x9"):
        g, fn = cf.ALL[name]()
        for r in range(0, g.n, 3):
            if not np.array_equal(oracle.bfs(g.off, g.idx, r, lib=lib).depth, fn(r)):
                failed.add("closed_form")
    fx = json.load(open(os.path.join(GOLDEN, "directed6.json")))
    s, t = zip(*fx["edges"])
    g = gg.from_edges(fx["n"], s, t, symmetrize=False)
    for c in fx["cases"]:
        res = oracle.bfs(g.off, g.idx, c["root"], lib=lib)
        if res.edges_reached != c["edges_reached"]:
            failed.add("golden_edges")
        if res.level_count.tolist() != c["level_count"]:
            failed.add("golden_levels")
        if res.depth.tolist() != c["depth"]:
            failed.add("golden_depth")
    return failed


def test_battery_passes_on_real_oracle():
    assert pin_battery(oracle._load()) == set()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "bfs_oracle_mut.c"
    mutated.write_text(src.replace(before, after))
    so = oracle.build(force=True, src=str(mutated), out=str(tmp_path / f"libmut_{name}.so"))
    lib = oracle.load_variant(so)
    assert pin_battery(lib), f"mutant {name} was not caught by any pin"
