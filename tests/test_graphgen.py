"""Input generator checks: determinism, CSR shape, symmetry, no self-loops or
duplicates, and the expected sizes and degree structure. CPU only."""
import numpy as np
import pytest

import graphgen as gg


def csr_ok(g):
    off, idx = g.off, g.idx
    assert off[0] == 0 and off[-1] == g.m
    assert np.all(np.diff(off) >= 0)
    assert idx.min(initial=0) >= 0 and idx.max(initial=-1) < g.n
    src = np.repeat(np.arange(g.n), np.diff(off))
    assert not np.any(src == idx), "self-loop"
    # rows strictly ascending -> sorted and duplicate-free
    same_row = src[1:] == src[:-1]
    assert np.all(idx[1:][same_row] > idx[:-1][same_row])
    # symmetric: the multiset of (u, v) equals that of (v, u)
    a = np.sort(src.astype(np.int64) * g.n + idx)
    b = np.sort(idx.astype(np.int64) * g.n + src)
    assert np.array_equal(a, b)


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first two outputs of the published generator
    assert gg.splitmix64_at(0, 0) == 0xE220A8397B1DCDAF
    assert gg.splitmix64_at(0, 1) == 0x6E789E6AA1B965F4


@pytest.mark.parametrize("make", [
    lambda: gg.rmat(12, 16, seed=1),
    lambda: gg.rmat(10, 8, seed=2, permute=True),
    lambda: gg.grid(40, 33, 0.1, seed=3),
    lambda: gg.grid(20, 20, 0.0, seed=3, permute=False),
    lambda: gg.erdos_renyi(5000, 8.0, seed=4),
])
def test_csr_well_formed_and_deterministic(make):
    g1, g2 = make(), make()
    csr_ok(g1)
    assert np.array_equal(g1.off, g2.off) and np.array_equal(g1.idx, g2.idx)


def test_sizes():
    g = gg.grid(20, 20, 0.0, permute=False)
    assert g.m == 2 * (2 * 20 * 19)
    g = gg.grid(64, 64, 0.1, seed=9)
    full = 2 * 64 * 63
    assert 0.85 * full < g.m / 2 < 0.95 * full
    g = gg.erdos_renyi(20000, 8.0, seed=5)
    assert abs(g.m / g.n - 8.0) < 0.2
    g = gg.rmat(14, 16, seed=1000)
    assert g.n == 16384 and 0.6 * 2 * 16 * 16384 < g.m <= 2 * 16 * 16384
    deg = g.degrees()
    assert deg.max() > 50 * deg.mean()  # skewed


def test_roots():
    g = gg.rmat(12, 8, seed=3)
    r = gg.sample_roots(g, 16, seed=5)
    assert r.shape == (16,) and len(set(r.tolist())) == 16
    assert np.all(g.degrees()[r] > 0)
    comp, size, lab = gg.components(g)
    rg = gg.sample_roots(g, 16, seed=5, giant=True)
    assert np.all(comp[rg] == lab) and size == int((comp == lab).sum())
    assert np.array_equal(rg, gg.sample_roots(g, 16, seed=5, giant=True))
