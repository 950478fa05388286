"""Input generator checks: structure (symmetric, sorted, no self-loops or
duplicates), determinism across thread counts, weights and sources."""
import numpy as np
import pytest

import graphgen as G


def _structure_ok(g):
    off, tgt = g.off.astype(np.int64), g.tgt.astype(np.int64)
    assert off[0] == 0 and np.all(np.diff(off) >= 0) and off[-1] == len(tgt)
    assert tgt.min(initial=0) >= 0 and tgt.max(initial=0) < g.n
    src = np.repeat(np.arange(g.n), np.diff(off))
    assert not np.any(src == tgt), "self-loop"
    key = src * g.n + tgt
    assert np.all(np.diff(key) > 0), "unsorted or duplicate arcs"
    rev = np.sort(tgt * g.n + src)
    assert np.array_equal(rev, key), "not symmetric"
    return src


def test_rmat_structure_and_thread_invariance():
    G.set_threads(1)
    a = G.rmat(12, 16, seed=11)
    G.set_threads(0)
    b = G.rmat(12, 16, seed=11)
    assert np.array_equal(a.off, b.off) and np.array_equal(a.tgt, b.tgt)
    _structure_ok(a)
    c = G.rmat(12, 16, seed=12)
    assert not np.array_equal(a.tgt[:1000], c.tgt[:1000])


def test_rmat_power_law_shape():
    g = G.rmat(14, 16, seed=1)
    d = g.degrees()
    # skewed degrees: the max is far above the mean, many vertices are light
    assert d.max() > 20 * d.mean()
    assert g.m > 10 * g.n


def test_rmat_unpermuted_hub_is_vertex_zero():
    g = G.rmat(10, 16, seed=3, permute=False)
    assert G.max_degree_vertex(g) == 0


def test_grid_structure():
    g = G.grid(30, 40, 0.1, seed=5)
    src = _structure_ok(g)
    d = np.abs(g.tgt.astype(np.int64) - src)
    assert set(np.unique(d)) <= {1, 40}
    full = 2 * (30 * 39 + 29 * 40)
    assert 0.85 * full < g.m < 0.95 * full
    g0 = G.grid(30, 40, 0.0, seed=5)
    assert g0.m == full


def test_weights_symmetric_and_in_range():
    g = G.add_weights(G.rmat(11, 16, seed=2), 1, 22, seed=9)
    assert g.w.min() >= 1 and g.w.max() <= 21
    src = np.repeat(np.arange(g.n), np.diff(g.off.astype(np.int64)))
    fwd = dict(zip((src * g.n + g.tgt).tolist(), g.w.tolist()))
    for s, t, w in zip(src[:5000], g.tgt[:5000], g.w[:5000]):
        assert fwd[int(t) * g.n + int(s)] == w
    counts = np.bincount(g.w, minlength=22)[1:]
    assert counts.min() > 0.5 * counts.mean()


def test_sources_have_degree():
    g = G.rmat(12, 4, seed=8)
    s = G.sources(g, 64, seed=3)
    assert np.all(g.degrees()[s] > 0)
    assert np.array_equal(s, G.sources(g, 64, seed=3))


def test_max_degree_vertex_tie_break():
    g = G.csr_from_edges(6, [(1, 2), (1, 3), (4, 2), (4, 3), (5, 0)])
    assert G.max_degree_vertex(g) == 1
