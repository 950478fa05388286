"""Pins for the oracle's single-source betweenness (Alg. 2), against facts
fixed by the definition rather than by the algorithm's rounds:
  - closed forms on paths, stars, complete graphs, and shortest-path counts
    on an intact grid (binomial coefficients);
  - the definition itself on many tiny graphs: for v != s, the sum over
    targets t of sigma_st(v) / sigma_st with sigma_st(v) = sigma_sv *
    sigma_vt when d(s,v) + d(v,t) = d(s,t), from all-pairs BFS path counts;
    at v = s the algorithm's accumulation gives the number of other
    reachable vertices;
  - the identity sum_{v != s} D[v] = sum_t (d(s,t) - 1) over reachable t.
"""
import math

import numpy as np
import pytest

import graphgen as G
import oracle

INF = oracle.INF


def _bfs_counts(g, s):
    n = g.n
    d = np.full(n, -1, dtype=np.int64)
    sig = np.zeros(n, dtype=np.float64)
    d[s], sig[s] = 0, 1.0
    q = [s]
    for u in q:
        for k in range(g.off[u], g.off[u + 1]):
            v = int(g.tgt[k])
            if d[v] < 0:
                d[v] = d[u] + 1
                q.append(v)
            if d[v] == d[u] + 1:
                sig[v] += sig[u]
    return d, sig


def _definition(g, s):
    n = g.n
    ds, ss = _bfs_counts(g, s)
    allc = [_bfs_counts(g, v) for v in range(n)]
    out = np.zeros(n, dtype=np.float64)
    for v in range(n):
        if v == s:
            out[v] = float((ds >= 0).sum() - 1)
            continue
        if ds[v] < 0:
            continue
        dv, sv = allc[v]
        tot = 0.0
        for t in range(n):
            if t in (s, v) or ds[t] < 0:
                continue
            if dv[t] >= 0 and ds[v] + dv[t] == ds[t]:
                tot += ss[v] * sv[t] / ss[t]
        out[v] = tot
    return out


def test_path_star_complete():
    n = 9
    assert oracle.betweenness(G.path_graph(n), 0).tolist() == [n - 1 - v for v in range(n)]
    D = oracle.betweenness(G.path_graph(n), 4)
    assert D.tolist() == [0, 1, 2, 3, 8, 3, 2, 1, 0]
    st = G.star_graph(7)
    assert oracle.betweenness(st, 0).tolist() == [6, 0, 0, 0, 0, 0, 0]
    assert oracle.betweenness(st, 3).tolist() == [5, 0, 0, 6, 0, 0, 0]
    assert oracle.betweenness(G.complete_graph(8), 2).tolist() == [0, 0, 7, 0, 0, 0, 0, 0]


def test_grid_path_counts_and_levels():
    R, C = 7, 9
    g = G.grid_graph(R, C)
    D, paths, level = oracle.betweenness(g, 0, full=True)
    for r in range(R):
        for c in range(C):
            v = r * C + c
            assert level[v] == r + c
            assert paths[v] == math.comb(r + c, r)
    hops, _ = oracle.bfs(g, 17, parents=False)
    assert np.array_equal(oracle.betweenness(g, 17, full=True)[2], hops)


@pytest.mark.parametrize("seed", range(40))
def test_definition_on_tiny_graphs(seed):
    g = G.random_small(8 + seed % 6, 0.3, seed=300 + seed)
    for s in range(g.n):
        assert np.allclose(oracle.betweenness(g, s), _definition(g, s), rtol=1e-12, atol=1e-12)


def test_dependency_sum_identity_rmat():
    g = G.rmat(11, 8, seed=41)
    for s in G.sources(g, 3, seed=3):
        D, _, level = oracle.betweenness(g, int(s), full=True)
        others = np.ones(g.n, bool)
        others[int(s)] = False
        reach = (level > 0)
        lhs = D[others].sum()
        rhs = float((level[reach] - 1).sum())
        assert abs(lhs - rhs) <= 1e-9 * max(1.0, rhs)


def test_unreachable_zero_and_isolated_source():
    g = G.csr_from_edges(8, [(0, 1), (1, 2), (4, 5)])
    D, paths, level = oracle.betweenness(g, 0, full=True)
    assert D.tolist() == [2, 1, 0, 0, 0, 0, 0, 0]
    assert level.tolist() == [0, 1, 2, -1, -1, -1, -1, -1]
    assert oracle.betweenness(g, 7).tolist() == [0] * 8
