"""Pins for the oracle's Bellman-Ford (Alg. 4) and widest path (the same
rounds over the (max, min) semiring, §5 "Widest Path"), checked against
facts fixed by other methods, never against the oracle itself:
  - Bellman-Ford distances equal Dijkstra's and brute-force Floyd–Warshall's,
    unit weights give hop distances, and its round count on unit weights is
    the source's eccentricity + 1 (one round per nonempty frontier);
  - widest-path widths equal the bottleneck on the path of a maximum
    spanning forest (an independent characterisation), the max-min over all
    simple paths enumerated on tiny graphs, and closed forms on paths, stars
    and constant weights.
"""
import itertools

import numpy as np
import pytest

import graphgen as G
import oracle

INF = oracle.INF


# ------------------------------------------------------------ Bellman-Ford
def test_bf_path_prefix_sums():
    w = [3, 1, 4, 1, 5, 9, 2, 6]
    g = G.path_graph(len(w) + 1, weights=w)
    d = oracle.bellman_ford(g, 0)
    assert d.tolist() == np.concatenate([[0], np.cumsum(w)]).tolist()


@pytest.mark.parametrize("seed", range(40))
def test_bf_equals_dijkstra_and_floyd_warshall(seed):
    g = G.random_small(9 + seed % 7, 0.35, seed=seed, w_hi=9)
    fw = oracle.floyd_warshall(g, weighted=True)
    for s in range(g.n):
        d = oracle.bellman_ford(g, s)
        assert np.array_equal(d, oracle.dijkstra(g, s))
        row = fw[s].copy()
        row[row == np.iinfo(np.int64).max] = INF
        assert np.array_equal(d.astype(np.int64), row)


def test_bf_rmat_equals_dijkstra():
    g = G.add_weights(G.rmat(11, 8, seed=21), 1, 22, seed=22)
    for s in G.sources(g, 4, seed=3):
        assert np.array_equal(oracle.bellman_ford(g, int(s)), oracle.dijkstra(g, int(s)))


def test_bf_unit_weights_hops_and_rounds():
    g = G.add_weights(G.grid(12, 15, 0.1, seed=8), 1, 2, seed=9)  # all weights 1
    for s in (0, 57, 179):
        d, r = oracle.bellman_ford(g, s, rounds=True)
        hops, _ = oracle.bfs(g, s, parents=False)
        assert np.array_equal(d, hops)
        assert r == int(hops[hops != INF].max()) + 1


# ------------------------------------------------------------- widest path
def _widest_by_max_spanning_forest(g, s):
    """Kruskal on decreasing weights (union-find), then the smallest weight on
    each tree path from s."""
    n = g.n
    u = np.repeat(np.arange(n), np.diff(g.off.astype(np.int64)))
    v = g.tgt.astype(np.int64)
    w = g.w.astype(np.int64)
    keep = u < v
    u, v, w = u[keep], v[keep], w[keep]
    order = np.argsort(-w, kind="stable")
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    adj = [[] for _ in range(n)]
    for i in order:
        a, b = find(int(u[i])), find(int(v[i]))
        if a != b:
            parent[a] = b
            adj[int(u[i])].append((int(v[i]), int(w[i])))
            adj[int(v[i])].append((int(u[i]), int(w[i])))
    out = np.full(n, INF, dtype=np.int64)
    stack, seen = [(s, INF)], {s}
    while stack:
        x, bw = stack.pop()
        out[x] = bw
        for y, wy in adj[x]:
            if y not in seen:
                seen.add(y)
                stack.append((y, min(bw, wy)))
    return out  # unreachable stays INF (the output convention)


def _widest_brute(g, s):
    n = g.n
    nbr = {x: {} for x in range(n)}
    for x in range(n):
        for k in range(g.off[x], g.off[x + 1]):
            nbr[x][int(g.tgt[k])] = int(g.w[k])
    best = np.full(n, INF, dtype=np.int64)
    found = np.zeros(n, bool)
    found[s] = True

    def dfs(x, width, visited):
        for y, wy in nbr[x].items():
            if y in visited:
                continue
            nw = min(width, wy)
            if not found[y] or nw > best[y]:
                best[y] = nw
                found[y] = True
            dfs(y, nw, visited | {y})

    dfs(s, INF, {s})
    best[s] = INF
    return best


def test_widest_path_graph_prefix_min():
    w = [7, 3, 9, 2, 8, 8, 1, 5]
    g = G.path_graph(len(w) + 1, weights=w)
    d = oracle.widest_path(g, 0)
    assert d[0] == INF
    assert d[1:].tolist() == np.minimum.accumulate(w).tolist()
    d4 = oracle.widest_path(g, 4)
    assert d4[3] == 2 and d4[5] == 8 and d4[0] == 2 and d4[8] == 1


def test_widest_star_and_constant_weights():
    g = G.star_graph(6)
    # weight of the undirected edge (0, i) = 10 i, the same in both directions
    w = np.empty(g.m, dtype=np.uint32)
    for x in range(g.n):
        for k in range(g.off[x], g.off[x + 1]):
            y = int(g.tgt[k])
            w[k] = 10 * max(x, y)
    g.w = w
    assert oracle.widest_path(g, 0).tolist() == [INF, 10, 20, 30, 40, 50]
    assert oracle.widest_path(g, 3).tolist() == [30, 10, 20, INF, 30, 30]
    h = G.add_weights(G.grid(6, 7, 0.0, seed=1), 4, 5, seed=1)  # every weight 4
    d = oracle.widest_path(h, 10)
    assert d[10] == INF and set(np.delete(d, 10).tolist()) == {4}


@pytest.mark.parametrize("seed", range(30))
def test_widest_equals_bruteforce_and_spanning_forest(seed):
    g = G.random_small(7 + seed % 3, 0.45, seed=100 + seed, w_hi=6)
    for s in range(g.n):
        d = oracle.widest_path(g, s).astype(np.int64)
        assert np.array_equal(d, _widest_brute(g, s)), s
        assert np.array_equal(d, _widest_by_max_spanning_forest(g, s)), s


def test_widest_rmat_equals_spanning_forest():
    g = G.add_weights(G.rmat(9, 8, seed=31), 1, 22, seed=32)
    for s in G.sources(g, 3, seed=3):
        d = oracle.widest_path(g, int(s)).astype(np.int64)
        assert np.array_equal(d, _widest_by_max_spanning_forest(g, int(s)))
