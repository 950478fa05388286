"""Pins for the oracle: checks against facts fixed by the mathematics and the
paper's problem statements (§4, BFS and integral-weight SSSP), never against
the oracle itself.  A plausible mistake (a dropped relaxation, an off-by-one
level, a wrong heap order, a transposed index) fails at least one of these.
"""
import os

import numpy as np
import pytest

import graphgen as G
import oracle

INF = oracle.INF
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fw_row(d, s):
    r = d[s].copy()
    r[r == np.iinfo(np.int64).max] = INF
    return r.astype(np.int64)


# --------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n,s", [(1, 0), (2, 1), (17, 0), (17, 16), (33, 9)])
def test_path_hops(n, s):
    g = G.path_graph(n)
    d, p = oracle.bfs(g, s)
    assert np.array_equal(d, np.abs(np.arange(n) - s))
    for v in range(n):
        if v != s:
            assert abs(p[v] - v) == 1 and d[p[v]] == d[v] - 1


def test_path_weighted_prefix_sums():
    n = 40
    w = np.arange(1, n) % 7 + 1          # edge i-(i+1) has weight w[i]
    g = G.path_graph(n, weights=w)
    pref = np.concatenate([[0], np.cumsum(w)])
    for s in (0, 13, n - 1):
        d = oracle.dijkstra(g, s)
        assert np.array_equal(d, np.abs(pref - pref[s]))


def test_star():
    n = 50
    g = G.star_graph(n)
    d, _ = oracle.bfs(g, 0)
    assert d[0] == 0 and np.all(d[1:] == 1)
    d, p = oracle.bfs(g, 7)
    exp = np.full(n, 2)
    exp[0], exp[7] = 1, 0
    assert np.array_equal(d, exp)
    assert p[0] == 7 and np.all(p[np.arange(n) > 0][np.arange(1, n) != 7] == 0)


def test_complete():
    for n in (2, 5, 30):
        g = G.complete_graph(n)
        for s in (0, n - 1):
            d, _ = oracle.bfs(g, s)
            exp = np.ones(n, dtype=np.int64)
            exp[s] = 0
            assert np.array_equal(d, exp)


@pytest.mark.parametrize("R,C,src", [(1, 9, 4), (7, 5, 0), (12, 13, 77), (30, 30, 899)])
def test_grid_manhattan(R, C, src):
    g = G.grid_graph(R, C)
    d, _ = oracle.bfs(g, src)
    r0, c0 = divmod(src, C)
    rr, cc = np.divmod(np.arange(R * C), C)
    man = np.abs(rr - r0) + np.abs(cc - c0)
    assert np.array_equal(d, man)
    gw = G.grid_graph(R, C, weight=5)
    assert np.array_equal(oracle.dijkstra(gw, src), 5 * man)


def test_two_components():
    g = G.csr_from_edges(10, [(0, 1), (1, 2), (2, 3), (5, 6), (6, 7), (7, 8), (8, 9)],
                         weights=[3, 3, 3, 1, 1, 1, 1])
    d, p = oracle.bfs(g, 1)
    assert list(d[:4]) == [1, 0, 1, 2]
    assert np.all(d[4:] == INF) and np.all(p[4:] == -1)
    dw = oracle.dijkstra(g, 1)
    assert list(dw[:4]) == [3, 0, 3, 6] and np.all(dw[4:] == INF)


def test_isolated_source():
    g = G.csr_from_edges(5, [(1, 2), (2, 3)])
    d, p = oracle.bfs(g, 0)
    assert d[0] == 0 and p[0] == 0 and np.all(d[1:] == INF) and np.all(p[1:] == -1)


# --------------------------------------------------------- hand-worked fixture
def _read_golden(name):
    n = src = None
    edges, ws, rows = [], [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            t = line.split("#")[0].split()
            if not t:
                continue
            if t[0] == "n":
                n = int(t[1])
            elif t[0] == "src":
                src = int(t[1])
            elif t[0] == "edge":
                edges.append((int(t[1]), int(t[2])))
                ws.append(int(t[3]))
            else:
                rows[t[0]] = np.array([INF if x == "inf" else int(x) for x in t[1:]])
    return n, src, edges, ws, rows


def test_golden_hand_worked():
    n, src, edges, ws, rows = _read_golden("hand_worked_8v.txt")
    g = G.csr_from_edges(n, edges, ws)
    d, p = oracle.bfs(g, src)
    assert np.array_equal(d, rows["bfs"])
    assert np.array_equal(oracle.dijkstra(g, src), rows["sssp"])


# ------------------------------------------------------- brute force (n <= 64)
def test_floyd_warshall_closed_form():
    # FW itself is pinned on a grid (Manhattan) before it pins anything else.
    g = G.grid_graph(6, 7, weight=3)
    d = oracle.floyd_warshall(g, weighted=True)
    rr, cc = np.divmod(np.arange(42), 7)
    man = np.abs(rr[:, None] - rr[None, :]) + np.abs(cc[:, None] - cc[None, :])
    assert np.array_equal(d, 3 * man)


def test_bruteforce_many_tiny_graphs():
    count = 0
    for seed in range(260):
        n = 2 + seed % 63
        p = [0.03, 0.08, 0.2, 0.5][seed % 4]
        g = G.random_small(n, p, seed, w_hi=[2, 5, 22, 100][(seed // 4) % 4])
        dfw_u = oracle.floyd_warshall(g, weighted=False)
        dfw_w = oracle.floyd_warshall(g, weighted=True)
        for s in {0, n - 1, seed % n}:
            d, par = oracle.bfs(g, s)
            assert np.array_equal(d, _fw_row(dfw_u, s)), (seed, s)
            ok, v, why = oracle.check_bfs(g, s, d, par)
            assert ok, (seed, s, v, why)
            dw = oracle.dijkstra(g, s)
            assert np.array_equal(dw, _fw_row(dfw_w, s)), (seed, s)
            count += 2
    assert count >= 500


def test_scipy_csgraph_agrees():
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    for seed in range(12):
        g = G.random_small(300, 0.01 + 0.004 * seed, 1000 + seed, w_hi=22)
        A = sp.csr_matrix((g.w.astype(np.float64), g.tgt, g.off.astype(np.int64)),
                          shape=(g.n, g.n))
        U = sp.csr_matrix((np.ones(g.m), g.tgt, g.off.astype(np.int64)), shape=(g.n, g.n))
        for s in (0, 17, 299):
            ref_w = csg.dijkstra(A, directed=True, indices=s)
            ref_u = csg.shortest_path(U, method="D", directed=True, unweighted=True, indices=s)
            for ref, got in ((ref_w, oracle.dijkstra(g, s)), (ref_u, oracle.bfs(g, s)[0])):
                exp = np.where(np.isinf(ref), INF, ref).astype(np.int64)
                assert np.array_equal(got, exp)


def test_rmat_scipy_bfs_and_dijkstra():
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    g = G.add_weights(G.rmat(12, 8, seed=5), 1, 22, seed=6)
    A = sp.csr_matrix((g.w.astype(np.float64), g.tgt, g.off.astype(np.int64)), shape=(g.n, g.n))
    for s in G.sources(g, 3, seed=7):
        exp = csg.dijkstra(A, directed=True, indices=int(s))
        exp = np.where(np.isinf(exp), INF, exp).astype(np.int64)
        assert np.array_equal(oracle.dijkstra(g, int(s)), exp)
        ok, v, why = oracle.check_sssp(g, int(s), oracle.dijkstra(g, int(s)))
        assert ok, (v, why)


# ------------------------------------------------------------ identities
def test_unit_weight_sssp_equals_bfs():
    g = G.rmat(11, 8, seed=9)
    g.w = np.ones(g.m, dtype=np.uint32)
    for s in G.sources(g, 5, seed=1):
        d, _ = oracle.bfs(g, int(s))
        assert np.array_equal(oracle.dijkstra(g, int(s)), d)


def test_constant_weight_scales_bfs():
    g = G.grid(20, 25, 0.1, seed=4)
    g.w = np.full(g.m, 7, dtype=np.uint32)
    d, _ = oracle.bfs(g, 0)
    dw = oracle.dijkstra(g, 0)
    reach = d != INF
    assert np.array_equal(dw[reach], 7 * d[reach]) and np.all(dw[~reach] == INF)


# ---------------------------------------------- validators reject planted bugs
def test_validators_reject_planted_mistakes():
    g = G.add_weights(G.rmat(10, 8, seed=3), 1, 22, seed=4)
    s = int(G.sources(g, 1, seed=2)[0])
    d, p = oracle.bfs(g, s)
    assert oracle.check_bfs(g, s, d, p)[0]
    reached = np.flatnonzero((d != INF) & (np.arange(g.n) != s))
    v = int(reached[len(reached) // 2])
    bad = d.copy(); bad[v] += 1
    assert not oracle.check_bfs(g, s, bad, p)[0]
    bad = d.copy(); bad[s] = 1
    assert not oracle.check_bfs(g, s, bad, p)[0]
    badp = p.copy(); badp[v] = v
    assert not oracle.check_bfs(g, s, d, badp)[0]
    # a parent that is adjacent but on the same level
    nb = g.tgt[g.off[v]:g.off[v + 1]]
    same = [u for u in nb if d[u] == d[v]]
    if same:
        badp = p.copy(); badp[v] = same[0]
        assert not oracle.check_bfs(g, s, d, badp)[0]
    unreached = np.flatnonzero(d == INF)
    if len(unreached):
        badp = p.copy(); badp[unreached[0]] = s
        assert not oracle.check_bfs(g, s, d, badp)[0]
    dw = oracle.dijkstra(g, s)
    assert oracle.check_sssp(g, s, dw)[0]
    for delta in (+1, -1):
        bad = dw.copy(); bad[v] += delta
        assert not oracle.check_sssp(g, s, bad)[0]
    # distances from BFS are not shortest weighted distances
    assert not oracle.check_sssp(g, s, d)[0]
