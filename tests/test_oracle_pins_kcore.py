"""Pins for the oracle's coreness (§4 "k-core"), against the definition:
closed forms, brute-force k-cores by repeated deletion, networkx's
core_number (an independent implementation), and the defining invariant
(the vertices of coreness >= k induce a subgraph of minimum degree >= k,
and no vertex of coreness k lies in a (k+1)-core)."""
import numpy as np
import pytest

import graphgen as G
import oracle


def _kcore_members(g, k):
    alive = np.ones(g.n, bool)
    deg = np.diff(g.off.astype(np.int64)).copy()
    changed = True
    while changed:
        changed = False
        for v in range(g.n):
            if alive[v] and deg[v] < k:
                alive[v] = False
                changed = True
                for e in range(g.off[v], g.off[v + 1]):
                    deg[int(g.tgt[e])] -= 1
    return alive


def _brute(g):
    core = np.zeros(g.n, dtype=np.int64)
    maxd = int(np.diff(g.off.astype(np.int64)).max()) if g.n else 0
    for k in range(1, maxd + 1):
        mem = _kcore_members(g, k)
        if not mem.any():
            break
        core[mem] = k
    return core


def test_closed_forms():
    assert oracle.coreness(G.path_graph(7)).tolist() == [1] * 7
    assert oracle.coreness(G.complete_graph(6)).tolist() == [5] * 6
    assert oracle.coreness(G.star_graph(9)).tolist() == [1] * 9
    assert oracle.coreness(G.grid_graph(5, 6)).tolist() == [2] * 30
    cyc = G.csr_from_edges(7, [(i, (i + 1) % 7) for i in range(7)])
    assert oracle.coreness(cyc).tolist() == [2] * 7
    # K5 on 0..4, a pendant path 4-5-6, an isolated vertex 7
    edges = [(i, j) for i in range(5) for j in range(i + 1, 5)] + [(4, 5), (5, 6)]
    assert oracle.coreness(G.csr_from_edges(8, edges)).tolist() == [4, 4, 4, 4, 4, 1, 1, 0]


@pytest.mark.parametrize("seed", range(30))
def test_bruteforce_definition(seed):
    g = G.random_small(12 + seed % 9, 0.25 + 0.02 * (seed % 10), seed=500 + seed)
    assert np.array_equal(oracle.coreness(g), _brute(g))


def test_networkx_rmat():
    nx = pytest.importorskip("networkx")
    for sc, seed in ((10, 3), (11, 4)):
        g = G.rmat(sc, 8, seed=seed)
        h = nx.Graph()
        h.add_nodes_from(range(g.n))
        u = np.repeat(np.arange(g.n), np.diff(g.off.astype(np.int64)))
        h.add_edges_from(zip(u.tolist(), g.tgt.tolist()))
        ref = nx.core_number(h)
        assert oracle.coreness(g).tolist() == [ref[v] for v in range(g.n)]


def test_invariant_rmat():
    g = G.rmat(12, 16, seed=7)
    core = oracle.coreness(g)
    deg = np.diff(g.off.astype(np.int64))
    assert np.all(core <= deg)
    u = np.repeat(np.arange(g.n), deg)
    for k in sorted(set(core.tolist()))[::7]:
        inside = core >= k
        # degree inside the subgraph induced by coreness >= k
        din = np.bincount(u[inside[u] & inside[g.tgt]], minlength=g.n)
        assert np.all(din[inside] >= k)
