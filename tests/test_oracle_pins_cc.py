"""Pins for the oracle's connected components (§4 "Connectivity"): closed
forms, SciPy's connected_components (an independent implementation) mapped to
the canonical labelling (the smallest id of each component), a union-find
over the arc list on seeded tiny graphs, and the labelling's invariants."""
import numpy as np
import pytest

import graphgen as G
import oracle


def _canonical(n, labels):
    """Relabel any partition by the smallest vertex id of each part."""
    first = {}
    out = np.empty(n, dtype=np.int64)
    for v in range(n):
        out[v] = first.setdefault(int(labels[v]), v)
    return out


def _union_find(g):
    parent = list(range(g.n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for u in range(g.n):
        for e in range(int(g.off[u]), int(g.off[u + 1])):
            a, b = find(u), find(int(g.tgt[e]))
            if a != b:
                parent[max(a, b)] = min(a, b)
    return np.array([find(v) for v in range(g.n)], dtype=np.int64)


def test_closed_forms():
    assert oracle.components(G.path_graph(9)).tolist() == [0] * 9
    assert oracle.components(G.star_graph(7)).tolist() == [0] * 7
    assert oracle.components(G.grid_graph(6, 7)).tolist() == [0] * 42
    assert oracle.components(G.csr_from_edges(5, [])).tolist() == [0, 1, 2, 3, 4]
    # a triangle on {4, 6, 2}, an edge {7, 3}, isolated 0, 1, 5
    g = G.csr_from_edges(8, [(4, 6), (6, 2), (2, 4), (7, 3)])
    assert oracle.components(g).tolist() == [0, 1, 2, 3, 2, 5, 2, 3]


@pytest.mark.parametrize("seed", range(25))
def test_union_find_on_tiny_graphs(seed):
    g = G.random_small(5 + seed % 30, [0.02, 0.08, 0.2][seed % 3], 700 + seed)
    assert np.array_equal(oracle.components(g), _union_find(g))


def test_scipy_on_rmat_and_deleted_grid():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for g in (G.rmat(14, 4, seed=31), G.grid(80, 90, 0.45, seed=32)):
        a = sp.csr_matrix((np.ones(g.m, dtype=np.int8), g.tgt, g.off.astype(np.int64)),
                          shape=(g.n, g.n))
        k, lab = csgraph.connected_components(a, directed=False)
        ours = oracle.components(g)
        assert np.array_equal(ours, _canonical(g.n, lab))
        assert int((ours == np.arange(g.n)).sum()) == k


def test_invariants_rmat():
    g = G.rmat(15, 8, seed=33)
    lab = oracle.components(g).astype(np.int64)
    v = np.arange(g.n)
    assert np.all(lab <= v) and np.all(lab[lab] == lab)
    src = np.repeat(v, np.diff(g.off.astype(np.int64)))
    assert np.array_equal(lab[src], lab[g.tgt])        # no arc crosses components
    # each component's BFS from its label reaches exactly its members
    for root in np.unique(lab)[:20]:
        d, _ = oracle.bfs(g, int(root), parents=False)
        assert np.array_equal(d != oracle.INF, lab == root)
