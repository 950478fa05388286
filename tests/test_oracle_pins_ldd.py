"""Pins for the oracle's low-diameter decomposition (§4; Alg. 6) with the
shifts given as an input.

The round T[u] in which u joins a frontier has a closed form: waves start at
each v in round s(v) = floor(max delta - delta[v]) and advance one hop per
round through any vertex, so T[u] = min over v of s(v) + dist(u, v).  This is
checked against SciPy's all-pairs shortest paths on seeded tiny graphs and
special cases.  The cluster choice where waves tie is not unique, so C is
checked by the invariants every run satisfies: a centre is its own centre and
joined in its start round; any other vertex has a neighbour in its cluster one
round earlier; clusters are connected through such neighbours."""
import numpy as np
import pytest

import graphgen as G
import oracle


def _start_rounds(delta):
    return np.maximum(np.floor(delta.max() - delta), 0).astype(np.int64)


def _check_clusters(g, delta, C, T):
    s = _start_rounds(delta)
    for u in range(g.n):
        c = int(C[u])
        assert 0 <= c < g.n and int(C[c]) == c, u
        if c == u:
            assert T[u] == s[u], u
        else:
            nb = g.tgt[g.off[u]:g.off[u + 1]]
            assert np.any((C[nb] == c) & (T[nb] == T[u] - 1)), u
        assert T[u] <= s[u], u  # nobody joins after its own start round


def _t_closed_form(g, delta):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    a = sp.csr_matrix((np.ones(g.m), g.tgt, g.off.astype(np.int64)), shape=(g.n, g.n))
    dist = csgraph.shortest_path(a, unweighted=True, directed=False)
    s = _start_rounds(delta)
    return np.min(dist + s[None, :], axis=1)


def test_special_cases():
    g = G.path_graph(6)
    # one shift far above the rest: a single wave from vertex 5
    C, T = oracle.ldd(g, np.array([0, 0, 0, 0, 0, 5.0]))
    assert C.tolist() == [5] * 6 and T.tolist() == [5, 4, 3, 2, 1, 0]
    # equal shifts: every vertex starts its own cluster in round 0
    C, T = oracle.ldd(g, np.full(6, 0.7))
    assert C.tolist() == list(range(6)) and T.tolist() == [0] * 6
    # isolated vertices are their own clusters
    g = G.csr_from_edges(4, [(0, 1)])
    C, T = oracle.ldd(g, np.array([3.0, 0.0, 0.5, 2.5]))
    assert C.tolist() == [0, 0, 2, 3] and T.tolist() == [0, 1, 2, 0]


@pytest.mark.parametrize("seed", range(30))
def test_rounds_closed_form_and_cluster_invariants(seed):
    g = G.random_small(6 + seed % 40, [0.05, 0.12, 0.3][seed % 3], 900 + seed)
    if g.m == 0:
        pytest.skip("no arcs")
    delta = G.exp_shifts(g.n, [0.1, 0.3, 1.0][seed % 3], seed=seed)
    C, T = oracle.ldd(g, delta)
    assert np.array_equal(T, _t_closed_form(g, delta))
    _check_clusters(g, delta, C, T)


def test_grid_and_rmat_invariants_and_cut_fraction():
    for g, beta in ((G.grid(40, 50, 0.1, seed=3), 0.2), (G.rmat(12, 8, seed=4), 0.2)):
        delta = G.exp_shifts(g.n, beta, seed=11)
        C, T = oracle.ldd(g, delta)
        _check_clusters(g, delta, C, T)
        src = np.repeat(np.arange(g.n), np.diff(g.off.astype(np.int64)))
        cut = float(np.mean(C[src] != C[g.tgt]))
        # O(beta) cut arcs: the expected fraction is at most about 2 beta
        assert cut <= 2 * beta + 0.05, cut
