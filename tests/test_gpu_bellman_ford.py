"""GPU parity: frontier Bellman-Ford (Alg. 4) and widest path ((max, min)
rounds, §5) through the C ABI against the oracle, element by element and
bit-exact (integer values, unique answers)."""
import numpy as np
import pytest

import graphgen as G
import oracle

pytestmark = pytest.mark.gpu

INF = oracle.INF


@pytest.fixture(scope="module")
def gb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_05208_gb300 as gb
    return gb


OPTS = (None, dict(block=128, heavy_cutoff=256, ctas=7), dict(block=512), dict(block=1024, heavy_cutoff=4096))


def _parity(gb, csr, srcs, opts=OPTS):
    g = gb.Graph(csr, validate=gb.VALIDATE_BASIC | gb.VALIDATE_SYMMETRIC)
    for s in srcs:
        ref_d = oracle.bellman_ford(csr, int(s))
        ref_w = oracle.widest_path(csr, int(s))
        for o in opts:
            opt = None if o is None else gb.gbf_options_default(**o)
            d = g.bellman_ford(int(s), opt)
            assert np.array_equal(d, ref_d), (csr.name, int(s), o, "bf")
            w = g.widest_path(int(s), opt)
            assert np.array_equal(w, ref_w), (csr.name, int(s), o, "widest")
            st = g.stats()
            assert st["device_error"] == 0
    g.close()


def test_closed_forms(gb):
    w = [3, 1, 4, 1, 5, 9, 2, 6]
    _parity(gb, G.path_graph(len(w) + 1, weights=w), [0, 4, 8])
    _parity(gb, G.add_weights(G.grid_graph(30, 40), 1, 2, seed=1), [0, 617])   # unit weights
    _parity(gb, G.add_weights(G.csr_from_edges(10, [(0, 1), (1, 2), (5, 6), (6, 7)]), 2, 9, seed=3),
            [1, 5, 9])                                                          # components, isolated


def test_unit_weights_equal_bfs(gb):
    csr = G.add_weights(G.rmat(12, 16, seed=4), 1, 2, seed=5)
    g = gb.Graph(csr)
    for s in G.sources(csr, 3, seed=3):
        hops, _ = oracle.bfs(csr, int(s), parents=False)
        assert np.array_equal(g.bellman_ford(int(s)), hops)
    g.close()


@pytest.mark.parametrize("scale,ef", [(10, 4), (13, 16), (16, 16)])
def test_rmat(gb, scale, ef):
    csr = G.add_weights(G.rmat(scale, ef, seed=scale), 1, 22, seed=scale + 1)
    _parity(gb, csr, list(G.sources(csr, 3, seed=3)) + [G.max_degree_vertex(csr)])


def test_grid_deleted_edges(gb):
    csr = G.add_weights(G.grid(150, 200, 0.1, seed=7), 1, 16, seed=8)
    _parity(gb, csr, [0, 12345], opts=(None, dict(ctas=3)))


def test_rmat18_default(gb):
    csr = G.add_weights(G.rmat(18, 16, seed=18), 1, 22, seed=19)
    _parity(gb, csr, G.sources(csr, 2, seed=3), opts=(None,))
