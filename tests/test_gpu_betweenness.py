"""GPU parity: single-source betweenness (Alg. 2) through the C ABI against
the oracle.  Dependencies are fp64 sums whose order differs (fetch-and-add
from many warps), so they are compared with a stated tolerance: each value
is a sum over at most (levels x max degree) products, each rounded once in
fp64 (2^-53), so the relative error stays below 1e-9 for every graph here;
values that are integers in closed form (paths, stars, complete graphs)
are checked exactly."""
import numpy as np
import pytest

import graphgen as G
import oracle

pytestmark = pytest.mark.gpu

RTOL = 1e-9


@pytest.fixture(scope="module")
def gb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_05208_gb300 as gb
    return gb


def _close(a, b):
    scale = np.maximum(1.0, np.abs(b))
    return np.all(np.abs(a - b) <= RTOL * scale)


def _parity(gb, csr, srcs, opts=(None,)):
    g = gb.Graph(csr, validate=gb.VALIDATE_BASIC | gb.VALIDATE_SYMMETRIC)
    for s in srcs:
        ref = oracle.betweenness(csr, int(s))
        for o in opts:
            opt = None if o is None else gb.gbf_options_default(**o)
            d = g.betweenness(int(s), opt)
            assert _close(d, ref), (csr.name, int(s), o, float(np.max(np.abs(d - ref))))
            assert g.stats()["device_error"] == 0
    g.close()


def test_closed_forms_exact(gb):
    n = 9
    g = gb.Graph(G.path_graph(n))
    assert g.betweenness(0).tolist() == [n - 1 - v for v in range(n)]
    assert g.betweenness(4).tolist() == [0, 1, 2, 3, 8, 3, 2, 1, 0]
    g.close()
    st = gb.Graph(G.star_graph(7))
    assert st.betweenness(3).tolist() == [5, 0, 0, 6, 0, 0, 0]
    st.close()
    k = gb.Graph(G.complete_graph(8))
    assert k.betweenness(2).tolist() == [0, 0, 7, 0, 0, 0, 0, 0]
    k.close()
    iso = gb.Graph(G.csr_from_edges(8, [(0, 1), (1, 2), (4, 5)]))
    assert iso.betweenness(0).tolist() == [2, 1, 0, 0, 0, 0, 0, 0]
    assert iso.betweenness(7).tolist() == [0] * 8
    iso.close()


def test_grid(gb):
    _parity(gb, G.grid_graph(40, 50), [0, 1234], opts=(None, dict(ctas=3)))
    _parity(gb, G.grid(120, 150, 0.1, seed=7), [0, 9000])


@pytest.mark.parametrize("scale,ef", [(10, 4), (13, 16), (16, 16)])
def test_rmat(gb, scale, ef):
    csr = G.rmat(scale, ef, seed=scale)
    _parity(gb, csr, list(G.sources(csr, 3, seed=3)) + [G.max_degree_vertex(csr)],
            opts=(None, dict(block=128, heavy_cutoff=256, ctas=7), dict(block=1024, heavy_cutoff=4096)))


def test_rmat18(gb):
    csr = G.rmat(18, 16, seed=18)
    _parity(gb, csr, G.sources(csr, 2, seed=3))
