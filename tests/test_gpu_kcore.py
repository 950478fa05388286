"""GPU parity: coreness (§4 "k-core"; Alg. 16) through the C ABI against the
pinned oracle, element by element (integers, unique answer)."""
import numpy as np
import pytest

import graphgen as G
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_05208_gb300 as gb
    return gb


OPTS = (None, dict(block=128, heavy_cutoff=256, ctas=7), dict(block=512), dict(block=1024, heavy_cutoff=4096))


def _parity(gb, csr, opts=OPTS):
    g = gb.Graph(csr, validate=gb.VALIDATE_BASIC | gb.VALIDATE_SYMMETRIC)
    ref = oracle.coreness(csr)
    for o in opts:
        c = g.kcore(None if o is None else gb.gbf_options_default(**o))
        assert np.array_equal(c, ref), (csr.name, o, int(np.sum(c != ref)))
        assert g.stats()["device_error"] == 0
    g.close()


def test_closed_forms(gb):
    _parity(gb, G.path_graph(50))
    _parity(gb, G.complete_graph(40))
    _parity(gb, G.star_graph(300))
    _parity(gb, G.grid_graph(30, 40))
    edges = [(i, j) for i in range(5) for j in range(i + 1, 5)] + [(4, 5), (5, 6)]
    _parity(gb, G.csr_from_edges(8, edges))


@pytest.mark.parametrize("scale,ef", [(10, 4), (13, 16), (16, 16)])
def test_rmat(gb, scale, ef):
    _parity(gb, G.rmat(scale, ef, seed=scale))


def test_grid_deleted_and_rmat18(gb):
    _parity(gb, G.grid(150, 200, 0.1, seed=7), opts=(None, dict(ctas=3)))
    _parity(gb, G.rmat(18, 16, seed=18), opts=(None,))
