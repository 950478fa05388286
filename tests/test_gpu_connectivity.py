"""GPU parity: connected components through the C ABI against the oracle's
canonical labelling (the smallest vertex id of each component), element by
element: closed forms, isolated vertices, tiny graphs, RMAT graphs with many
isolated vertices, grids cut into many pieces, a long path (many rounds),
device buffers and streams."""
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


def _parity(gb, csr, opts=(None,)):
    g = gb.Graph(csr)
    ref = oracle.components(csr)
    for o in opts:
        assert np.array_equal(g.connectivity(opt=o), ref), (csr.name, o and o.block)
    g.close()


def test_closed_forms(gb):
    for csr in (G.path_graph(5000), G.star_graph(3000), G.grid_graph(60, 70),
                G.csr_from_edges(9, [(4, 6), (6, 2), (2, 4), (7, 3)]),
                G.csr_from_edges(3, [])):
        _parity(gb, csr)


def test_tiny_many(gb):
    for s in range(40):
        _parity(gb, G.random_small(2 + s % 60, [0.01, 0.05, 0.2][s % 3], 1300 + s))


@pytest.mark.parametrize("scale,ef", [(10, 2), (14, 4), (16, 16)])
def test_rmat(gb, scale, ef):
    _parity(gb, G.rmat(scale, ef, seed=scale + 40),
            opts=(None, gb.gbf_options_default(block=512, ctas=9),
                  gb.gbf_options_default(block=128)))


def test_grid_pieces(gb):
    _parity(gb, G.grid(200, 210, 0.45, seed=41))
    _parity(gb, G.grid(300, 300, 0.1, seed=42))


def test_device_buffers(gb):
    torch = pytest.importorskip("torch")
    csr = G.rmat(13, 4, seed=43)
    g = gb.Graph(csr)
    st = torch.cuda.Stream()
    lab = torch.empty(csr.n, dtype=torch.int32, device="cuda")
    gb.gbf_connectivity(g.h, lab, None, st)
    stats = gb.gbf_wait(g.h, st)
    assert stats["device_error"] == 0 and stats["rounds"] >= 1
    assert np.array_equal(lab.cpu().numpy(), oracle.components(csr))
