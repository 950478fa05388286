"""GPU parity: low-diameter decomposition (Alg. 6) through the C ABI against
the oracle, with the shifts as an input.  The join round of every vertex is
unique and must match bit for bit; the cluster choice where searches tie is
not, so clusters are checked by the invariants every run satisfies (a centre
is its own centre and joined in its start round; any other vertex has a
neighbour of its cluster one round earlier)."""
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


def _check(g, delta, C, T):
    s = np.maximum(np.floor(delta.max() - delta), 0).astype(np.int64)
    assert np.all((C >= 0) & (C < g.n))
    assert np.all(C[C] == C)
    src = np.repeat(np.arange(g.n), np.diff(g.off.astype(np.int64)))
    ok_nb = np.zeros(g.n, bool)
    same = (C[src] == C[g.tgt]) & (T[g.tgt] == T[src] - 1)
    np.logical_or.at(ok_nb, src, same)
    centre = C == np.arange(g.n)
    assert np.all(T[centre] == s[centre])
    assert np.all(ok_nb[~centre])
    assert np.all(T <= s)


def _parity(gb, csr, delta, opts=(None,)):
    g = gb.Graph(csr)
    _, Tref = oracle.ldd(csr, delta)
    for o in opts:
        C, T = g.ldd(delta, opt=o)
        assert np.array_equal(T, Tref), (csr.name, o and o.block)
        _check(csr, delta, C, T)
    g.close()


def test_special_cases(gb):
    g = gb.Graph(G.path_graph(6))
    C, T = g.ldd(np.array([0, 0, 0, 0, 0, 5.0]))
    assert C.tolist() == [5] * 6 and T.tolist() == [5, 4, 3, 2, 1, 0]
    C, T = g.ldd(np.full(6, 0.7))
    assert C.tolist() == list(range(6)) and T.tolist() == [0] * 6
    g2 = gb.Graph(G.csr_from_edges(4, [(0, 1)]))
    C, T = g2.ldd(np.array([3.0, 0.0, 0.5, 2.5]))
    assert C.tolist() == [0, 0, 2, 3] and T.tolist() == [0, 1, 2, 0]


def test_tiny_many(gb):
    for s in range(30):
        csr = G.random_small(6 + s % 50, [0.05, 0.12, 0.3][s % 3], 900 + s)
        _parity(gb, csr, G.exp_shifts(csr.n, [0.1, 0.3, 1.0][s % 3], seed=s))


@pytest.mark.parametrize("scale", [10, 14, 16])
def test_rmat(gb, scale):
    csr = G.rmat(scale, 16, seed=scale + 3)
    for beta in (0.05, 0.2, 1.0):
        _parity(gb, csr, G.exp_shifts(csr.n, beta, seed=scale),
                opts=(None, gb.gbf_options_default(block=512, ctas=7)))


def test_grid(gb):
    csr = G.grid(150, 160, 0.1, seed=5)
    _parity(gb, csr, G.exp_shifts(csr.n, 0.1, seed=6))


def test_device_buffers_and_invalid_shifts(gb):
    torch = pytest.importorskip("torch")
    csr = G.rmat(12, 16, seed=8)
    g = gb.Graph(csr)
    delta = G.exp_shifts(csr.n, 0.2, seed=9)
    st = torch.cuda.Stream()
    d = torch.from_numpy(delta).cuda()
    C = torch.empty(csr.n, dtype=torch.int32, device="cuda")
    T = torch.empty(csr.n, dtype=torch.int32, device="cuda")
    gb.gbf_ldd(g.h, d, C, T, None, st)
    stats = gb.gbf_wait(g.h, st)
    assert stats["device_error"] == 0 and stats["vertices_reached"] == csr.n
    _, Tref = oracle.ldd(csr, delta)
    assert np.array_equal(T.cpu().numpy(), Tref)
    _check(csr, delta, C.cpu().numpy(), T.cpu().numpy())
    for bad in (-1.0, float("nan"), float("inf")):
        b = delta.copy()
        b[17] = bad
        with pytest.raises(gb.GbfError) as e:
            g.ldd(b)
        assert e.value.status == 1
    wide = delta.copy()
    wide[3] = 1e8  # a start round beyond 2^22
    with pytest.raises(gb.GbfError):
        g.ldd(wide)
    C2, T2 = g.ldd(delta)  # the handle stays usable
    assert np.array_equal(T2, Tref)
