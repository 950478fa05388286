"""GPU parity for the multi-source integral-weight SSSP (gbf_mssp): row i must
equal the oracle's Dijkstra from srcs[i], bit for bit, for every source, on
closed-form graphs, seeded RMAT graphs and a high-diameter grid, with
duplicate and isolated sources, 1 to 8 lanes, and every knob setting."""
import numpy as np
import pytest

import graphgen as G
import oracle

pytestmark = pytest.mark.gpu

INF = 2**31 - 1


@pytest.fixture(scope="module")
def gb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_05208_gb300 as gb
    return gb


def _check(gb, csr, srcs, opts=(None,)):
    g = gb.Graph(csr)
    ref = np.stack([oracle.dijkstra(csr, int(s)) for s in srcs])
    for o in opts:
        d = g.mssp(srcs, opt=o)
        assert d.shape == (len(srcs), csr.n)
        bad = np.flatnonzero((d != ref).any(axis=1))
        assert bad.size == 0, (csr.name, bad[:5])
    st = g.stats()
    assert st["device_error"] == 0
    g.close()


def test_mssp_closed_forms(gb):
    n = 400
    wpath = (np.arange(1, n) % 7 + 1)
    path = G.path_graph(n, weights=wpath)
    pre = np.concatenate([[0], np.cumsum(wpath)])
    g = gb.Graph(path)
    srcs = [0, 399, 200]
    d = g.mssp(srcs)
    for i, s in enumerate(srcs):
        assert np.array_equal(d[i], np.abs(pre - pre[s]))   # prefix sums along the path
    g.close()
    grid = G.grid_graph(30, 40, weight=3)
    g = gb.Graph(grid)
    srcs = [0, 777, 1199]
    d = g.mssp(srcs)
    r, c = np.divmod(np.arange(grid.n), 40)
    for i, s in enumerate(srcs):
        assert np.array_equal(d[i], 3 * (np.abs(r - s // 40) + np.abs(c - s % 40)))
    g.close()
    comp = G.csr_from_edges(10, [(0, 1), (1, 2), (5, 6)], [3, 4, 5])
    g = gb.Graph(comp)
    d = g.mssp([1, 5, 9])
    assert d[0].tolist() == [3, 0, 4, INF, INF, INF, INF, INF, INF, INF]
    assert d[1].tolist() == [INF] * 5 + [0, 5] + [INF] * 3
    assert d[2].tolist() == [INF] * 9 + [0]
    g.close()


@pytest.mark.parametrize("scale", [10, 14, 16])
def test_mssp_rmat(gb, scale):
    csr = G.add_weights(G.rmat(scale, 16, seed=60 + scale), 1, 22, seed=61)
    s = list(G.sources(csr, 8, seed=62))
    s[3] = s[1]                                   # duplicate lane
    iso = np.flatnonzero(csr.degrees() == 0)
    if iso.size:
        s[6] = int(iso[0])                        # an isolated source
    opts = (None, gb.gbf_options_default(block=128, heavy_cutoff=256, ctas=7),
            gb.gbf_options_default(block=1024, heavy_cutoff=4096))
    for k in (1, 2, 5, 8):
        _check(gb, csr, np.array(s[:k], dtype=np.int32), opts=opts)


def test_mssp_grid_high_diameter(gb):
    csr = G.add_weights(G.grid(120, 150, 0.1, seed=3), 1, 16, seed=4)
    _check(gb, csr, np.array([0, 9000, 17999, 123, 4567, 8888, 13000, 50], dtype=np.int32))


def test_mssp_tiny_many(gb):
    for s in range(30):
        csr = G.random_small(2 + (s % 60), [0.05, 0.15, 0.4][s % 3], 300 + s, w_hi=[2, 9, 30][s % 3])
        k = 1 + s % 8
        srcs = np.array([(7 * i + s) % csr.n for i in range(k)], dtype=np.int32)
        _check(gb, csr, srcs)


def test_mssp_device_buffers_and_errors(gb):
    import torch
    csr = G.add_weights(G.rmat(12, 16, seed=70), 1, 22, seed=71)
    g = gb.Graph(csr)
    srcs = G.sources(csr, 8, seed=72)
    st = torch.cuda.Stream()
    out = torch.full((8, csr.n), -3, dtype=torch.int32, device="cuda")
    for rep in range(2):                          # the workspace is reused
        gb.gbf_mssp(g.h, srcs, out, None, st)
        assert gb.gbf_wait(g.h, st)["device_error"] == 0
        for i, s in enumerate(srcs):
            assert np.array_equal(out[i].cpu().numpy(), oracle.dijkstra(csr, int(s))), (rep, i)
    with pytest.raises(gb.GbfError):
        gb.gbf_mssp(g.h, np.zeros(9, dtype=np.int32), np.empty((9, csr.n), dtype=np.int32))
    with pytest.raises(gb.GbfError):
        gb.gbf_mssp(g.h, np.array([csr.n], dtype=np.int32), np.empty((1, csr.n), dtype=np.int32))
    g.close()
    unweighted = gb.Graph(G.path_graph(10))
    with pytest.raises(gb.GbfError):
        unweighted.mssp([0])
    unweighted.close()


def test_mssp_lane_width_limit_and_fallback(gb):
    """A query first runs with 16-bit lanes, which hold distances up to
    65,534.  A distance of 65,534 is exact in them; one of 65,535 does not
    fit, and the launch reruns the query with 32-bit lanes, bit-exact all the
    same, as are later calls on that graph (which start with 32-bit lanes).
    Lanes with near and far sources share one launch."""
    for wt, srcs in ((65534, [0, 1]), (65535, [0, 1]), (65536, [1, 0, 1])):
        csr = G.csr_from_edges(3, [(0, 1)], [wt])
        g = gb.Graph(csr)
        for rep in range(3):
            d = g.mssp(srcs)
            for i, s in enumerate(srcs):
                ref = oracle.dijkstra(csr, int(s))
                assert np.array_equal(d[i], ref), (wt, rep, i, d[i], ref)
        g.close()
    n = 300
    w = np.full(n - 1, 500, dtype=np.int64)     # distances up to 149,500
    path = G.path_graph(n, weights=w)
    pre = np.concatenate([[0], np.cumsum(w)])
    g = gb.Graph(path)
    srcs = [0, 150, 299, 10, 149]
    for rep in range(3):
        d = g.mssp(srcs)
        for i, s in enumerate(srcs):
            assert np.array_equal(d[i], np.abs(pre - pre[s])), (rep, i)
    assert g.stats()["device_error"] == 0
    g.close()
