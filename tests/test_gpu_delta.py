"""GPU parity: Δ-stepping (the bucket coarsening of wBFS that the SSSP
discussion of §7 compares with) through the C ABI against the oracle's
Dijkstra.  Distances are unique, so every Δ must reproduce them bit-exactly;
Δ = 1 is the exact wBFS of Alg. 3.  Small bucket windows force the overflow
bucket and its refills; the grid forces many re-expansions inside a bucket."""
import numpy as np
import pytest

import graphgen as G
import oracle

pytestmark = pytest.mark.gpu

INF = oracle.INF
DELTAS = (1, 2, 4, 8, 32, 1024)


@pytest.fixture(scope="module")
def gb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_05208_gb300 as gb
    return gb


def _parity(gb, csr, srcs, deltas=DELTAS, opts=(None,)):
    g = gb.Graph(csr, validate=gb.VALIDATE_BASIC | gb.VALIDATE_SYMMETRIC)
    for s in srcs:
        ref = oracle.dijkstra(csr, int(s))
        for dl in deltas:
            for o in opts:
                d = g.delta_stepping(int(s), dl, opt=o)
                assert np.array_equal(d, ref), (csr.name, s, dl, o and o.bucket_window)
    g.close()


def test_closed_forms(gb):
    n = 500
    wpath = (np.arange(1, n) % 7 + 1)
    for csr, srcs in [(G.path_graph(n, weights=wpath), [0, 250, 499]),
                      (G.grid_graph(40, 50, weight=5), [0, 777]),
                      (G.star_graph(3000), [0, 5]),
                      (G.csr_from_edges(10, [(0, 1), (1, 2), (5, 6)], [3, 4, 5]), [1, 5, 9])]:
        if csr.w is None:
            csr = G.add_weights(csr, 1, 22, seed=7)
        _parity(gb, csr, srcs, opts=(None, gb.gbf_options_default(bucket_window=1),
                                     gb.gbf_options_default(bucket_window=2)))


def test_golden(gb):
    edges = [(0, 1), (0, 2), (2, 1), (1, 3), (2, 3), (2, 4), (3, 4), (3, 5), (4, 5), (6, 7)]
    ws = [4, 1, 2, 5, 8, 10, 2, 6, 3, 1]
    g = gb.Graph(G.csr_from_edges(8, edges, ws))
    for dl in DELTAS:
        assert g.delta_stepping(0, dl).tolist() == [0, 3, 1, 8, 10, 13, INF, INF]


@pytest.mark.parametrize("scale", [10, 14, 16])
def test_rmat(gb, scale):
    csr = G.add_weights(G.rmat(scale, 16, seed=scale + 1), 1, 22, seed=2)
    srcs = G.sources(csr, 3, seed=3)
    _parity(gb, csr, srcs, opts=(None, gb.gbf_options_default(bucket_window=2),
                                 gb.gbf_options_default(block=512, heavy_cutoff=2048, ctas=11)))


def test_delta_one_is_wbfs(gb):
    csr = G.add_weights(G.rmat(14, 16, seed=9), 1, 22, seed=2)
    g = gb.Graph(csr)
    for s in G.sources(csr, 3, seed=4):
        assert np.array_equal(g.delta_stepping(int(s), 1), g.wbfs(int(s)))


def test_grid(gb):
    csr = G.add_weights(G.grid(120, 150, 0.1, seed=3), 1, 16, seed=4)
    _parity(gb, csr, [0, 9000], opts=(None, gb.gbf_options_default(bucket_window=3)))


def test_tiny_many(gb):
    for s in range(40):
        csr = G.random_small(2 + (s % 60), [0.05, 0.15, 0.4][s % 3], 100 + s, w_hi=[2, 9, 30][s % 3])
        _parity(gb, csr, [0, csr.n - 1], deltas=(2, 8, 64),
                opts=(None, gb.gbf_options_default(bucket_window=1)))


def test_device_buffers_and_stream(gb):
    torch = pytest.importorskip("torch")
    csr = G.add_weights(G.rmat(12, 16, seed=5), 1, 22, seed=6)
    g = gb.Graph(csr)
    s = int(G.sources(csr, 1, seed=7)[0])
    ref = oracle.dijkstra(csr, s)
    st = torch.cuda.Stream()
    d = torch.empty(csr.n, dtype=torch.int32, device="cuda")
    gb.gbf_delta_stepping(g.h, s, 8, d, None, st)
    stats = gb.gbf_wait(g.h, st)
    assert stats["device_error"] == 0
    assert np.array_equal(d.cpu().numpy(), ref)


def test_invalid(gb):
    csr = G.add_weights(G.path_graph(10), 1, 5, seed=1)
    g = gb.Graph(csr)
    d = np.empty(10, dtype=np.int32)
    for bad in (0, -4, 3, 12, 1 << 21):
        with pytest.raises(gb.GbfError) as e:
            gb.gbf_delta_stepping(g.h, 0, bad, d)
        assert e.value.status == 1
    with pytest.raises(gb.GbfError):
        gb.gbf_delta_stepping(g.h, 10, 4, d)
    unweighted = gb.Graph(G.path_graph(10))
    with pytest.raises(gb.GbfError):
        gb.gbf_delta_stepping(unweighted.h, 0, 4, d)
    # the graph stays usable
    assert np.array_equal(g.delta_stepping(3, 4), oracle.dijkstra(csr, 3))
