"""GPU parity for the multi-source BFS (64-bit lanes, and 8-bit lanes for 2..8
sources): lane i must equal a BFS from srcs[i] (the oracle's, bit-exact), for
every lane, on seeded graphs, with duplicate and isolated sources, both
directions of edgeMap, and CUDA-graph replays with new sources, new output
buffers and alternating lane widths."""
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


def _check(gb, csr, srcs, opts=(None,)):
    g = gb.Graph(csr)
    ref = oracle.msbfs(csr, srcs)
    for o in opts:
        d = g.msbfs(srcs, opt=o)
        assert d.shape == (len(srcs), csr.n)
        bad = np.flatnonzero((d != ref).any(axis=1))
        assert bad.size == 0, (csr.name, o and o.pull_divisor, bad[:5])
    g.close()


@pytest.mark.parametrize("scale,ef", [(10, 8), (14, 16), (16, 16)])
def test_msbfs_rmat_64_lanes(gb, scale, ef):
    csr = G.rmat(scale, ef, seed=30 + scale)
    srcs = G.sources(csr, 64, seed=4)
    _check(gb, csr, srcs, opts=(None, gb.gbf_options_default(pull_divisor=-1),
                                gb.gbf_options_default(pull_divisor=1000),
                                gb.gbf_options_default(block=512, heavy_cutoff=1024, ctas=5)))


def test_msbfs_k_sizes_duplicates_isolated(gb):
    csr = G.rmat(12, 8, seed=7)
    deg = csr.degrees()
    iso = np.flatnonzero(deg == 0)
    s = list(G.sources(csr, 40, seed=9))
    s[3] = s[7]                      # duplicate lane
    if iso.size:
        s[5] = int(iso[0])           # an isolated source
    for k in (1, 2, 31, 32, 33, 40):
        _check(gb, csr, np.array(s[:k], dtype=np.int32))


@pytest.mark.parametrize("scale", [12, 16])
def test_msbfs_narrow_lanes(gb, scale):
    """2..8 sources run with 8-bit lanes (four vertices per atomic word); 9 is
    the first batch with 64-bit lanes."""
    csr = G.rmat(scale, 16, seed=50 + scale)
    s = list(G.sources(csr, 9, seed=51))
    s[2] = s[1]                      # duplicate lane
    opts = (None, gb.gbf_options_default(pull_divisor=-1),
            gb.gbf_options_default(pull_divisor=1000),
            gb.gbf_options_default(block=128, heavy_cutoff=256, ctas=7))
    for k in (2, 3, 4, 7, 8, 9):
        _check(gb, csr, np.array(s[:k], dtype=np.int32), opts=opts)


def test_msbfs_replay_alternating_widths(gb):
    import torch
    csr = G.rmat(13, 16, seed=12)
    g = gb.Graph(csr)
    for rep, k in enumerate((4, 64, 4, 8, 64, 2)):
        srcs = G.sources(csr, k, seed=200 + rep)
        out = torch.full((k, csr.n), -5, dtype=torch.int32, device="cuda")
        gb.gbf_msbfs(g.h, srcs, out)
        assert gb.gbf_wait(g.h)["device_error"] == 0
        assert np.array_equal(out.cpu().numpy(), oracle.msbfs(csr, srcs)), (rep, k)
    g.close()


def test_msbfs_grid_and_paths(gb):
    _check(gb, G.grid(60, 70, 0.1, seed=3), np.array([0, 100, 4199, 2000], dtype=np.int32))
    _check(gb, G.path_graph(300), np.arange(0, 300, 5, dtype=np.int32)[:60])
    comp = G.csr_from_edges(20, [(0, 1), (1, 2), (5, 6), (6, 7), (10, 11)])
    _check(gb, comp, np.arange(20, dtype=np.int32))


def test_msbfs_graph_replay_new_sources_and_buffers(gb):
    import torch
    csr = G.rmat(13, 16, seed=11)
    g = gb.Graph(csr)
    dev = torch.device("cuda")
    for rep in range(3):
        srcs = G.sources(csr, 64, seed=100 + rep)
        out = torch.full((64, csr.n), -5, dtype=torch.int32, device=dev)
        gb.gbf_msbfs(g.h, srcs, out)
        st = gb.gbf_wait(g.h)
        assert st["device_error"] == 0 and st["rounds"] >= 1
        assert np.array_equal(out.cpu().numpy(), oracle.msbfs(csr, srcs))
    g.close()


def test_msbfs_matches_single_bfs(gb):
    csr = G.rmat(14, 8, seed=21)
    g = gb.Graph(csr)
    srcs = G.sources(csr, 64, seed=22)
    d = g.msbfs(srcs)
    for i in (0, 17, 63):
        single, _ = g.bfs(int(srcs[i]))
        assert np.array_equal(d[i], single)


def test_msbfs_invalid(gb):
    csr = G.path_graph(10)
    g = gb.Graph(csr)
    out = np.empty((65, 10), dtype=np.int32)
    with pytest.raises(gb.GbfError):
        gb.gbf_msbfs(g.h, np.zeros(65, dtype=np.int32), out)
    with pytest.raises(gb.GbfError):
        gb.gbf_msbfs(g.h, np.array([10], dtype=np.int32), out[:1])


def test_autotune_results_invariant(gb, tmp_path, monkeypatch):
    """The tuner returns valid knobs, caches them, and the tuned queries give
    the same distances (knobs never change results)."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("GBF_TUNE_CACHE", str(cache))
    csr = G.add_weights(G.rmat(13, 16, seed=41), 1, 22, seed=42)
    g = gb.Graph(csr)
    srcs = G.sources(csr, 64, seed=43)
    for kind in (gb.TUNE_BFS, gb.TUNE_MSBFS, gb.TUNE_WBFS):
        o = gb.gbf_autotune(g.h, kind)
        assert o.block in (128, 256, 512, 1024)
        assert o.pull_divisor in (10, 14, 20, 28, 40)
        assert o.heavy_cutoff in (256, 512, 1024, 2048, 4096, 8192, 16384)
        o2 = gb.gbf_autotune(g.h, kind)          # cached
        assert (o2.block, o2.pull_divisor, o2.heavy_cutoff) == (o.block, o.pull_divisor,
                                                                o.heavy_cutoff)
        s = int(srcs[0])
        if kind == gb.TUNE_BFS:
            assert np.array_equal(g.bfs(s, opt=o)[0], oracle.bfs(csr, s)[0])
        elif kind == gb.TUNE_WBFS:
            assert np.array_equal(g.wbfs(s, opt=o), oracle.dijkstra(csr, s))
        else:
            assert np.array_equal(g.msbfs(srcs, opt=o), oracle.msbfs(csr, srcs))
    assert len(cache.read_text().splitlines()) == 3
