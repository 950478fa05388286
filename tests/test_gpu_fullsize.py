"""GPU parity at the full sizes of the benchmark's configurations, in the
launch configuration bench.py times (its graph and source generators, default
options; the autotuned options for the multi-source BFS).

Where the oracle finishes in seconds the comparison is element by element on
every vertex (wBFS and its neighbours at RMAT scale 22, the grid, one RMAT
scale-26 BFS, four lanes of the multi-source BFS).  Elsewhere the oracle's
certificates check every vertex: for BFS, D[src] = 0, no arc joins levels more
than one apart or a reached and an unreached vertex, and every reached vertex
has a neighbour one level closer; for positive weights, D[src] = 0, every arc
satisfies D[v] <= D[u] + w and every reached vertex has a tight arc.  Either
set of conditions holds for the exact distances and for nothing else.
"""
import numpy as np
import pytest

import bench
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


@pytest.fixture(scope="module")
def rmat22(gb):
    wl = bench.WORKLOADS["wbfs-rmat22"]
    csr = bench.make_graph(wl)
    g = gb.Graph(csr, validate=gb.VALIDATE_BASIC)
    yield csr, g, bench.make_sources(csr, wl)
    g.close()


def _device_run(gb, fn, n, dtype=None):
    import torch
    out = torch.empty(n, dtype=dtype or torch.int32, device="cuda")
    fn(out)
    return out.cpu().numpy()


def test_wbfs_rmat22_all_sources(gb, rmat22):
    """The default workload: 8 seeded sources, every distance against Dijkstra."""
    csr, g, srcs = rmat22
    for s in srcs:
        d = _device_run(gb, lambda o: gb.gbf_wbfs(g.h, int(s), o), csr.n)
        gb.gbf_wait(g.h)
        assert np.array_equal(d, oracle.dijkstra(csr, int(s))), int(s)


def test_rmat22_next_rows(gb, rmat22):
    """Bellman-Ford, widest path, Δ-stepping, betweenness and coreness on the
    same scale-22 graph (one source each; the k-core covers every vertex)."""
    csr, g, srcs = rmat22
    s = int(srcs[0])
    ref = oracle.dijkstra(csr, s)
    assert np.array_equal(_device_run(gb, lambda o: gb.gbf_bellman_ford(g.h, s, o), csr.n), ref)
    assert np.array_equal(_device_run(gb, lambda o: gb.gbf_delta_stepping(g.h, s, 4, o), csr.n), ref)
    assert np.array_equal(_device_run(gb, lambda o: gb.gbf_widest_path(g.h, s, o), csr.n),
                          oracle.widest_path(csr, s))
    import torch
    bc = _device_run(gb, lambda o: gb.gbf_betweenness(g.h, s, o), csr.n, torch.float64)
    np.testing.assert_allclose(bc, oracle.betweenness(csr, s), rtol=1e-9, atol=1e-9)
    core = _device_run(gb, lambda o: gb.gbf_kcore(g.h, o), csr.n)
    gb.gbf_wait(g.h)
    assert np.array_equal(core, oracle.coreness(csr))


def test_grid_bfs_wbfs_delta(gb):
    """The 4096 x 4096 grid with 10 % of edges deleted: BFS (with parents),
    wBFS and Δ-stepping from vertex 0 and the seeded sources."""
    wl = bench.WORKLOADS["wbfs-grid"]
    csr = bench.make_graph(wl)
    g = gb.Graph(csr, validate=gb.VALIDATE_BASIC)
    for s in bench.make_sources(csr, wl)[:2]:
        s = int(s)
        d, p = g.bfs(s)
        ref, _ = oracle.bfs(csr, s, parents=False)
        assert np.array_equal(d, ref), s
        ok, v, why = oracle.check_bfs(csr, s, d, p)
        assert ok, (s, v, why)
        ref = oracle.dijkstra(csr, s)
        assert np.array_equal(g.wbfs(s), ref), s
        assert np.array_equal(g.delta_stepping(s, 64), ref), s
    g.close()


def test_msbfs_rmat24_autotuned(gb):
    """64 sources in one launch with the autotuned knobs: every one of the 64
    lanes against the oracle's BFS from its source, element by element (the
    oracle queries run one per host thread; its C calls release the GIL)."""
    import concurrent.futures as cf
    import os

    import torch
    wl = bench.WORKLOADS["msbfs-rmat24"]
    csr = bench.make_graph(wl)
    srcs = bench.make_sources(csr, wl)
    g = gb.Graph(csr, validate=gb.VALIDATE_BASIC)
    opt = gb.gbf_autotune(g.h, gb.TUNE_MSBFS)
    out = torch.empty((len(srcs), csr.n), dtype=torch.int32, device="cuda")
    gb.gbf_msbfs(g.h, srcs, out, opt)
    st = gb.gbf_wait(g.h)
    assert st["device_error"] == 0
    d = out.cpu().numpy()
    g.close()

    def lane_ok(i):
        ref, _ = oracle.bfs(csr, int(srcs[i]), parents=False)
        return i, bool(np.array_equal(d[i], ref))
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        res = dict(ex.map(lane_ok, range(len(srcs))))
    bad = [i for i, ok in res.items() if not ok]
    assert len(res) == 64 and not bad, bad


def test_rmat26_bfs_and_wbfs(gb):
    """RMAT scale 26 (2.15 B arcs): one BFS against the oracle on every vertex
    plus the parent invariants, a second source against the BFS certificate,
    one wBFS against the shortest-path certificate."""
    wl = bench.WORKLOADS["bfs-rmat26"]
    csr = bench.make_graph(wl)
    G.add_weights(csr, 1, 22, seed=2)
    srcs = bench.make_sources(csr, wl)
    g = gb.Graph(csr, validate=gb.VALIDATE_BASIC)
    for i, s in enumerate(srcs[:2]):
        s = int(s)
        d, p = g.bfs(s)
        ok, v, why = oracle.check_bfs(csr, s, d, p)
        assert ok, (s, v, why)
        if i == 0:
            ref, _ = oracle.bfs(csr, s, parents=False)
            assert np.array_equal(d, ref)
    s = int(srcs[0])
    dw = g.wbfs(s)
    ok, v, why = oracle.check_sssp(csr, s, dw)
    assert ok, (s, v, why)
    g.close()
