"""GPU parity: BFS and weighted BFS through the C ABI against the oracle.

Distances are compared element by element and must be bit-exact (integer
work).  Parents are not unique (test-and-set winners, Alg. 1), so they are
checked by the oracle's BFS-tree invariants.  Inputs are seeded synthetic
graphs at sizes the oracle finishes in seconds that still span many chunks
of the blocked edgeMap and ragged tails.
"""
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


def _bfs_parity(gb, csr, srcs, opts=(None,)):
    g = gb.Graph(csr, validate=gb.VALIDATE_BASIC | gb.VALIDATE_SYMMETRIC)
    for s in srcs:
        ref, _ = oracle.bfs(csr, int(s), parents=False)
        for o in opts:
            d, p = g.bfs(int(s), opt=o)
            assert np.array_equal(d, ref), (csr.name, s, o and o.pull_divisor)
            ok, v, why = oracle.check_bfs(csr, int(s), d, p)
            assert ok, (csr.name, s, v, why)
    g.close()


def _wbfs_parity(gb, csr, srcs, opts=(None,)):
    """Every option set bit-exact against Dijkstra; an option set with the
    dense switch on must have run at least one dense round on the graph."""
    g = gb.Graph(csr, validate=gb.VALIDATE_BASIC | gb.VALIDATE_SYMMETRIC)
    dense_rounds = {}
    for s in srcs:
        ref = oracle.dijkstra(csr, int(s))
        for i, o in enumerate(opts):
            d = g.wbfs(int(s), opt=o)
            assert np.array_equal(d, ref), (csr.name, s, o and (o.bucket_window, o.dense_wbfs))
            if o is not None and o.dense_wbfs:
                dense_rounds[i] = dense_rounds.get(i, 0) + g.stats()["pull_rounds"]
    g.close()
    for i, r in dense_rounds.items():
        assert r > 0, f"dense_wbfs option set {i} never ran a dense round on {csr.name}"


# -------------------------------------------------------------- closed forms
def test_bfs_closed_forms(gb):
    for csr, srcs in [(G.path_graph(1000), [0, 999, 500]), (G.star_graph(3000), [0, 7]),
                      (G.complete_graph(120), [0, 119]), (G.grid_graph(50, 70), [0, 1234, 3499]),
                      (G.csr_from_edges(10, [(0, 1), (1, 2), (5, 6), (6, 7)]), [1, 5, 9])]:
        _bfs_parity(gb, csr, srcs, opts=(None, gb.gbf_options_default(pull_divisor=-1),
                                         gb.gbf_options_default(pull_divisor=1000000)))


def test_bfs_isolated_source(gb):
    csr = G.csr_from_edges(70, [(1, 2), (2, 3)])
    g = gb.Graph(csr)
    d, p = g.bfs(0)
    assert d[0] == 0 and p[0] == 0 and np.all(d[1:] == INF) and np.all(p[1:] == -1)


def test_bfs_single_vertex(gb):
    csr = G.csr_from_edges(1, np.zeros((0, 2), dtype=np.int64))
    g = gb.Graph(csr)
    d, p = g.bfs(0)
    assert d.tolist() == [0] and p.tolist() == [0]


# ------------------------------------------------------------------ RMAT
@pytest.mark.parametrize("scale,ef", [(10, 4), (13, 16), (16, 16)])
def test_bfs_rmat(gb, scale, ef):
    csr = G.rmat(scale, ef, seed=scale)
    srcs = list(G.sources(csr, 4, seed=3)) + [G.max_degree_vertex(csr)]
    opts = (None,
            gb.gbf_options_default(pull_divisor=-1),                 # push only
            gb.gbf_options_default(pull_divisor=2),                  # late pull
            gb.gbf_options_default(pull_divisor=10000, pull_serial=1),  # early pull, warp scans
            gb.gbf_options_default(block=1024, heavy_cutoff=4096),
            gb.gbf_options_default(block=128, heavy_cutoff=256, ctas=7))
    _bfs_parity(gb, csr, srcs, opts)


def test_bfs_config_rmat16_max_degree_source(gb):
    """RMAT scale 16, edge factor 16, max-degree source: distances + parents."""
    csr = G.rmat(16, 16, seed=1)
    s = G.max_degree_vertex(csr)
    g = gb.Graph(csr)
    ref, _ = oracle.bfs(csr, s)
    for _ in range(5):   # repeated runs catch racy compaction
        d, p = g.bfs(s)
        assert np.array_equal(d, ref)
        assert oracle.check_bfs(csr, s, d, p)[0]
    st = g.stats()
    assert st["device_error"] == 0


def test_bfs_repeated_block1024_conversions(gb):
    """Block 1024 with dense levels followed by sparse ones (bitmap -> queue
    conversions) and one CTA doing most of a dense level, repeated: this
    caught warps disagreeing on whether to flush the shared staging area."""
    csr = G.rmat(13, 16, seed=13)
    srcs = list(G.sources(csr, 4, seed=3)) + [G.max_degree_vertex(csr)]
    refs = {int(s): oracle.bfs(csr, int(s), parents=False)[0] for s in srcs}
    g = gb.Graph(csr)
    for blk, hc in ((1024, 0), (1024, 4096), (512, 0)):
        opt = gb.gbf_options_default(block=blk, heavy_cutoff=hc)
        for _ in range(20):
            for s in srcs:
                d, _ = g.bfs(int(s), opt=opt)
                assert np.array_equal(d, refs[int(s)]), (blk, hc, int(s))
    # a shape whose shared memory does not fit one CTA is refused, not run
    with pytest.raises(gb.GbfError) as e:
        g.bfs(int(srcs[0]), opt=gb.gbf_options_default(block=1024, heavy_cutoff=16384))
    assert e.value.status == 1
    d, _ = g.bfs(int(srcs[0]))
    assert np.array_equal(d, refs[int(srcs[0])])
    g.close()


def test_bfs_host_batch_matches_single_queries(gb):
    """gbf_bfs_host_batch (each query's read-back running while the next one
    searches, two device result buffers in turn) gives every row as gbf_bfs
    does, for 1, 2, 3 and 5 sources, with and without parents, into pinned
    and pageable host memory; bad arguments are refused."""
    torch = pytest.importorskip("torch")
    csr = G.rmat(14, 16, seed=81)
    g = gb.Graph(csr, validate=gb.VALIDATE_BASIC | gb.VALIDATE_SYMMETRIC)
    srcs = G.sources(csr, 5, seed=82)
    refs = [oracle.bfs(csr, int(s), parents=False)[0] for s in srcs]
    for k in (1, 2, 3, 5):
        for pinned in (True, False):
            def rows():
                if pinned:
                    return torch.empty((k, csr.n), dtype=torch.int32, pin_memory=True).numpy()
                return np.empty((k, csr.n), dtype=np.int32)
            d, p = rows(), rows()
            gb.gbf_bfs_host_batch(g.h, srcs[:k], d, p)
            for i in range(k):
                assert np.array_equal(d[i], refs[i]), (k, pinned, i)
                ok, v, why = oracle.check_bfs(csr, int(srcs[i]), d[i], p[i])
                assert ok, (k, pinned, i, v, why)
            d2 = rows()
            gb.gbf_bfs_host_batch(g.h, srcs[:k], d2)
            assert np.array_equal(d2, d)
    with pytest.raises(ValueError):
        gb.gbf_bfs_host_batch(g.h, srcs[:2], np.empty((1, csr.n), dtype=np.int32))
    with pytest.raises(gb.GbfError):
        gb.gbf_bfs_host_batch(g.h, np.array([csr.n], dtype=np.int32),
                              np.empty((1, csr.n), dtype=np.int32))
    g.close()


def test_bfs_grid_deleted_edges(gb):
    csr = G.grid(200, 300, 0.1, seed=7)
    _bfs_parity(gb, csr, [0, 123, 59999], opts=(None, gb.gbf_options_default(ctas=3)))


def test_bfs_repeat_determinism_tiny(gb):
    # tiny graphs, many seeds: exact against Floyd-Warshall-pinned oracle
    g_list = [G.random_small(2 + (s % 60), [0.05, 0.15, 0.4][s % 3], s) for s in range(60)]
    for csr in g_list:
        _bfs_parity(gb, csr, [0, csr.n - 1])


# --------------------------------------------------------------------- wBFS
def test_wbfs_closed_forms(gb):
    n = 500
    wpath = (np.arange(1, n) % 7 + 1)
    for csr, srcs in [(G.path_graph(n, weights=wpath), [0, 250, 499]),
                      (G.grid_graph(40, 50, weight=5), [0, 777]),
                      (G.csr_from_edges(10, [(0, 1), (1, 2), (5, 6)], [3, 4, 5]), [1, 5, 9])]:
        _wbfs_parity(gb, csr, srcs, opts=(None, gb.gbf_options_default(bucket_window=1),
                                          gb.gbf_options_default(bucket_window=2)))


def test_wbfs_golden(gb):
    edges = [(0, 1), (0, 2), (2, 1), (1, 3), (2, 3), (2, 4), (3, 4), (3, 5), (4, 5), (6, 7)]
    ws = [4, 1, 2, 5, 8, 10, 2, 6, 3, 1]
    csr = G.csr_from_edges(8, edges, ws)
    g = gb.Graph(csr)
    assert g.wbfs(0).tolist() == [0, 3, 1, 8, 10, 13, INF, INF]


@pytest.mark.parametrize("scale", [10, 14, 16])
def test_wbfs_rmat(gb, scale):
    csr = G.add_weights(G.rmat(scale, 16, seed=scale + 1), 1, 22, seed=2)
    srcs = G.sources(csr, 3, seed=3)
    opts = (None,
            gb.gbf_options_default(bucket_window=1),
            gb.gbf_options_default(bucket_window=2),
            gb.gbf_options_default(bucket_window=128),
            gb.gbf_options_default(dense_wbfs=1, pull_divisor=50),
            gb.gbf_options_default(block=512, heavy_cutoff=2048, ctas=11))
    _wbfs_parity(gb, csr, srcs, opts)


def test_wbfs_unit_weights_equal_bfs(gb):
    csr = G.rmat(14, 8, seed=4)
    csr.w = np.ones(csr.m, dtype=np.uint32)
    g = gb.Graph(csr)
    for s in G.sources(csr, 3, seed=5):
        d, _ = g.bfs(int(s))
        assert np.array_equal(g.wbfs(int(s)), d)


def test_wbfs_grid(gb):
    csr = G.add_weights(G.grid(120, 150, 0.1, seed=3), 1, 16, seed=4)
    _wbfs_parity(gb, csr, [0, 9000], opts=(None, gb.gbf_options_default(bucket_window=4)))


def test_wbfs_cta_local_rounds(gb):
    """With local_arcs set, small buckets are expanded by one CTA alone
    (local_rounds > 0); the distances equal Dijkstra's with the mode off (the
    default), with an arc limit so small that runs start and stop every few
    rounds, and with the largest limit, on a graph of few hubs and on a
    high-diameter grid."""
    for csr in (G.add_weights(G.rmat(14, 16, seed=61), 1, 22, seed=62),
                G.add_weights(G.grid(120, 130, 0.1, seed=63), 1, 16, seed=64)):
        g = gb.Graph(csr)
        for s in G.sources(csr, 2, seed=65):
            ref = oracle.dijkstra(csr, int(s))
            local = {}
            for la in (0, -1, 3, 4096, (1 << 20) - 1):
                d = g.wbfs(int(s), opt=gb.gbf_options_default(local_arcs=la))
                st = g.stats()
                assert np.array_equal(d, ref), (csr.name, int(s), la)
                assert st["device_error"] == 0
                local[la] = st["local_rounds"]
            assert local[0] == 0 and local[-1] == 0, (csr.name, local)
            assert local[4096] > 0 and local[(1 << 20) - 1] > 0, (csr.name, local)
        g.close()


def test_wbfs_tiny_many(gb):
    for s in range(40):
        csr = G.random_small(2 + (s % 60), [0.05, 0.15, 0.4][s % 3], 100 + s, w_hi=[2, 9, 30][s % 3])
        _wbfs_parity(gb, csr, [0, csr.n - 1], opts=(None, gb.gbf_options_default(bucket_window=1)))


# ------------------------------------------------------- errors and faults
def test_invalid_inputs(gb):
    csr = G.path_graph(10)
    g = gb.Graph(csr)
    d = np.empty(10, dtype=np.int32)
    with pytest.raises(gb.GbfError) as e:
        gb.gbf_bfs(g.h, 10, d)
    assert e.value.status == 1
    with pytest.raises(gb.GbfError) as e:
        gb.gbf_wbfs(g.h, 0, d)   # unweighted graph
    assert e.value.status == 1
    bad = G.path_graph(10)
    tgt = bad.tgt.copy(); tgt[3] = 99
    with pytest.raises(gb.GbfError):
        gb.Graph(n=10, off=bad.off, tgt=tgt)
    tgt = bad.tgt.copy(); tgt[0] = 0   # self-loop at vertex 0
    with pytest.raises(gb.GbfError):
        gb.Graph(n=10, off=bad.off, tgt=tgt)
    wcsr = G.path_graph(10, weights=np.ones(9))
    w = wcsr.w.copy(); w[2] = 0
    with pytest.raises(gb.GbfError):
        gb.Graph(n=10, off=wcsr.off, tgt=wcsr.tgt, w=w)
    asym = G.csr_from_edges(4, [(0, 1), (1, 2)])
    t2 = asym.tgt.copy(); t2[-1] = 0   # vertex 2's arc now points at 0: not symmetric
    with pytest.raises(gb.GbfError):
        gb.Graph(n=4, off=asym.off, tgt=t2, validate=gb.VALIDATE_SYMMETRIC)


def test_overflow_rejected(gb):
    n = 3
    csr = G.csr_from_edges(n, [(0, 1), (1, 2)], [2**30, 2**30])
    with pytest.raises(gb.GbfError) as e:
        gb.Graph(csr)
    assert e.value.status == 5


def test_injected_timeout_then_recovers(gb):
    csr = G.add_weights(G.rmat(12, 8, seed=2), 1, 22, seed=1)
    g = gb.Graph(csr)
    d = np.empty(csr.n, dtype=np.int32)
    for fn in (lambda o: gb.gbf_bfs(g.h, 0, d, None, o), lambda o: gb.gbf_wbfs(g.h, 0, d, o)):
        with pytest.raises(gb.GbfError) as e:
            fn(gb.gbf_options_default(inject_wait=1, spin_cap_us=20000))
        assert e.value.status == 4
    s = int(G.sources(csr, 1)[0])
    ref, _ = oracle.bfs(csr, s)
    assert np.array_equal(g.bfs(s)[0], ref)
    assert np.array_equal(g.wbfs(s), oracle.dijkstra(csr, s))


def test_device_buffers_and_streams(gb):
    import torch
    csr = G.add_weights(G.rmat(13, 16, seed=6), 1, 22, seed=7)
    dev = torch.device("cuda")
    off = torch.from_numpy(csr.off.view(np.int32).copy()).to(dev)
    tgt = torch.from_numpy(csr.tgt.copy()).to(dev)
    w = torch.from_numpy(csr.w.view(np.int32).copy()).to(dev)
    st = torch.cuda.Stream()
    h = gb.gbf_graph_create(csr.n, off, tgt, w, gb.VALIDATE_BASIC, st)
    dist = torch.empty(csr.n, dtype=torch.int32, device=dev)
    par = torch.empty(csr.n, dtype=torch.int32, device=dev)
    s = int(G.sources(csr, 1, seed=9)[0])
    gb.gbf_bfs(h, s, dist, par, None, st)
    stats = gb.gbf_wait(h, st)
    ref, _ = oracle.bfs(csr, s)
    assert np.array_equal(dist.cpu().numpy(), ref)
    assert oracle.check_bfs(csr, s, dist.cpu().numpy(), par.cpu().numpy())[0]
    assert stats["rounds"] >= 1 and stats["vertices_reached"] == int((ref != INF).sum())
    gb.gbf_wbfs(h, s, dist, None, st)
    gb.gbf_wait(h, st)
    assert np.array_equal(dist.cpu().numpy(), oracle.dijkstra(csr, s))
    gb.gbf_graph_destroy(h)


def test_round_trace(gb):
    csr = G.add_weights(G.rmat(14, 16, seed=12), 1, 22, seed=13)
    g = gb.Graph(csr)
    s = int(G.sources(csr, 1, seed=14)[0])
    d, _ = g.bfs(s)
    tr = gb.gbf_trace(g.h)
    st = g.stats()
    assert len(tr) == st["rounds"] and len(tr) >= int(d[d != INF].max())
    assert [r[0] for r in tr] == list(range(1, len(tr) + 1))
    assert all(b[4] >= a[4] for a, b in zip(tr, tr[1:]))
    assert {r[1] for r in tr} <= {1, 2, 4, 6, 7}
    g.wbfs(s)
    tr = gb.gbf_trace(g.h)
    assert len(tr) == g.stats()["rounds"] > 0
    assert {r[1] for r in tr} <= {1, 2, 3}
    g.wbfs(s, opt=gb.gbf_options_default(local_arcs=4096))
    tr = gb.gbf_trace(g.h)
    assert len(tr) == g.stats()["rounds"] > 0
    assert [r[0] for r in tr] == list(range(1, len(tr) + 1))
    assert {r[1] for r in tr} <= {1, 2, 3, 8}
    assert sum(r[1] == 8 for r in tr) == g.stats()["local_rounds"] > 0


def test_sparse_graphs_default_to_half_the_sms(gb):
    """With ctas left at 0, a graph with fewer than 8 arcs per vertex runs on
    half as many CTAs as SMs; a denser graph gets every resident CTA.  The
    distances do not depend on it."""
    torch = pytest.importorskip("torch")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sparse = G.add_weights(G.grid(60, 70, 0.1, seed=3), 1, 16, seed=4)
    dense = G.add_weights(G.rmat(12, 16, seed=5), 1, 22, seed=6)
    for csr, expect_half in ((sparse, True), (dense, False)):
        g = gb.Graph(csr)
        s = int(G.sources(csr, 1, seed=7)[0])
        d = torch.empty(csr.n, dtype=torch.int32, device="cuda")
        for run in (lambda: gb.gbf_bfs(g.h, s, d), lambda: gb.gbf_wbfs(g.h, s, d),
                    lambda: gb.gbf_delta_stepping(g.h, s, 4, d)):
            run()
            st = gb.gbf_wait(g.h)
            if expect_half:
                assert st["grid_ctas"] == max(sms // 2, 1), csr.name
            else:
                assert st["grid_ctas"] > sms // 2, csr.name
        assert np.array_equal(d.cpu().numpy(), oracle.dijkstra(csr, s))
        g.close()
