"""The allocation-free BFS entry point, gbf_bfs_noalloc.

It serves callers that cannot allocate device memory (their device memory is
owned by another allocator, or cudaMalloc's possible device-wide
synchronisation is not acceptable where they run).  Its results must match
the regular gbf_bfs: distances bit-exact, parents a valid BFS tree.  Two calls
in a row check that the shared fixed scratch array is reset correctly between
calls; graphs at the size limits (2^20 vertices; an RMAT graph just under
2^25 arcs) fill every region of that array.  A malformed CSR and buffers
shorter than n or m are rejected.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import graphgen as G
import oracle

pytestmark = pytest.mark.gpu


def test_bfs_noalloc_matches_gbf_bfs_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_05208_gb300 as gb

    dev = torch.device("cuda")
    for scale, seed in ((14, 21), (16, 22)):
        csr = G.rmat(scale, 16, seed=seed)
        off = torch.from_numpy(csr.off.view(np.int32).copy()).to(dev)
        tgt = torch.from_numpy(csr.tgt.copy()).to(dev)
        ref_graph = gb.Graph(csr)
        srcs = [G.max_degree_vertex(csr), int(G.sources(csr, 1, seed=seed)[0])]
        for s in srcs:                                  # two calls in a row
            dist = torch.full((csr.n,), -7, dtype=torch.int32, device=dev)
            par = torch.full((csr.n,), -7, dtype=torch.int32, device=dev)
            gb.gbf_bfs_noalloc(csr.n, csr.m, off, tgt, s, dist, par)
            d_ref, _ = ref_graph.bfs(s)
            d = dist.cpu().numpy()
            assert np.array_equal(d, d_ref)
            ok, v, why = oracle.check_bfs(csr, s, d, par.cpu().numpy())
            assert ok, (v, why)
        ref_graph.close()


def test_bfs_noalloc_rejects_oversize():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_05208_gb300 as gb

    dev = torch.device("cuda")
    off = torch.zeros(4, dtype=torch.int32, device=dev)
    tgt = torch.zeros(4, dtype=torch.int32, device=dev)
    dist = torch.zeros(4, dtype=torch.int32, device=dev)
    with pytest.raises(gb.GbfError) as e:
        gb.gbf_bfs_noalloc((1 << 20) + 1, 0, off, tgt, 0, dist)
    assert e.value.status == 1
    with pytest.raises(gb.GbfError) as e:
        gb.gbf_bfs_noalloc(3, (1 << 25) + 1, off, tgt, 0, dist)
    assert e.value.status == 1


def _dev_csr(torch, csr, dev):
    off = torch.from_numpy(csr.off.view(np.int32).copy()).to(dev)
    tgt = torch.from_numpy(csr.tgt.copy()).to(dev)
    return off, tgt


@pytest.mark.parametrize("kind", ["grid1024", "rmat20"])
def test_bfs_noalloc_at_the_size_limits(kind):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_05208_gb300 as gb

    dev = torch.device("cuda")
    csr = G.grid(1024, 1024, 0.1, seed=1) if kind == "grid1024" else G.rmat(20, 16, seed=23)
    assert csr.n == 1 << 20 and csr.m < 1 << 25
    off, tgt = _dev_csr(torch, csr, dev)
    ref_graph = gb.Graph(csr)
    srcs = [0, int(G.sources(csr, 1, seed=5)[0])]
    for s in srcs:                                      # two calls in a row
        dist = torch.full((csr.n,), -7, dtype=torch.int32, device=dev)
        par = torch.full((csr.n,), -7, dtype=torch.int32, device=dev)
        gb.gbf_bfs_noalloc(csr.n, csr.m, off, tgt, s, dist, par)
        d_ref, _ = ref_graph.bfs(s)
        d = dist.cpu().numpy()
        assert np.array_equal(d, d_ref)
        ok, v, why = oracle.check_bfs(csr, s, d, par.cpu().numpy())
        assert ok, (v, why)
    ref_graph.close()


def test_bfs_noalloc_rejects_malformed_csr_and_short_buffers():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_05208_gb300 as gb

    dev = torch.device("cuda")
    csr = G.rmat(10, 8, seed=3)
    off, tgt = _dev_csr(torch, csr, dev)
    dist = torch.empty(csr.n, dtype=torch.int32, device=dev)
    # m smaller than off[n]: rejected on the device before the search
    with pytest.raises(gb.GbfError) as e:
        gb.gbf_bfs_noalloc(csr.n, csr.m - 1, off, tgt, 0, dist)
    assert e.value.status == 1
    # a target outside [0, n)
    bad = tgt.clone()
    bad[csr.m // 2] = csr.n + 5
    with pytest.raises(gb.GbfError) as e:
        gb.gbf_bfs_noalloc(csr.n, csr.m, off, bad, 0, dist)
    assert e.value.status == 1
    # decreasing offsets
    boff = off.clone()
    boff[csr.n // 2] = int(csr.m)
    with pytest.raises(gb.GbfError) as e:
        gb.gbf_bfs_noalloc(csr.n, csr.m, boff, tgt, 0, dist)
    assert e.value.status == 1
    # buffers shorter than n / m are refused by the binding, before any launch
    with pytest.raises(ValueError):
        gb.gbf_bfs_noalloc(csr.n, csr.m, off[: csr.n], tgt, 0, dist)
    with pytest.raises(ValueError):
        gb.gbf_bfs_noalloc(csr.n, csr.m, off, tgt[:-1], 0, dist)
    with pytest.raises(ValueError):
        gb.gbf_bfs_noalloc(csr.n, csr.m, off, tgt, 0, dist[:-1])
    # the same buffers, well formed, still give the right answer afterwards
    gb.gbf_bfs_noalloc(csr.n, csr.m, off, tgt, 0, dist)
    ref, _ = oracle.bfs(csr, 0)
    assert np.array_equal(dist.cpu().numpy(), ref)
