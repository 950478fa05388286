"""CPU tests of bench.py's host logic: the byte model, the traversed-edge
count, the traffic lookup keyed by the kernel's own sources, and the
multi-rank reduction (covered in test_multirank_cpu.py)."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import graphgen as G  # noqa: E402


def test_traversed_edges_counts_reached_component():
    csr = G.csr_from_edges(6, [(0, 1), (1, 2), (3, 4)])
    dist = np.array([0, 1, 2, bench.INF, bench.INF, bench.INF], dtype=np.int64)
    # reached {0, 1, 2}: degrees 1 + 2 + 1 = 4 arcs = 2 undirected edges
    assert bench.traversed_edges(csr, dist) == 2


def test_bytes_model_terms():
    st = dict(edges_scanned=10, vertices_expanded=3, relaxations=4, bucket_inserts=5,
              vertices_reached=6, pull_rounds=1, heavy_vertices=2)
    n = 64
    assert bench.bytes_model("wbfs", n, st) == 4 * n + 20 * 5 + 12 * 10 + 8 * 4 + 16 * 2
    assert bench.bytes_model("bfs", n, st) == 8 * n + n // 8 + 12 * 3 + 8 * 10 + 24 * 6 + 3 * (n // 8)
    assert bench.bytes_model("delta", n, st) == 8 * n + n // 4 + 24 * 5 + 12 * 10 + 8 * 4 + 16 * 2
    # k-core: one vertex pass per bucket; rounds count bucket passes and peeling rounds
    kst = dict(st, rounds=9, push_rounds=6)
    assert bench.bytes_model("kcore", n, kst) == 4 * n + n // 8 + 3 * (4 * n + n // 8) + 12 * 10 + 16 * n


def test_trace_summary_groups_rounds_by_kind():
    tr = [(1, 5, 10, 20, 1000, 0), (2, 1, 10, 20, 4000, 0), (3, 1, 2, 3, 5000, 0),
          (4, 5, 7, 9, 9000, 0)]
    out = bench.trace_summary(tr)
    assert out["rounds"] == 4 and out["end_us"] == 9.0
    assert out["by_kind"]["bucket"] == {"rounds": 2, "us": 5.0, "frontier": 17}
    assert out["by_kind"]["sparse"] == {"rounds": 2, "us": 4.0, "frontier": 12}


def test_kernel_source_hash_tracks_only_its_sources():
    h = {k: bench.kernel_source_hash(k) for k in bench.KERNEL_SOURCES}
    assert len(set(h.values())) == len(h)          # different file sets
    assert all(len(v) == 16 for v in h.values())
    assert h == {k: bench.kernel_source_hash(k) for k in bench.KERNEL_SOURCES}  # stable


def test_measured_traffic_needs_matching_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({
        "w": {"kernel": "wbfs_kernel", "csrc_hash": bench.kernel_source_hash("wbfs_kernel"),
              "bytes_per_launch": 123},
        "b": {"kernel": "bfs_kernel", "csrc_hash": "0" * 16, "bytes_per_launch": 456}}))
    csrc = tmp_path / "paper_1805_05208_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in {n for v in bench.KERNEL_SOURCES.values() for n in v}:
        with open(os.path.join(ROOT, "paper_1805_05208_gb300", "csrc", name), "rb") as f:
            (csrc / name).write_bytes(f.read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("w", "wbfs_kernel") == 123
    assert bench.measured_traffic("w", "bfs_kernel") is None      # other kernel
    assert bench.measured_traffic("b", "bfs_kernel") is None      # sources changed since
    assert bench.measured_traffic("missing", "bfs_kernel") is None


def test_cpu_parallel_sample_counts_every_query():
    done = []

    def task(i):
        def run():
            done.append(i)
            return i
        return run
    total, q, wall, th = bench.cpu_parallel_sample((task(i) for i in range(10)), budget_s=60, threads=3)
    assert q == 10 and total == sum(range(10)) and sorted(done) == list(range(10)) and th == 3
    # a spent budget stops new submissions after the first wave
    total, q, wall, th = bench.cpu_parallel_sample((task(i) for i in range(10)), budget_s=0, threads=3)
    assert q == 3


def test_serve_cpu_tasks_run_the_oracle():
    import graphgen as G
    csrs = [G.add_weights(G.rmat(8, 8, seed=s), 1, 22, seed=2) for s in (1, 2)]
    _, q, _, _ = bench.cpu_parallel_sample(bench.serve_cpu_tasks(csrs, seed=5), budget_s=0.2, threads=2)
    assert q >= 2


def test_host_cpu_names_model_and_cores():
    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count() and isinstance(h["model"], str) and h["model"]


def test_every_workload_has_an_oracle_leg():
    """The reference arm and the CPU baseline run the oracle for every kind
    of workload: each one answers on a tiny graph of the same kind."""
    import graphgen as G
    kinds = {wl["kind"] for wl in bench.WORKLOADS.values()} - {"serve", "msbfs"}
    for kind in kinds:
        wl = next(w for w in bench.WORKLOADS.values() if w["kind"] == kind)
        g = G.rmat(8, 8, seed=3)
        if wl["w"] is not None:
            G.add_weights(g, wl["w"][0], wl["w"][1], seed=2)
        srcs = G.sources(g, 2, seed=3)
        te, t, q = bench.cpu_reference_sample(g, wl, srcs, budget_s=5.0, max_queries=1)
        assert q == 1 and te > 0 and t >= 0, kind
        assert kind in bench.ORACLE_NAME, kind


def test_bytes_algorithmic_terms():
    st = dict(edges_scanned=10, vertices_expanded=3, vertices_pulled=7, relaxations=4,
              bucket_inserts=5, vertices_reached=6, pull_rounds=2, heavy_vertices=2, rounds=4)
    n = 65
    nb = (n + 7) // 8
    assert bench.bytes_algorithmic("bfs", n, st) == \
        4 * 10 + 8 * 3 + 4 * 7 + 12 * 6 + 4 * 3 + 2 * nb * 2 + 8 * n
    assert bench.bytes_algorithmic("wbfs", n, st) == \
        8 * 10 + 8 * 3 + 4 * 7 + 12 * 6 + 8 * 5 + 2 * nb * 2 + 8 * n
    assert bench.bytes_algorithmic("msbfs", n, st, lanes=64) == 12 * 10 + 24 * n * 4 + 4 * 64 * n
    assert bench.bytes_algorithmic("kcore", n, st) is None
    for k in ("bfs", "wbfs", "delta", "msbfs"):
        assert k in bench.ALG_MODEL
    assert set(bench.STAT_TERMS) <= set(st) | {"vertices_pulled"}


def test_reference_arm_line_has_the_gpu_arms_config(capsys):
    """The reference arm prints one line whose config is the GPU arm's
    (same keys, same values) for the same workload."""
    import argparse
    wl = dict(kind="bfs", graph="rmat", scale=9, ef=8, w=None, nsrc=3, desc="tiny BFS")
    args = argparse.Namespace(steps=4, warmup=1, workload="tiny", rates="", serve_warm=0,
                              serve_meas=0)
    assert bench.run_reference(args, wl, 0, 1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    g = bench.make_graph(wl)
    assert line["config"] == bench.workload_config("tiny", wl, g, 3)
    assert line["impl"] == "reference" and line["steps"] == 4 and line["warmup"] == 1
    assert line["value"] > 0 and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
