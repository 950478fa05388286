#!/usr/bin/env python3
"""Benchmark of the frontier-traversal path on one GB300 (or N replicas).

Default workload (the largest single-GPU configuration, the one the HBM
roofline target is set on): BFS with distances and parents on a seeded RMAT
graph, scale 26 (67,108,864 vertices, ~2.1 B arcs), edge factor 16,
a/b/c/d = .57/.19/.19/.05, symmetrized and deduplicated; 4 seeded sources
run one at a time.  One step = those 4 queries.  Other workloads:
--workload wbfs-rmat22, bfs-rmat22, wbfs-rmat26, bfs-grid, wbfs-grid,
msbfs-rmat24, serve, and the next rows' kernels.

Metric: GTEPS, Graph500 convention: per query, the undirected edges of the
reached component (sum of reached degrees / 2), summed over queries, over the
device time.  The graph (8.4 GB of targets at scale 26) is larger than L2,
so no flush is needed between steps.

Roofline: algorithmic bytes per launch from the query's device counters
(4 B per scanned arc, 8 per expanded frontier vertex, 4 per dense-round
candidate, 12 per reached vertex, 4 per queue read, two bitmap passes per
dense round, 8 n for the initialisation; weighted BFS counts 8 B per arc and
4 B per bucket write and read) over the CUDA-event time of the launch;
a richer model that also counts the per-arc distance and bitmap reads is
reported beside it as `extended`.

Prints ONE JSON line.  --impl reference times the oracle (the serial CPU
reference) on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as G  # noqa: E402

INF = 2**31 - 1

WORKLOADS = {
    "wbfs-rmat22": dict(kind="wbfs", graph="rmat", scale=22, ef=16, w=(1, 22), nsrc=8,
                        desc="wBFS, RMAT scale 22 ef16, w in [1,22), 8 seeded sources one at a time"),
    "wbfs-rmat20": dict(kind="wbfs", graph="rmat", scale=20, ef=16, w=(1, 22), nsrc=8,
                        desc="wBFS, RMAT scale 20 ef16, w in [1,22), 8 seeded sources (profiling size)"),
    "bfs-rmat20": dict(kind="bfs", graph="rmat", scale=20, ef=16, w=None, nsrc=8,
                       desc="BFS (dist+parent), RMAT scale 20 ef16, 8 seeded sources (profiling size)"),
    "bfs-rmat22": dict(kind="bfs", graph="rmat", scale=22, ef=16, w=None, nsrc=8,
                       desc="BFS (dist+parent), RMAT scale 22 ef16, 8 seeded sources"),
    "bfs-rmat24": dict(kind="bfs", graph="rmat", scale=24, ef=16, w=None, nsrc=4,
                       desc="BFS (dist+parent), RMAT scale 24 ef16, 4 seeded sources (profiling size)"),
    "bfs-rmat26": dict(kind="bfs", graph="rmat", scale=26, ef=16, w=None, nsrc=4,
                       desc="BFS (dist+parent), RMAT scale 26 ef16 (~2.1B arcs), 4 seeded sources"),
    "bf-rmat22": dict(kind="bf", graph="rmat", scale=22, ef=16, w=(1, 22), nsrc=8,
                      desc="Bellman-Ford (Alg. 4), RMAT scale 22 ef16, w in [1,22), 8 seeded sources"),
    "widest-rmat22": dict(kind="widest", graph="rmat", scale=22, ef=16, w=(1, 22), nsrc=8,
                          desc="widest path ((max,min) Bellman-Ford rounds), RMAT scale 22 ef16, "
                               "w in [1,22), 8 seeded sources"),
    "bc-rmat22": dict(kind="bc", graph="rmat", scale=22, ef=16, w=None, nsrc=8,
                      desc="single-source betweenness (Alg. 2, forward path counts + backward "
                           "dependencies, fp64), RMAT scale 22 ef16, 8 seeded sources"),
    "kcore-rmat22": dict(kind="kcore", graph="rmat", scale=22, ef=16, w=None, nsrc=1,
                         desc="coreness of every vertex (Alg. 16 peeling), RMAT scale 22 ef16; "
                              "one step = one full decomposition; GTEPS = undirected edges / time"),
    "ldd-rmat22": dict(kind="ldd", beta=0.2, graph="rmat", scale=22, ef=16, w=None, nsrc=1,
                       desc="low-diameter decomposition (Alg. 6), beta 0.2, shifts seeded "
                            "(graphgen.exp_shifts, seed 5), RMAT scale 22 ef16; one step = one "
                            "decomposition; GTEPS = undirected edges / time"),
    "cc-rmat22": dict(kind="cc", graph="rmat", scale=22, ef=16, w=None, nsrc=1,
                      desc="connected components (smallest-id labels), RMAT scale 22 ef16; one "
                           "step = one labelling; GTEPS = undirected edges / time"),
    "wbfs-rmat26": dict(kind="wbfs", graph="rmat", scale=26, ef=16, w=(1, 22), nsrc=2,
                        desc="wBFS, RMAT scale 26 ef16, w in [1,22), 2 seeded sources"),
    "msbfs-rmat24": dict(kind="msbfs", graph="rmat", scale=24, ef=16, w=None, nsrc=64,
                         desc="multi-source BFS, 64 seeded sources in one uint64-lane launch, "
                              "RMAT scale 24 ef16, autotuned; vs 64 single-source BFS launches"),
    "msbfs-rmat20": dict(kind="msbfs", graph="rmat", scale=20, ef=16, w=None, nsrc=64,
                         desc="multi-source BFS, 64 sources, RMAT scale 20 (profiling size)"),
    "mssp-rmat22": dict(kind="mssp", graph="rmat", scale=22, ef=16, w=(1, 22), nsrc=8,
                        desc="multi-source SSSP, 8 seeded sources in one launch (8 distance lanes, "
                             "shared Bellman-Ford rounds), RMAT scale 22 ef16, w in [1,22); vs the "
                             "8 queries as single-source weighted BFS launches"),
    "mssp-rmat20": dict(kind="mssp", graph="rmat", scale=20, ef=16, w=(1, 22), nsrc=8,
                        desc="multi-source SSSP, 8 sources in one launch, RMAT scale 20 ef16, "
                             "w in [1,22)"),
    "mssp-rmat24": dict(kind="mssp", graph="rmat", scale=24, ef=16, w=(1, 22), nsrc=8,
                        desc="multi-source SSSP, 8 sources in one launch, RMAT scale 24 ef16, "
                             "w in [1,22) (the serving mix's largest graph)"),
    "serve": dict(kind="serve", graph="rmat", scales=(18, 20, 22, 24), ef=16, w=(1, 22), nsrc=0,
                  rates=(1000, 2000, 5000, 10000, 20000, 50000), warm=2000, meas=20000,
                  desc="serving: 4 resident RMAT graphs (scales 18/20/22/24, ef16, w in [1,22)), "
                       "Poisson arrivals, 80% BFS / 20% wBFS, uniform sources with degree > 0"),
    "bfs-grid": dict(kind="bfs", graph="grid", R=4096, C=4096, w=None, nsrc=4,
                     desc="BFS, 4096x4096 grid, 10% edges deleted, source 0 + 3 seeded"),
    "wbfs-grid": dict(kind="wbfs", graph="grid", R=4096, C=4096, w=(1, 16), nsrc=4,
                      desc="wBFS, 4096x4096 grid, 10% deleted, w in [1,16), source 0 + 3 seeded"),
    "delta-grid": dict(kind="delta", delta=64, graph="grid", R=4096, C=4096, w=(1, 16), nsrc=4,
                       desc="delta-stepping (delta 64), 4096x4096 grid, 10% deleted, w in [1,16), "
                            "source 0 + 3 seeded"),
    "delta-rmat22": dict(kind="delta", delta=4, graph="rmat", scale=22, ef=16, w=(1, 22), nsrc=8,
                         desc="delta-stepping (delta 4), RMAT scale 22 ef16, w in [1,22), "
                              "8 seeded sources one at a time"),
}


def reduce_job(ms, te, dist_mod, device):
    """Whole-job timing across ranks: the slowest rank's time and the sum of
    the traversed edges (queries are sharded across ranks, no data exchange)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    e = torch.tensor([float(te)], dtype=torch.float64, device=device)
    dist_mod.all_reduce(e, op=dist_mod.ReduceOp.SUM)
    return float(t.item()), float(e.item())


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def make_graph(wl):
    if wl["graph"] == "rmat":
        g = G.rmat(wl["scale"], wl["ef"], 0.57, 0.19, 0.19, seed=1, permute=True)
    else:
        g = G.grid(wl["R"], wl["C"], 0.1, seed=1)
    if wl["w"] is not None:
        G.add_weights(g, wl["w"][0], wl["w"][1], seed=2)
    return g


def make_sources(g, wl, rank=0):
    k = wl["nsrc"]
    if wl["graph"] == "grid":
        s = G.sources(g, k, seed=3 + 1000 * rank)
        if rank == 0:
            s[0] = 0
        return s
    return G.sources(g, k, seed=3 + 1000 * rank)


ORACLE_NAME = {"bfs": "FIFO BFS", "msbfs": "FIFO BFS per source", "mssp": "binary-heap Dijkstra per source", "wbfs": "binary-heap Dijkstra", "delta": "binary-heap Dijkstra",
               "ldd": "MPX rounds", "cc": "FIFO search per component",
               "bf": "frontier Bellman-Ford", "widest": "(max,min) Bellman-Ford rounds",
               "bc": "betweenness forward + backward passes", "kcore": "bucket peeling"}


def reach_of(kind, g, src, out):
    """Values whose finite entries mark the source's component.  Widest path
    gives unreachable vertices INF, like the source itself, so its component
    is every vertex with a finite width plus the source."""
    d = out.cpu().numpy() if hasattr(out, "cpu") else out
    if kind != "widest":
        return d
    reach = np.where(d != INF, 0, INF).astype(np.int64)
    reach[src] = 0
    return reach


def traversed_edges(g, dist):
    """Graph500 TEPS numerator: undirected edges in the reached component."""
    deg = np.diff(g.off.astype(np.int64))
    return int(deg[dist != INF].sum() // 2)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.rows = []
        self.proc = None
        self.dev = device_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=3)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = {
    "bfs_kernel": ("bfs.cu", "dev_common.cuh", "gbf_dev.h"),
    "wbfs_kernel": ("wbfs.cu", "dev_common.cuh", "gbf_dev.h"),
    "msbfs_kernel": ("msbfs.cu", "dev_common.cuh", "gbf_dev.h"),
    "bf_kernel": ("bellman_ford.cu", "dev_common.cuh", "gbf_dev.h"),
    "bc_kernel": ("betweenness.cu", "dev_common.cuh", "gbf_dev.h"),
    "kcore_kernel": ("kcore.cu", "dev_common.cuh", "gbf_dev.h"),
    "mssp_kernel": ("mssp.cu", "dev_common.cuh", "gbf_dev.h"),
    "ldd_kernel": ("ldd.cu", "dev_common.cuh", "gbf_dev.h"),
    "cc_kernel": ("connectivity.cu", "dev_common.cuh", "gbf_dev.h"),
}


def kernel_source_hash(kernel):
    """Short hash of the CUDA sources a kernel is built from: a DRAM-traffic
    figure taken with ncu is only reported while those are unchanged."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1805_05208_gb300", "csrc", name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(workload, kernel):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch of `kernel` on
    `workload` from profiles/traffic.json (written from an ncu capture), or
    None if there is none for the current sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            table = json.load(f)
    except (OSError, ValueError):
        return None
    e = table.get(workload)
    if not e or e.get("kernel") != kernel or e.get("csrc_hash") != kernel_source_hash(kernel):
        return None
    return e.get("bytes_per_launch")


def bytes_algorithmic(kind, n, st, lanes=64):
    """Algorithmic bytes of one query for the traversal kernels, from the
    query's device counters: E arcs scanned, Vx frontier vertices expanded
    (each read from its queue), Vp dense-round candidates, R vertices
    reached, Dn dense rounds, I bucket filings.  Random accesses count their
    own bytes, not a 32 B sector.  None for kernels without such a model."""
    E, Vx, Vp = st["edges_scanned"], st["vertices_expanded"], st.get("vertices_pulled", 0)
    R, Dn, I = st["vertices_reached"], st["pull_rounds"], st["bucket_inserts"]
    nb = (n + 7) // 8
    if kind == "bfs":
        # target per arc; offsets pair and queue entry per expanded vertex;
        # the extra offset of each dense candidate; D, parent and queue entry
        # per reached vertex; frontier and visited bitmaps per dense round;
        # D and parent initialised
        return 4 * E + 8 * Vx + 4 * Vp + 12 * R + 4 * Vx + 2 * nb * Dn + 8 * n
    if kind in ("wbfs", "delta"):
        # as BFS with target + weight per arc and no queue reads; every bucket
        # filing is written once and read once when its bucket is taken
        return 8 * E + 8 * Vx + 4 * Vp + 12 * R + 8 * I + 2 * nb * Dn + 8 * n
    if kind == "msbfs":
        # target and the neighbour's 8-byte lane word per arc; seen, visit and
        # next (8 B each) per vertex and level; every distance written once
        return 12 * E + 24 * n * st["rounds"] + 4 * lanes * n
    return None


def bytes_model(kind, n, st):
    """Extended bytes of one query (every access counted once, 4 B per
    word, random or not), from the device statistics of the query."""
    E, V, R, I = st["edges_scanned"], st["vertices_expanded"], st["relaxations"], st["bucket_inserts"]
    if kind == "delta":
        # as wBFS, plus the expansion stamps and side-list flags set up (4n +
        # n/4) and one stamp exchange per extracted entry (4)
        return 8 * n + n // 4 + 24 * I + 12 * E + 8 * R + 16 * st["heavy_vertices"]
    if kind == "wbfs":
        # init D (4n); per filing: the bucket write, then at extraction the
        # ring slot, D[v], offsets pair (20; filings I, stale ones included,
        # degree-1 vertices not filed); per scanned arc: tgt, w, D[v] (12);
        # per successful writeMin: atomicMin and the degree-1 bitmap word (8);
        # per heavy vertex: queue + degree prefix written and read (16)
        return 4 * n + 20 * I + 12 * E + 8 * R + 16 * st["heavy_vertices"]
    if kind == "cc":
        # init labels and the queue of vertices with arcs (4n + 12n); per
        # round every arc: target, both labels (12), and the shortcut pass
        # over every vertex: its label and the label it names (8n)
        return 16 * n + 12 * E + st["rounds"] * 8 * n
    if kind == "ldd":
        # read the shifts (8n), write C and T (8n); per round the centre pass
        # reads C and T of every vertex (8n); per frontier vertex its queue
        # entry, prefix and first arc written and read (24); per scanned arc:
        # target, the source's cluster, the target's cluster (12)
        return 16 * n + st["rounds"] * 8 * n + 24 * n + 12 * E
    if kind == "kcore":
        # init remaining degrees and the finished bitmap (4n + n/8); per
        # bucket one pass over them (remaining degree and finished word of
        # every vertex; the next bucket's minimum is gathered in the same
        # pass); per arc of a peeled vertex: target, its remaining degree, the
        # fetch-and-add (12); per vertex: queue entry written and read,
        # coreness written (16)
        nk = st["rounds"] - st["push_rounds"]  # bucket passes (rounds counts both kinds)
        return 4 * n + n // 8 + nk * (4 * n + n // 8) + 12 * E + 16 * n
    if kind == "bc":
        # init path counts, dependencies (fp64) and levels (20n); per scanned
        # arc in either pass: target, its level, one 8-byte value (16); per
        # reached vertex: its queue entry written and read twice (24), path
        # count and dependency (16)
        return 20 * n + 16 * E + 40 * st["vertices_reached"]
    if kind in ("bf", "widest"):
        # init values (4n) and both flag bitmaps (n/4); per frontier vertex:
        # queue, degree prefix, first arc, flag reset (16); per scanned arc:
        # target, weight, source value, target value (16); per successful
        # writeMin/Max: the atomic and the flag test-and-set (8)
        return 4 * n + n // 4 + 16 * V + 16 * E + 8 * R
    if kind == "mssp":
        # 16-bit lanes (the bench's graphs never need the 32-bit rerun: their
        # distances stay far below 65,535): init and final read of the 8
        # distance lanes (2 x 16n), every row written once (4kn, k = 8); per
        # scanned arc: target, weight and the target's 16-byte lane word (24);
        # per frontier vertex: queue entry, prefix, first arc and its lane
        # byte (16); per successful lowering: the swap and the lane-mask OR (8)
        return 32 * n + 32 * n + 24 * E + 16 * V + 8 * R
    if kind == "msbfs":
        # init seen/visit/next (32n); every dist[i][v] written once (4kn); per
        # scanned arc: target + the neighbour's lane word (12); per frontier
        # vertex / pull candidate: offsets, lane words, queue (24); per dense
        # level: seen read and next-lane word written for every vertex (16n)
        return 32 * n + 4 * 64 * n + 12 * E + 24 * V + 16 * n * st["pull_rounds"]
    # BFS: init D, parent (8n) + visited bitmap (n/8); per frontier vertex or
    # pull candidate: queue/offset reads (12); per arc: target + bitmap word (8);
    # per reached vertex: D, parent, offsets, queue+qoff write (24); bitmaps per
    # dense round (3 passes of n/8)
    return 8 * n + n // 8 + 12 * V + 8 * E + 24 * st["vertices_reached"] + \
        3 * (n // 8) * st["pull_rounds"]


ALG_MODEL = {
    "bfs": "4 E + 8 Vx + 4 Vp + 12 R + 4 Vx + 2 ceil(n/8) Dn + 8 n",
    "wbfs": "8 E + 8 Vx + 4 Vp + 12 R + 8 I + 2 ceil(n/8) Dn + 8 n",
    "delta": "8 E + 8 Vx + 4 Vp + 12 R + 8 I + 2 ceil(n/8) Dn + 8 n",
    "msbfs": "12 E + 24 n L + 4 k n",
}
EXT_MODEL = "extended: every access of the kernel counted once at 4 B per word (bench.bytes_model)"
# device counters the byte models read (E, Vx, Vp, R, Dn, I, L)
STAT_TERMS = ("edges_scanned", "vertices_expanded", "vertices_pulled", "vertices_reached",
              "pull_rounds", "bucket_inserts", "rounds")


def trace_summary(tr):
    """Per-kind round counts and device time of one query's round trace."""
    out, prev = {}, 0
    names = {1: "sparse", 2: "dense", 3: "sparse+heavy", 4: "conversion+sparse", 5: "bucket",
             6: "sparse-bitmap", 7: "conversion+sparse-bitmap", 8: "cta-local"}
    for (_, kind, fr, fe, t, _tm) in tr:
        k = names.get(kind, str(kind))
        d = out.setdefault(k, {"rounds": 0, "us": 0.0, "frontier": 0})
        d["rounds"] += 1
        d["us"] += (t - prev) / 1e3
        d["frontier"] += fr
        prev = t
    for d in out.values():
        d["us"] = round(d["us"], 1)
    return {"rounds": len(tr), "end_us": round(prev / 1e3, 1), "by_kind": out}


def cpu_reference_sample(g, wl, srcs, budget_s=15.0, max_queries=None):
    """Time the oracle on a bounded sample of the workload's queries."""
    import oracle
    te, t = 0, 0.0
    done = 0
    for s in srcs:
        t0 = time.perf_counter()
        if wl["kind"] in ("wbfs", "delta", "mssp"):
            d = oracle.dijkstra(g, int(s))
        elif wl["kind"] == "bf":
            d = oracle.bellman_ford(g, int(s))
        elif wl["kind"] == "widest":
            # the widest-path output marks unreachable vertices INF too: count
            # the source's component by hops
            oracle.widest_path(g, int(s))
            d, _ = oracle.bfs(g, int(s), parents=False)
        elif wl["kind"] == "bc":
            _, _, lv = oracle.betweenness(g, int(s), full=True)
            d = np.where(lv >= 0, lv, INF)
        elif wl["kind"] == "kcore":
            oracle.coreness(g)
            d = np.zeros(g.n, dtype=np.int64)  # every edge is processed
        elif wl["kind"] == "ldd":
            oracle.ldd(g, G.exp_shifts(g.n, wl["beta"], seed=5))
            d = np.zeros(g.n, dtype=np.int64)
        elif wl["kind"] == "cc":
            oracle.components(g)
            d = np.zeros(g.n, dtype=np.int64)
        else:
            d, _ = oracle.bfs(g, int(s))
        t += time.perf_counter() - t0
        te += traversed_edges(g, d)
        done += 1
        if t > budget_s or (max_queries and done >= max_queries):
            break
    return te, t, done


_ARM_PARTS = {0xd0c: "Neoverse-N1", 0xd40: "Neoverse-V1", 0xd49: "Neoverse-N2",
              0xd4f: "Neoverse-V2", 0xd8e: "Neoverse-N3", 0xd84: "Neoverse-V3"}


def host_cpu():
    """The host CPU the oracle is timed on: model and logical cores."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                k, v = k.strip(), v.strip()
                if k == "model name" and v:
                    model = v
                    break
                if k == "CPU part" and v:
                    part = int(v, 16)
                    model = _ARM_PARTS.get(part, f"Arm part {v}")
                    break
    except (OSError, ValueError):
        pass
    import platform
    return {"model": model or platform.machine(), "nproc": os.cpu_count()}


def cpu_parallel_sample(tasks, budget_s, threads=None):
    """Run independent oracle queries (callables returning a count) on all
    host cores until about `budget_s` seconds have passed: one thread per core
    (the oracle's C entry points release the GIL).  Returns (sum of counts,
    queries done, wall seconds, threads)."""
    import concurrent.futures as cf
    threads = threads or os.cpu_count() or 1
    it = iter(tasks)
    total, done = 0, 0
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        futs = set()
        for _ in range(threads):
            nxt = next(it, None)
            if nxt is None:
                break
            futs.add(ex.submit(nxt))
        while futs:
            fin, futs = cf.wait(futs, return_when=cf.FIRST_COMPLETED)
            for f in fin:
                total += f.result()
                done += 1
                if time.perf_counter() - t0 < budget_s:
                    nxt = next(it, None)
                    if nxt is not None:
                        futs.add(ex.submit(nxt))
    return total, done, time.perf_counter() - t0, threads


def serve_cpu_tasks(csrs, seed):
    """The serving mix (uniform graph, 80 % BFS / 20 % Dijkstra, sources of
    degree > 0) as oracle calls returning 1.  At most two Dijkstra queries run
    at once: the oracle's heap holds one entry per arc."""
    import oracle
    rng = np.random.default_rng(seed)
    heavy = threading.Semaphore(2)

    def bfs(g, s):
        return lambda: (oracle.bfs(g, s, parents=False), 1)[1]

    def sssp(g, s):
        def run():
            with heavy:
                oracle.dijkstra(g, s)
            return 1
        return run

    while True:
        j = int(rng.integers(len(csrs)))
        s = int(G.sources(csrs[j], 1, seed=int(rng.integers(1 << 30)))[0])
        yield sssp(csrs[j], s) if rng.random() >= 0.8 else bfs(csrs[j], s)


def workload_config(name, wl, g, nsrc):
    """The `config` object of a bench line: the workload and its sizes (the
    same keys and values in the GPU arm and the reference arm)."""
    seeds = {"graph": 1, "sources": 3}
    if wl["w"] is not None:
        seeds["weights"] = 2
    return {"workload": name, "desc": wl["desc"], "n": int(g.n), "arcs": int(g.m),
            "sources_per_step": int(nsrc), "seeds": seeds,
            "l2": "inputs larger than L2 (graph arrays exceed 129 MB); no flush"}


def serve_config(wl, csrs, rates, warm, meas):
    return {"workload": "serve", "desc": wl["desc"], "rates": rates,
            "queries_per_rate": {"warmup": warm, "measured": meas},
            "graphs": [{"scale": sc, "n": c.n, "arcs": c.m} for sc, c in zip(wl["scales"], csrs)],
            "arrival_seed": 4}


def serve_graphs(wl):
    csrs = []
    for sc in wl["scales"]:
        g = G.rmat(sc, wl["ef"], 0.57, 0.19, 0.19, seed=1, permute=True)
        G.add_weights(g, wl["w"][0], wl["w"][1], seed=2)
        csrs.append(g)
    return csrs


def run_reference(args, wl, rank, world):
    """The reference arm: the oracle as it stands, on the host cores.  Each
    step is one single-source oracle query of the workload (one decomposition
    for the whole-graph kernels; one query of the serving mix for `serve`),
    a bounded sample of the GPU arm's step.  The steps run as independent
    queries on all host cores (one thread each; the oracle's C calls release
    the GIL), so that a scale-26 run of the default K and W ends within a
    few minutes."""
    if rank != 0:
        return 0
    threads = max(1, min(os.cpu_count() or 1, args.steps))
    if wl["kind"] == "serve":
        csrs = serve_graphs(wl)
        rates = [int(r) for r in (args.rates.split(",") if args.rates else wl["rates"])]
        warm, meas = (args.serve_warm or wl["warm"]), (args.serve_meas or wl["meas"])
        cfg = serve_config(wl, csrs, rates, warm, meas)
        tasks = serve_cpu_tasks(csrs, seed=7)
        _, _, _, _ = cpu_parallel_sample((next(tasks) for _ in range(args.warmup)), 1e9, threads)
        _, q, wall, th = cpu_parallel_sample((next(tasks) for _ in range(args.steps)), 1e9, threads)
        val, unit, metric = q / wall, "queries/s", "served queries/s"
        what = f"{q} queries of the serving mix (FIFO BFS / binary-heap Dijkstra)"
    else:
        g = make_graph(wl)
        srcs = make_sources(g, wl)
        cfg = workload_config(args.workload, wl, g, len(srcs))

        def task(i):
            s = srcs[i % len(srcs)]
            return lambda: cpu_reference_sample(g, wl, [s], budget_s=1e9, max_queries=1)[0]
        cpu_parallel_sample((task(i) for i in range(args.warmup)), 1e9, threads)
        te, q, wall, th = cpu_parallel_sample((task(args.warmup + i) for i in range(args.steps)),
                                              1e9, threads)
        val, unit, metric = te / wall / 1e9, "GTEPS", "GTEPS"
        what = (f"{q} single-source oracle queries ({ORACLE_NAME[wl['kind']]}), one per step, "
                f"of the {wl['nsrc']}-source step")
    line = {"metric": metric, "value": val, "unit": unit, "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * wall / max(q, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": val, "unit": unit, "cores": th, "kind": "oracle",
                             "host": host_cpu(),
                             "sample": f"{what}, run as independent queries on {th} host threads, "
                                       f"{wall:.1f} s"},
            "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def serve_run(gb, hs, csrs, opt, rate, n_warm, n_meas, seed):
    """Offer Poisson arrivals at `rate` q/s to a fresh server; returns
    (throughput q/s over the measured queries, p50 us, p99 us, stats)."""
    srv = gb.gbf_server_create([h.h for h in hs], opt)
    rng = np.random.default_rng(seed)
    total = n_warm + n_meas
    gaps = rng.exponential(1.0 / rate, size=total)
    arrive = np.cumsum(gaps)
    gi = rng.integers(len(hs), size=total)
    kind = (rng.random(total) >= 0.8).astype(np.int64)  # 80% BFS, 20% wBFS
    srcs = np.empty(total, dtype=np.int64)
    for j in range(len(hs)):
        idx = np.flatnonzero(gi == j)
        if idx.size:
            srcs[idx] = G.sources(csrs[j], idx.size, seed=seed * 7 + j)
    index = {}
    lat = np.full(total, np.nan)
    t_done = np.full(total, np.nan)
    stop = threading.Event()
    lock = threading.Lock()

    def collector():
        while not stop.is_set() or True:
            t, l, st = gb.gbf_server_collect(srv, 4096)
            now = time.perf_counter()
            if len(t):
                with lock:
                    for tk, lv in zip(t.tolist(), l.tolist()):
                        q = index.pop(tk, None)
                        if q is not None:
                            lat[q] = lv
                            t_done[q] = now
            elif stop.is_set():
                break
            else:
                time.sleep(0.0002)

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = time.perf_counter()
    i = 0
    while i < total:
        now = time.perf_counter() - t0
        while i < total and arrive[i] <= now:
            tk = gb.gbf_server_submit(srv, int(gi[i]), int(kind[i]), int(srcs[i]))
            if tk is None:          # not admissible now: offered again shortly
                break
            with lock:
                index[tk] = i
            i += 1
        else:
            time.sleep(0.00005)
            continue
        time.sleep(0.0001)
    # wait for completion
    while True:
        with lock:
            left = len(index)
        if left == 0:
            break
        time.sleep(0.001)
    stop.set()
    th.join()
    st = gb.gbf_server_stats(srv)
    gb.gbf_server_destroy(srv)
    m = slice(n_warm, total)
    ml = lat[m]
    t_first = t0 + arrive[n_warm]
    thr = n_meas / (np.nanmax(t_done[m]) - t_first)
    return float(thr), float(np.nanpercentile(ml, 50)), float(np.nanpercentile(ml, 99)), st


def run_serve(args, wl, rank, world):
    """Serving workload: batched server vs one-query-per-launch FIFO."""
    import torch
    import paper_1805_05208_gb300 as gb
    if rank != 0:
        return 0
    torch.cuda.set_device(0)
    csrs = serve_graphs(wl)
    hs = [gb.Graph(c, validate=gb.VALIDATE_BASIC) for c in csrs]
    rates = [int(r) for r in (args.rates.split(",") if args.rates else wl["rates"])]
    warm, meas = (args.serve_warm or wl["warm"]), (args.serve_meas or wl["meas"])
    # each mode at every weighted-engine share of the GPU (0 = equal shares
    # per engine); each mode is credited with its best share
    shares = [int(x) for x in args.serve_shares.split(",")]
    modes = {
        "batched": dict(bfs_engines=args.serve_engines[0], wbfs_engines=args.serve_engines[1],
                        max_batch=64),
        "one_per_launch_fifo": dict(bfs_engines=1, wbfs_engines=1, max_batch=1),
    }
    res = {}
    with ClockSampler(0) as clk:
        for name, kw in modes.items():
            res[name] = []
            for sh in shares:
                opt = gb.gbf_server_options_default(wbfs_share=sh, **kw)
                for r in rates:
                    thr, p50, p99, st = serve_run(gb, hs, csrs, opt, r, warm, meas, seed=4)
                    res[name].append({"offered_qps": r, "wbfs_share": sh, "qps": thr,
                                      "p50_us": p50, "p99_us": p99,
                                      "mean_batch": st["batched_queries"] / max(1, st["batches"]),
                                      "failed": st["failed"]})
    best = max(x["qps"] for x in res["batched"])
    base = max(x["qps"] for x in res["one_per_launch_fifo"])
    clocks = clk.summary()
    cpu = cpu_all = None
    if not args.no_cpu_baseline:
        _, q1, t1, _ = cpu_parallel_sample(serve_cpu_tasks(csrs, seed=5), args.cpu_budget, threads=1)
        cpu = {"value": q1 / t1, "unit": "queries/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
               "sample": f"{q1} queries of the serving mix (FIFO BFS / binary-heap Dijkstra), "
                         f"{t1:.1f} s"}
        _, qa, ta, th = cpu_parallel_sample(serve_cpu_tasks(csrs, seed=6), args.cpu_budget)
        cpu_all = {"value": qa / ta, "unit": "queries/s", "cores": th, "kind": "oracle",
                   "host": host_cpu(),
                   "sample": f"{qa} independent queries of the serving mix, one thread per "
                             f"host core, {ta:.1f} s"}
    line = {
        "metric": "served queries/s", "value": best, "unit": "queries/s", "n_gpus": 1,
        "steps": len(rates), "warmup": warm, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": serve_config(wl, csrs, rates, warm, meas),
        "serve": res,
        "speedup_vs_one_per_launch": best / base,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "e2e": {"value": best, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "submit-to-completion through the C ABI; results left on the device"},
        "gpu_launches": None,
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
    }
    print(json.dumps(line))
    for h in hs:
        h.close()
    return 0


def run_msbfs(args, wl, g, srcs, graph, opt, stream, dev, rank, world, barrier, dist_mod):
    """One step = one multi-source BFS launch over the 64 sources; the same
    64 sources as single-source launches are timed beside it."""
    import torch
    import paper_1805_05208_gb300 as gb
    n, k = g.n, len(srcs)
    if not args.opt:
        opt = gb.gbf_autotune(graph.h, gb.TUNE_MSBFS)
    tuned = {f: getattr(opt, f) for f in ("block", "pull_divisor", "heavy_cutoff")}
    out = torch.empty((k, n), dtype=torch.int32, device=dev)
    deg = torch.from_numpy(np.diff(g.off.astype(np.int64))).to(dev)
    stats = None
    for w in range(args.warmup):
        gb.gbf_msbfs(graph.h, srcs, out, opt, stream)
        if w == 0:
            stats = gb.gbf_wait(graph.h, stream)
            trace0 = gb.gbf_trace(graph.h)
    gb.gbf_wait(graph.h, stream)
    te_step = int(((out != INF).to(torch.int64) * deg).sum().item() // 2)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s_ in range(args.steps):
            ev[s_][0].record(stream)
            gb.gbf_msbfs(graph.h, srcs, out, opt, stream)
            ev[s_][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
    barrier()
    st = gb.gbf_wait(graph.h, stream)
    if st["device_error"]:
        raise RuntimeError(f"device error {st['device_error']}")
    ms_total = t0.elapsed_time(t1)
    # the comparison: the same 64 queries as one single-source launch each
    d1 = torch.empty(n, dtype=torch.int32, device=dev)
    bopt = gb.gbf_autotune(graph.h, gb.TUNE_BFS) if not args.opt else opt
    for s_ in srcs[:4]:
        gb.gbf_bfs(graph.h, int(s_), d1, None, bopt, stream)
    gb.gbf_wait(graph.h, stream)
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for s_ in srcs:
        gb.gbf_bfs(graph.h, int(s_), d1, None, bopt, stream)
    a1.record(stream)
    torch.cuda.synchronize()
    ms_single64 = a0.elapsed_time(a1)
    if world > 1:
        ms_total, te_all = reduce_job(ms_total, te_step, dist_mod, dev)
    else:
        te_all = float(te_step)
    value = te_all * args.steps / (ms_total / 1e3) / 1e9
    launch_ms = [e[0].elapsed_time(e[1]) for e in ev]
    peak, peak_kind = load_peaks()
    bpl = bytes_algorithmic("msbfs", n, stats, lanes=k)
    bpl_ext = bytes_model("msbfs", n, stats)
    avg = sum(launch_ms) / len(launch_ms)
    # end to end: host output buffer, the 64 x n result copied back each step
    host = torch.empty((k, n), dtype=torch.int32, pin_memory=True).numpy()
    e2e_steps = max(1, min(args.steps, 3))
    gb.gbf_msbfs(graph.h, srcs, host, opt, None)  # untimed warm-up (first-call host-output buffer)
    torch.cuda.synchronize()
    barrier()
    tt0 = time.perf_counter()
    for _ in range(e2e_steps):
        gb.gbf_msbfs(graph.h, srcs, host, opt, None)
    e2e_s = time.perf_counter() - tt0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
        e2e_s = float(t.item())
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            te_c, t_c, q = cpu_reference_sample(g, dict(wl, kind="bfs"), srcs,
                                                budget_s=args.cpu_budget)
            cpu = {"value": te_c / t_c / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                   "host": host_cpu(),
                   "sample": f"{q} of the {k} single-source oracle BFS runs of one step, "
                             f"{t_c:.1f} s"}
        cpu_all = None
        if not args.no_cpu_baseline and world == 1:
            import oracle

            def task(s_):
                return lambda: traversed_edges(g, oracle.bfs(g, int(s_), parents=False)[0])
            te_a, qa, ta, th = cpu_parallel_sample((task(s_) for s_ in srcs), args.cpu_budget)
            cpu_all = {"value": te_a / ta / 1e9, "unit": "GTEPS", "cores": th, "kind": "oracle",
                       "host": host_cpu(),
                       "sample": f"{qa} of the {k} sources as independent oracle BFS runs, one "
                                 f"thread per host core, {ta:.1f} s"}
        clocks = clk.summary()
        line = {
            "metric": "GTEPS", "value": value, "unit": "GTEPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "uint64-lanes/int32",
            "data": "synthetic",
            "config": workload_config(args.workload, wl, g, k),
            "options": {"tuned": tuned},
            "vs_single_source_launches": {"ms_64_single": ms_single64,
                                          "ms_one_msbfs": ms_total / args.steps,
                                          "speedup": ms_single64 / (ms_total / args.steps),
                                          "single_options": {f: getattr(bopt, f) for f in
                                                             ("block", "pull_divisor", "heavy_cutoff")}},
            "roofline": {"bound": "hbm", "kernel": "msbfs_kernel", "achieved": bpl / (avg / 1e3) / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": bpl / (avg / 1e3) / 1e9 / peak,
                         "peak_source": f"{peak_kind} hbm_gbs (burst copy)", "bytes_per_launch": bpl,
                         "avg_launch_ms": avg, "model": ALG_MODEL["msbfs"],
                         "traffic": measured_traffic(args.workload, "msbfs_kernel"),
                         "extended": {"bytes_per_launch": bpl_ext,
                                      "achieved": bpl_ext / (avg / 1e3) / 1e9,
                                      "frac": bpl_ext / (avg / 1e3) / 1e9 / peak,
                                      "model": EXT_MODEL}},
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "e2e": {"value": te_all * e2e_steps / e2e_s / 1e9, "unit": "GTEPS",
                    "h2d_bytes_per_step": 4 * k, "d2h_bytes_per_step": 4 * k * n},
            "gpu_launches": args.steps,
            "clocks": {kk: clocks[kk] for kk in ("sm_mhz", "sm_max_mhz", "reasons")},
            "stats": {"levels": stats["rounds"], "pull_levels": stats["pull_rounds"],
                      "per_query": [{f: stats[f] for f in STAT_TERMS}],
                      "edges_scanned": stats["edges_scanned"], "traversed_edges_per_step": te_step,
                      "grid_ctas": stats["grid_ctas"], "block": stats["block"],
                      "query0_trace": trace_summary(trace0)},
        }
        print(json.dumps(line))
    graph.close()
    if world > 1:
        dist_mod.destroy_process_group()
    return 0


def run_mssp(args, wl, g, srcs, graph, opt, stream, dev, rank, world, barrier, dist_mod):
    """One step = one multi-source SSSP launch over the 8 sources; the same
    8 queries as single-source weighted BFS launches are timed beside it."""
    import torch
    import paper_1805_05208_gb300 as gb
    n, k = g.n, len(srcs)
    out = torch.empty((k, n), dtype=torch.int32, device=dev)
    deg = torch.from_numpy(np.diff(g.off.astype(np.int64))).to(dev)
    stats = trace0 = None
    for w in range(args.warmup):
        gb.gbf_mssp(graph.h, srcs, out, opt, stream)
        if w == 0:
            stats = gb.gbf_wait(graph.h, stream)
            trace0 = gb.gbf_trace(graph.h)
    gb.gbf_wait(graph.h, stream)
    te_step = int(((out != INF).to(torch.int64) * deg).sum().item() // 2)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s_ in range(args.steps):
            ev[s_][0].record(stream)
            gb.gbf_mssp(graph.h, srcs, out, opt, stream)
            ev[s_][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
    barrier()
    st = gb.gbf_wait(graph.h, stream)
    if st["device_error"]:
        raise RuntimeError(f"device error {st['device_error']}")
    ms_total = t0.elapsed_time(t1)
    # the comparison: the same queries as one weighted BFS launch each
    d1 = torch.empty(n, dtype=torch.int32, device=dev)
    for s_ in srcs[:2]:
        gb.gbf_wbfs(graph.h, int(s_), d1, opt, stream)
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for s_ in srcs:
        gb.gbf_wbfs(graph.h, int(s_), d1, opt, stream)
    a1.record(stream)
    torch.cuda.synchronize()
    ms_single = a0.elapsed_time(a1)
    if world > 1:
        ms_total, te_all = reduce_job(ms_total, te_step, dist_mod, dev)
    else:
        te_all = float(te_step)
    value = te_all * args.steps / (ms_total / 1e3) / 1e9
    launch_ms = [e[0].elapsed_time(e[1]) for e in ev]
    avg = sum(launch_ms) / len(launch_ms)
    peak, peak_kind = load_peaks()
    bpl = bytes_model("mssp", n, stats)
    host = torch.empty((k, n), dtype=torch.int32, pin_memory=True).numpy()
    e2e_steps = max(1, min(args.steps, 3))
    gb.gbf_mssp(graph.h, srcs, host, opt, None)  # untimed warm-up (first-call host-output buffer)
    torch.cuda.synchronize()
    barrier()
    tt0 = time.perf_counter()
    for _ in range(e2e_steps):
        gb.gbf_mssp(graph.h, srcs, host, opt, None)
    e2e_s = time.perf_counter() - tt0
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            te_c, t_c, q = cpu_reference_sample(g, wl, srcs, budget_s=args.cpu_budget)
            cpu = {"value": te_c / t_c / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                   "host": host_cpu(),
                   "sample": f"{q} of the {k} single-source Dijkstra runs of one step, {t_c:.1f} s"}
        clocks = clk.summary()
        line = {
            "metric": "GTEPS", "value": value, "unit": "GTEPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": workload_config(args.workload, wl, g, k),
            "vs_single_source_launches": {"ms_8_wbfs": ms_single, "ms_one_mssp": ms_total / args.steps,
                                          "speedup": ms_single / (ms_total / args.steps)},
            "roofline": {"bound": "hbm", "kernel": "mssp_kernel", "achieved": bpl / (avg / 1e3) / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": bpl / (avg / 1e3) / 1e9 / peak,
                         "peak_source": f"{peak_kind} hbm_gbs (burst copy)", "bytes_per_launch": bpl,
                         "avg_launch_ms": avg, "model": EXT_MODEL,
                         "traffic": measured_traffic(args.workload, "mssp_kernel")},
            "cpu_baseline": cpu,
            "e2e": {"value": te_all * e2e_steps / e2e_s / 1e9, "unit": "GTEPS",
                    "h2d_bytes_per_step": 4 * k, "d2h_bytes_per_step": 4 * k * n},
            "gpu_launches": args.steps,
            "clocks": {kk: clocks[kk] for kk in ("sm_mhz", "sm_max_mhz", "reasons")},
            "stats": {"rounds": stats["rounds"], "edges_scanned": stats["edges_scanned"],
                      "per_query": [{f: stats[f] for f in STAT_TERMS}],
                      "traversed_edges_per_step": te_step, "grid_ctas": stats["grid_ctas"],
                      "block": stats["block"], "query0_trace": trace_summary(trace0)},
        }
        print(json.dumps(line))
    graph.close()
    if world > 1:
        dist_mod.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbf", choices=["gbf", "reference"])
    ap.add_argument("--workload", default="bfs-rmat26", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--opt", default="", help="comma list of gbf_options overrides k=v")
    ap.add_argument("--rates", default="", help="serve: comma list of offered rates (q/s)")
    ap.add_argument("--serve-warm", type=int, default=0)
    ap.add_argument("--serve-meas", type=int, default=0)
    ap.add_argument("--serve-engines", default="1,1",
                    help="serve: BFS,wBFS engines of the batched server")
    ap.add_argument("--serve-shares", default="67",
                    help="serve: comma list of weighted-engine GPU shares (percent; 0 = equal)")
    args = ap.parse_args()
    args.serve_engines = tuple(int(x) for x in args.serve_engines.split(","))
    args.warmup = max(args.warmup, 3)
    wl = WORKLOADS[args.workload]

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, wl, rank, world)
    if wl["kind"] == "serve":
        return run_serve(args, wl, rank, world)

    import torch
    import torch.distributed as dist_mod
    torch.cuda.set_device(local)
    if world > 1:
        dist_mod.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist_mod.barrier()

    import paper_1805_05208_gb300 as gb

    g = make_graph(wl)
    srcs = make_sources(g, wl, rank)
    n = g.n
    dev = torch.device("cuda", local)
    opt = gb.gbf_options_default()
    for kv in filter(None, args.opt.split(",")):
        k, v = kv.split("=")
        setattr(opt, k, int(v))
    graph = gb.Graph(g, validate=gb.VALIDATE_BASIC)
    stream = torch.cuda.Stream(device=dev)
    kind = wl["kind"]
    if kind == "msbfs":
        return run_msbfs(args, wl, g, srcs, graph, opt, stream, dev, rank, world, barrier, dist_mod)
    if kind == "mssp":
        return run_mssp(args, wl, g, srcs, graph, opt, stream, dev, rank, world, barrier, dist_mod)
    out_dtype = torch.float64 if kind == "bc" else torch.int32
    outs = [torch.empty(n, dtype=out_dtype, device=dev) for _ in srcs]
    if kind == "ldd":  # the shifts are an input; the join rounds a second output
        ldd_delta = G.exp_shifts(n, wl["beta"], seed=5)
        ldd_delta_dev = torch.from_numpy(ldd_delta).to(dev)
        ldd_rounds = torch.empty(n, dtype=torch.int32, device=dev)
    pars = [torch.empty(n, dtype=torch.int32, device=dev) for _ in srcs] if kind == "bfs" else None

    def launch(i):
        if kind == "wbfs":
            gb.gbf_wbfs(graph.h, int(srcs[i]), outs[i], opt, stream)
        elif kind == "delta":
            gb.gbf_delta_stepping(graph.h, int(srcs[i]), wl["delta"], outs[i], opt, stream)
        elif kind == "bf":
            gb.gbf_bellman_ford(graph.h, int(srcs[i]), outs[i], opt, stream)
        elif kind == "widest":
            gb.gbf_widest_path(graph.h, int(srcs[i]), outs[i], opt, stream)
        elif kind == "bc":
            gb.gbf_betweenness(graph.h, int(srcs[i]), outs[i], opt, stream)
        elif kind == "kcore":
            gb.gbf_kcore(graph.h, outs[i], opt, stream)
        elif kind == "ldd":
            gb.gbf_ldd(graph.h, ldd_delta_dev, outs[i], ldd_rounds, opt, stream)
        elif kind == "cc":
            gb.gbf_connectivity(graph.h, outs[i], opt, stream)
        else:
            gb.gbf_bfs(graph.h, int(srcs[i]), outs[i], pars[i], opt, stream)

    # Warm-up; the first pass also records each query's statistics and TEPS numerator.
    stats, te = [], []
    for w in range(args.warmup):
        for i in range(len(srcs)):
            launch(i)
            if w == 0:
                stats.append(gb.gbf_wait(graph.h, stream))
                if kind in ("kcore", "ldd", "cc"):
                    te.append(g.m // 2)
                elif kind == "bc":
                    # the component, from one untimed BFS of this library
                    hops = torch.empty(n, dtype=torch.int32, device=dev)
                    gb.gbf_bfs(graph.h, int(srcs[i]), hops, None, None, stream)
                    gb.gbf_wait(graph.h, stream)
                    te.append(traversed_edges(g, hops.cpu().numpy()))
                    launch(i)
                    stats[-1] = gb.gbf_wait(graph.h, stream)
                else:
                    te.append(traversed_edges(g, reach_of(kind, g, int(srcs[i]), outs[i])))
                if i == 0:
                    trace0 = gb.gbf_trace(graph.h)
    gb.gbf_wait(graph.h, stream)
    te_step = sum(te)

    # Timed region: K steps, events per launch on the launching stream.
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps * len(srcs))]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        k = 0
        for s in range(args.steps):
            for i in range(len(srcs)):
                ev[k][0].record(stream)
                launch(i)
                ev[k][1].record(stream)
                k += 1
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier()
    st_last = gb.gbf_wait(graph.h, stream)
    if st_last["device_error"]:
        raise RuntimeError(f"device error {st_last['device_error']}")
    ms_total = t_start.elapsed_time(t_end)
    if world > 1:
        ms_total, te_all = reduce_job(ms_total, te_step, dist_mod, dev)
    else:
        te_all = float(te_step)
    launch_ms = [e[0].elapsed_time(e[1]) for e in ev]
    value = te_all * args.steps / (ms_total / 1e3) / 1e9

    # Roofline of the one persistent kernel (each query is one launch).
    peak, peak_kind = load_peaks()
    avg_launch_ms = sum(launch_ms) / len(launch_ms)
    ext_per_launch = sum(bytes_model(kind, n, s) for s in stats) / len(srcs)
    alg = [bytes_algorithmic(kind, n, s) for s in stats]
    has_alg = all(a is not None for a in alg)
    bytes_per_launch = sum(alg) / len(srcs) if has_alg else ext_per_launch
    achieved = bytes_per_launch / (avg_launch_ms / 1e3) / 1e9
    ext_achieved = ext_per_launch / (avg_launch_ms / 1e3) / 1e9

    # End to end: the C-ABI call with host buffers (D2H of each result inside).
    host_out = [torch.empty(n, dtype=out_dtype, pin_memory=True).numpy() for _ in srcs]
    # BFS: one batched call per step, each query's read-back overlapping the
    # next query's search (gbf_bfs_host_batch), into pinned rows
    host_d2 = torch.empty((len(srcs), n), dtype=torch.int32, pin_memory=True).numpy() \
        if kind == "bfs" else None
    host_p2 = torch.empty((len(srcs), n), dtype=torch.int32, pin_memory=True).numpy() \
        if kind == "bfs" else None
    srcs_np = np.asarray(srcs, dtype=np.int32)
    host_rounds = torch.empty(n, dtype=torch.int32, pin_memory=True).numpy() if kind == "ldd" else None
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for s in range(-1, e2e_steps):
        if s == 0:  # step -1 is an untimed warm-up (first-call buffers, copy stream)
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
        if kind == "bfs":
            gb.gbf_bfs_host_batch(graph.h, srcs_np, host_d2, host_p2, opt, None)
            continue
        for i in range(len(srcs)):
            if kind == "wbfs":
                gb.gbf_wbfs(graph.h, int(srcs[i]), host_out[i], opt, None)
            elif kind == "delta":
                gb.gbf_delta_stepping(graph.h, int(srcs[i]), wl["delta"], host_out[i], opt, None)
            elif kind == "bf":
                gb.gbf_bellman_ford(graph.h, int(srcs[i]), host_out[i], opt, None)
            elif kind == "widest":
                gb.gbf_widest_path(graph.h, int(srcs[i]), host_out[i], opt, None)
            elif kind == "bc":
                gb.gbf_betweenness(graph.h, int(srcs[i]), host_out[i], opt, None)
            elif kind == "kcore":
                gb.gbf_kcore(graph.h, host_out[i], opt, None)
            elif kind == "ldd":
                gb.gbf_ldd(graph.h, ldd_delta, host_out[i], host_rounds, opt, None)
            elif kind == "cc":
                gb.gbf_connectivity(graph.h, host_out[i], opt, None)
            else:
                raise ValueError(kind)
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_val = te_all * e2e_steps / e2e_s / 1e9
    d2h = len(srcs) * n * (8 if kind == "bc" else 4 * (2 if kind in ("bfs", "ldd") else 1))

    # widest path runs the Bellman-Ford kernel, Δ-stepping the wBFS kernel
    kname = {"widest": "bf_kernel", "delta": "wbfs_kernel"}.get(kind, f"{kind}_kernel")
    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            te_c, t_c, q = cpu_reference_sample(g, wl, srcs, budget_s=args.cpu_budget)
            cpu = {"value": te_c / t_c / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                   "host": host_cpu(),
                   "sample": f"{q} of the {len(srcs)} queries of one step, serial oracle "
                             f"({ORACLE_NAME[kind]}), "
                             f"{t_c:.1f} s"}
        clocks = clk.summary()
        line = {
            "metric": "GTEPS", "value": value, "unit": "GTEPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if kind == "bc" else "int32",
            "data": "synthetic",
            "config": workload_config(args.workload, wl, g, len(srcs)),
            "options": {f: getattr(opt, f) for f, _ in opt._fields_},
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                         "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_launch_ms,
                         "model": ALG_MODEL[kind] if has_alg else EXT_MODEL,
                         "traffic": measured_traffic(args.workload, kname),
                         "extended": {"bytes_per_launch": ext_per_launch, "achieved": ext_achieved,
                                      "frac": ext_achieved / peak, "model": EXT_MODEL}},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "GTEPS",
                    "h2d_bytes_per_step": 8 * n if kind == "ldd" else 4 * len(srcs),
                    "d2h_bytes_per_step": d2h,
                    "note": ("one gbf_bfs_host_batch call per step: each query's read-back overlaps "
                             "the next query's search; pinned host rows") if kind == "bfs" else
                            "one call per query with host buffers (blocking)"},
            "gpu_launches": args.steps * len(srcs),
            "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "stats": {"rounds": [s["rounds"] for s in stats],
                      "pull_rounds": [s["pull_rounds"] for s in stats],
                      "edges_scanned": sum(s["edges_scanned"] for s in stats),
                      "per_query": [{f: s[f] for f in STAT_TERMS} for s in stats],
                      "traversed_edges_per_step": te_step,
                      "grid_ctas": stats[0]["grid_ctas"], "block": stats[0]["block"],
                      "query0_trace": trace_summary(trace0)},
        }
        print(json.dumps(line))
    graph.close()
    if world > 1:
        dist_mod.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
