"""The oracle — TEST INFRASTRUCTURE, not part of the product.

A plain serial CPU statement of what the traversal path computes, written
from the paper's problem statements (§4, "Breadth-First Search",
"Integral-Weight SSSP", "General-Weight SSSP (Bellman-Ford)", "Widest
Path", "Single-Source Betweenness Centrality", "k-core"): hop distances,
shortest-path distances, widest-path widths, betweenness dependencies and
corenesses, each the unique answer to its definition.  ``oracle.c`` holds the arithmetic (FIFO
BFS, binary-heap Dijkstra, Floyd–Warshall, output validators); this module
only marshals numpy arrays into it.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library.

Pins (see tests/test_oracle_pins.py): closed forms on path, star, complete,
grid and disconnected graphs; brute-force Floyd–Warshall and SciPy's
csgraph on hundreds of seeded tiny graphs; wBFS with unit weights equal to
BFS; a hand-worked fixture under tests/golden/; and planted mistakes the
validators must reject.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

INF = 2**31 - 1
_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

CHECK_CODES = {0: "ok", 1: "bad source", 2: "edge gap", 3: "reach mismatch", 4: "bad parent",
               5: "unreached vertex has a parent", 6: "no tight arc", 7: "negative distance"}


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, serial, portable)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            lib.or_bfs.argtypes = [ctypes.c_int32, P, P, ctypes.c_int32, P, P]
            lib.or_bfs.restype = ctypes.c_int64
            lib.or_dijkstra.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_int32, P]
            lib.or_dijkstra.restype = ctypes.c_int64
            lib.or_bellman_ford.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_int32, ctypes.c_int,
                                            P]
            lib.or_bellman_ford.restype = ctypes.c_int64
            lib.or_betweenness.argtypes = [ctypes.c_int32, P, P, ctypes.c_int32, P, P, P]
            lib.or_betweenness.restype = ctypes.c_int64
            lib.or_coreness.argtypes = [ctypes.c_int32, P, P, P]
            lib.or_coreness.restype = ctypes.c_int64
            lib.or_components.argtypes = [ctypes.c_int32, P, P, P]
            lib.or_components.restype = ctypes.c_int64
            lib.or_ldd.argtypes = [ctypes.c_int32, P, P, P, P, P]
            lib.or_ldd.restype = ctypes.c_int64
            lib.or_floyd_warshall.argtypes = [ctypes.c_int32, P, P, P, P]
            lib.or_floyd_warshall.restype = ctypes.c_int
            lib.or_check_bfs.argtypes = [ctypes.c_int32, P, P, ctypes.c_int32, P, P,
                                         ctypes.POINTER(ctypes.c_int32)]
            lib.or_check_bfs.restype = ctypes.c_int64
            lib.or_check_sssp.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_int32, P,
                                          ctypes.POINTER(ctypes.c_int32)]
            lib.or_check_sssp.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def bfs(g, src: int, parents: bool = True):
    """Hop distances (int32, INF = 2**31-1) and a BFS tree (parent[src] = src,
    -1 for unreachable).  Returns (dist, parent) or (dist, None)."""
    lib = _load()
    off, po = _c(g.off, np.uint32)
    tgt, pt = _c(g.tgt, np.int32) if g.m else (np.zeros(1, np.int32), None)
    if pt is None:
        pt = tgt.ctypes.data
    dist = np.empty(g.n, dtype=np.int32)
    par = np.empty(g.n, dtype=np.int32) if parents else None
    rc = lib.or_bfs(g.n, po, pt, int(src), dist.ctypes.data, par.ctypes.data if parents else None)
    if rc < 0:
        raise ValueError("or_bfs: bad argument")
    return dist, par


def dijkstra(g, src: int, w=None):
    """Shortest-path distances with the graph's integer weights (int32, INF)."""
    lib = _load()
    w = g.w if w is None else w
    if w is None:
        raise ValueError("graph has no weights")
    off, po = _c(g.off, np.uint32)
    tgt = np.ascontiguousarray(g.tgt, dtype=np.int32) if g.m else np.zeros(1, np.int32)
    ww = np.ascontiguousarray(w, dtype=np.uint32) if g.m else np.zeros(1, np.uint32)
    dist = np.empty(g.n, dtype=np.int32)
    rc = lib.or_dijkstra(g.n, po, tgt.ctypes.data, ww.ctypes.data, int(src), dist.ctypes.data)
    if rc == -2:
        raise OverflowError("distance exceeds int32")
    if rc < 0:
        raise ValueError("or_dijkstra: bad argument")
    return dist


def _bellman_ford(g, src: int, mode: int):
    lib = _load()
    if g.w is None:
        raise ValueError("graph has no weights")
    off, po = _c(g.off, np.uint32)
    tgt = np.ascontiguousarray(g.tgt, dtype=np.int32) if g.m else np.zeros(1, np.int32)
    ww = np.ascontiguousarray(g.w, dtype=np.uint32) if g.m else np.zeros(1, np.uint32)
    out = np.empty(g.n, dtype=np.int32)
    rc = lib.or_bellman_ford(g.n, po, tgt.ctypes.data, ww.ctypes.data, int(src), mode,
                             out.ctypes.data)
    if rc == -2:
        raise OverflowError("distance exceeds int32")
    if rc < 0:
        raise ValueError("or_bellman_ford: bad argument")
    return out, int(rc)


def bellman_ford(g, src: int, rounds: bool = False):
    """General-weight SSSP by frontier Bellman-Ford rounds (Alg. 4): int32
    distances, INF if unreachable; with rounds=True also the round count."""
    d, r = _bellman_ford(g, src, 0)
    return (d, r) if rounds else d


def widest_path(g, src: int, rounds: bool = False):
    """Single-source widest path: for each v the largest, over paths from src,
    smallest weight on the path; INF at the source (empty path) and, by the
    paper's output convention, at unreachable vertices."""
    d, r = _bellman_ford(g, src, 1)
    return (d, r) if rounds else d


def betweenness(g, src: int, full: bool = False):
    """Single-source betweenness dependencies (Alg. 2), fp64; with full=True
    also the shortest-path counts and hop levels."""
    lib = _load()
    off, po = _c(g.off, np.uint32)
    tgt = np.ascontiguousarray(g.tgt, dtype=np.int32) if g.m else np.zeros(1, np.int32)
    D = np.empty(g.n, dtype=np.float64)
    paths = np.empty(g.n, dtype=np.float64)
    level = np.empty(g.n, dtype=np.int32)
    rc = lib.or_betweenness(g.n, po, tgt.ctypes.data, int(src), D.ctypes.data,
                            paths.ctypes.data, level.ctypes.data)
    if rc < 0:
        raise ValueError("or_betweenness: bad argument")
    return (D, paths, level) if full else D


def coreness(g):
    """Coreness of every vertex (int32): the largest k such that the vertex
    lies in a subgraph of minimum degree k."""
    lib = _load()
    off, po = _c(g.off, np.uint32)
    tgt = np.ascontiguousarray(g.tgt, dtype=np.int32) if g.m else np.zeros(1, np.int32)
    core = np.empty(g.n, dtype=np.int32)
    rc = lib.or_coreness(g.n, po, tgt.ctypes.data, core.ctypes.data)
    if rc < 0:
        raise ValueError("or_coreness: bad argument")
    return core


def components(g):
    """Connected components (§4 "Connectivity"): int32 label[v] = the smallest
    vertex id in v's component."""
    lib = _load()
    off, po = _c(g.off, np.uint32)
    tgt = np.ascontiguousarray(g.tgt, dtype=np.int32) if g.m else np.zeros(1, np.int32)
    label = np.empty(max(g.n, 1), dtype=np.int32)[:g.n]
    rc = lib.or_components(g.n, po, tgt.ctypes.data, label.ctypes.data)
    if rc < 0:
        raise ValueError("or_components: bad argument")
    return label


def ldd(g, delta):
    """Low-diameter decomposition (§4; Alg. 6) with the given shifts
    delta[v] ~ Exp(beta): (C, T), C[v] the centre of v's cluster (one valid
    choice where searches tie), T[v] the round v joined a frontier."""
    lib = _load()
    off, po = _c(g.off, np.uint32)
    tgt = np.ascontiguousarray(g.tgt, dtype=np.int32) if g.m else np.zeros(1, np.int32)
    d = np.ascontiguousarray(delta, dtype=np.float64)
    if d.shape != (g.n,):
        raise ValueError("delta must have one entry per vertex")
    C = np.empty(max(g.n, 1), dtype=np.int32)[:g.n]
    T = np.empty(max(g.n, 1), dtype=np.int32)[:g.n]
    rc = lib.or_ldd(g.n, po, tgt.ctypes.data, d.ctypes.data, C.ctypes.data, T.ctypes.data)
    if rc < 0:
        raise ValueError("or_ldd: bad argument")
    return C, T


def floyd_warshall(g, weighted: bool):
    """All-pairs distances (int64 n x n, INF = 2**63-1); tiny graphs only."""
    lib = _load()
    off, po = _c(g.off, np.uint32)
    tgt = np.ascontiguousarray(g.tgt, dtype=np.int32) if g.m else np.zeros(1, np.int32)
    ww = None
    if weighted:
        ww = np.ascontiguousarray(g.w, dtype=np.uint32) if g.m else np.zeros(1, np.uint32)
    d = np.empty((g.n, g.n), dtype=np.int64)
    rc = lib.or_floyd_warshall(g.n, po, tgt.ctypes.data, ww.ctypes.data if weighted else None,
                               d.ctypes.data)
    if rc != 0:
        raise ValueError("or_floyd_warshall: bad argument")
    return d


def msbfs(g, srcs):
    """Distances from each source, one oracle BFS per source: int32[k, n]."""
    out = np.empty((len(srcs), g.n), dtype=np.int32)
    for i, s in enumerate(srcs):
        out[i], _ = bfs(g, int(s), parents=False)
    return out


def check_bfs(g, src: int, dist, parent=None):
    """Validate BFS output invariants; returns (ok, vertex, reason)."""
    lib = _load()
    off, po = _c(g.off, np.uint32)
    tgt = np.ascontiguousarray(g.tgt, dtype=np.int32) if g.m else np.zeros(1, np.int32)
    d, pd = _c(dist, np.int32)
    pp = None
    if parent is not None:
        p, pp = _c(parent, np.int32)
    code = ctypes.c_int32(0)
    v = lib.or_check_bfs(g.n, po, tgt.ctypes.data, int(src), pd, pp, ctypes.byref(code))
    return v < 0, int(v), CHECK_CODES[code.value]


def check_sssp(g, src: int, dist):
    """Validate shortest-path invariants; returns (ok, vertex, reason)."""
    lib = _load()
    off, po = _c(g.off, np.uint32)
    tgt = np.ascontiguousarray(g.tgt, dtype=np.int32) if g.m else np.zeros(1, np.int32)
    ww = np.ascontiguousarray(g.w, dtype=np.uint32) if g.m else np.zeros(1, np.uint32)
    d, pd = _c(dist, np.int32)
    code = ctypes.c_int32(0)
    v = lib.or_check_sssp(g.n, po, tgt.ctypes.data, ww.ctypes.data, int(src), pd,
                          ctypes.byref(code))
    return v < 0, int(v), CHECK_CODES[code.value]
