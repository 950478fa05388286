"""Seeded synthetic graph inputs (RMAT, 2D grid, small closed-form graphs).

This module is shared by the tests, the benchmark and the oracle's callers.
It holds none of the traversal arithmetic: it only draws graphs, weights and
source vertices.  The heavy generators live in ``gen.c`` (built with gcc into
``_build/libgraphgen.so``); small helpers are numpy.

Every graph returned is a :class:`CSR`: symmetric, vertices ``0..n-1``,
sorted adjacency lists, no self-loops, no duplicate arcs, ``uint32`` offsets
and ``int32`` targets, optional ``uint32`` weights (one per undirected edge).
Inputs stand in for the paper's datasets (experiments section, Table 2); the
weight range convention follows the experiments section ([1, log n)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
import weakref
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libgraphgen.so")
_lock = threading.Lock()
_lib = None


class _GGCsr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_uint64),
                ("off", ctypes.POINTER(ctypes.c_uint32)),
                ("tgt", ctypes.POINTER(ctypes.c_int32))]


def build(force: bool = False) -> str:
    """Compile gen.c into _build/libgraphgen.so (gcc, portable flags)."""
    src = os.path.join(_HERE, "gen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                           "-o", tmp, src])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                    ctypes.POINTER(_GGCsr)]
            lib.gg_rmat.restype = ctypes.c_int
            lib.gg_grid.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.POINTER(_GGCsr)]
            lib.gg_grid.restype = ctypes.c_int
            lib.gg_release.argtypes = [ctypes.c_void_p]
            lib.gg_release.restype = None
            lib.gg_weights.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_void_p]
            lib.gg_weights.restype = ctypes.c_int
            lib.gg_sources.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint64,
                                       ctypes.c_int32, ctypes.c_void_p]
            lib.gg_sources.restype = ctypes.c_int
            lib.gg_max_degree_vertex.argtypes = [ctypes.c_int32, ctypes.c_void_p]
            lib.gg_max_degree_vertex.restype = ctypes.c_int32
            lib.gg_set_threads.argtypes = [ctypes.c_int]
            lib.gg_get_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def set_threads(t: int) -> None:
    """Thread count for the C generators (0 = all online cores)."""
    _load().gg_set_threads(int(t))


@dataclass
class CSR:
    n: int
    off: np.ndarray                 # uint32[n+1]
    tgt: np.ndarray                 # int32[m]
    w: Optional[np.ndarray] = None  # uint32[m] or None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.off[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.off.astype(np.int64))


def _owned(addr: int, count: int, ctype, dtype) -> np.ndarray:
    """numpy view of a malloc'd C array; the memory is released when the last
    view of it is garbage collected."""
    lib = _load()
    buf = (ctype * max(count, 1)).from_address(addr)
    weakref.finalize(buf, lib.gg_release, addr)
    return np.frombuffer(buf, dtype=dtype, count=count)


def _take(c: _GGCsr, name: str) -> CSR:
    """Adopt the C-allocated arrays without copying."""
    n, m = int(c.n), int(c.m)
    off_addr = ctypes.cast(c.off, ctypes.c_void_p).value
    tgt_addr = ctypes.cast(c.tgt, ctypes.c_void_p).value
    off = _owned(off_addr, n + 1, ctypes.c_uint32, np.uint32)
    tgt = _owned(tgt_addr, m, ctypes.c_int32, np.int32)
    return CSR(n=n, off=off, tgt=tgt, name=name)


def rmat(scale: int, edgefactor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True) -> CSR:
    """Seeded RMAT graph, symmetrized, self-loops and duplicates removed."""
    lib = _load()
    out = _GGCsr()
    rc = lib.gg_rmat(scale, edgefactor, a, b, c, seed, 1 if permute else 0, ctypes.byref(out))
    if rc != 0:
        raise MemoryError(f"gg_rmat failed ({rc})")
    g = _take(out, f"rmat{scale}_ef{edgefactor}")
    g.meta.update(kind="rmat", scale=scale, edgefactor=edgefactor, a=a, b=b, c=c, seed=seed,
                  permute=bool(permute))
    return g


def grid(R: int, C: int, delete_frac: float = 0.1, seed: int = 1) -> CSR:
    """R x C 4-neighbour grid (vertex id r*C+c), edges deleted with probability delete_frac."""
    lib = _load()
    out = _GGCsr()
    rc = lib.gg_grid(R, C, delete_frac, seed, ctypes.byref(out))
    if rc != 0:
        raise MemoryError(f"gg_grid failed ({rc})")
    g = _take(out, f"grid{R}x{C}")
    g.meta.update(kind="grid", R=R, C=C, delete_frac=delete_frac, seed=seed)
    return g


def add_weights(g: CSR, lo: int, hi: int, seed: int = 2) -> CSR:
    """Attach uint32 weights uniform in [lo, hi), symmetric per undirected edge."""
    lib = _load()
    w = np.empty(max(g.m, 1), dtype=np.uint32)[:g.m]
    rc = lib.gg_weights(g.n, g.off.ctypes.data, g.tgt.ctypes.data, lo, hi, seed, w.ctypes.data)
    if rc != 0:
        raise ValueError("bad weight range")
    g.w = w
    g.meta.update(w_lo=lo, w_hi=hi, w_seed=seed)
    return g


def sources(g: CSR, k: int, seed: int = 3) -> np.ndarray:
    """k seeded sources uniform over vertices with degree > 0."""
    lib = _load()
    out = np.zeros(k, dtype=np.int32)
    got = lib.gg_sources(g.n, g.off.ctypes.data, seed, k, out.ctypes.data)
    if got != k:
        raise ValueError("graph has no arcs")
    return out


def exp_shifts(n: int, beta: float, seed: int = 5) -> np.ndarray:
    """n seeded draws from the exponential distribution with rate beta
    (float64): the random shifts a low-diameter decomposition draws, passed
    to it as an input."""
    return np.random.default_rng(_u64(seed, n) & 0xffffffff).exponential(1.0 / beta, size=n)


def max_degree_vertex(g: CSR) -> int:
    """Highest-degree vertex, ties broken by the lowest id."""
    return int(_load().gg_max_degree_vertex(g.n, g.off.ctypes.data))


# ----------------------------------------------------------------- small graphs
def csr_from_edges(n: int, edges, weights=None, name: str = "") -> CSR:
    """Symmetric CSR from an undirected edge list (u, v); duplicates and
    self-loops are dropped (the first weight given for a pair is kept)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    wv = None if weights is None else np.asarray(weights, dtype=np.int64).reshape(-1)
    keep = e[:, 0] != e[:, 1]
    e = e[keep]
    if wv is not None:
        wv = wv[keep]
    lo = np.minimum(e[:, 0], e[:, 1])
    hi = np.maximum(e[:, 0], e[:, 1])
    key = lo * n + hi
    _, first = np.unique(key, return_index=True)
    lo, hi = lo[first], hi[first]
    if wv is not None:
        wv = wv[first]
    src = np.concatenate([lo, hi])
    dst = np.concatenate([hi, lo])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    off = np.zeros(n + 1, dtype=np.uint32)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off, dtype=np.uint64).astype(np.uint32)
    g = CSR(n=n, off=off, tgt=dst.astype(np.int32), name=name)
    if wv is not None:
        ww = np.concatenate([wv, wv])[order]
        g.w = ww.astype(np.uint32)
    return g


def path_graph(n: int, weights=None) -> CSR:
    return csr_from_edges(n, [(i, i + 1) for i in range(n - 1)], weights, name=f"path{n}")


def star_graph(n: int) -> CSR:
    """Vertex 0 is the centre, 1..n-1 leaves."""
    return csr_from_edges(n, [(0, i) for i in range(1, n)], name=f"star{n}")


def complete_graph(n: int) -> CSR:
    return csr_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)],
                          name=f"K{n}")


def grid_graph(R: int, C: int, weight: Optional[int] = None) -> CSR:
    """Intact R x C grid (id r*C+c); constant weight if given."""
    edges = []
    for r in range(R):
        for c in range(C):
            v = r * C + c
            if c + 1 < C:
                edges.append((v, v + 1))
            if r + 1 < R:
                edges.append((v, v + C))
    w = None if weight is None else [weight] * len(edges)
    return csr_from_edges(R * C, edges, w, name=f"grid{R}x{C}")


def _u64(seed: int, *xs: int) -> int:
    """Counter-based 64-bit draw (splitmix64 finaliser chain) for small graphs."""
    M = (1 << 64) - 1
    x = seed & M
    for v in (0x9e3779b97f4a7c15,) + tuple(xs):
        x = (x + v + 0x9e3779b97f4a7c15) & M
        x = ((x ^ (x >> 30)) * 0xbf58476d1ce4e5b9) & M
        x = ((x ^ (x >> 27)) * 0x94d049bb133111eb) & M
        x ^= x >> 31
    return x


def random_small(n: int, p: float, seed: int, w_hi: Optional[int] = None) -> CSR:
    """Seeded Erdos-Renyi-style graph on n vertices, each pair kept with
    probability p; weights uniform in [1, w_hi) when w_hi is given."""
    rng = np.random.default_rng(_u64(seed, n) & 0xffffffff)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p
    edges = np.stack([iu[keep], ju[keep]], axis=1)
    w = None
    if w_hi is not None:
        w = rng.integers(1, w_hi, size=edges.shape[0])
    return csr_from_edges(n, edges, w, name=f"er{n}_{seed}")
