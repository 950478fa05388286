"""Python binding of libgbf.so — the GB300 frontier-traversal library.

Argument marshalling only: every step of BFS, weighted BFS and multi-source
BFS runs in the library's CUDA kernels.  Functions carry the C ABI's names
(``gbf_graph_create``, ``gbf_bfs``, ...) and accept numpy arrays (host
memory) or torch CUDA tensors (device memory); torch is used only for device
memory and streams.  If the library has not been built, importing the
binding raises immediately: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

INF = 2**31 - 1
NOPARENT = -1
HOST = 0
DEVICE = 1
VALIDATE_BASIC = 1
VALIDATE_SYMMETRIC = 2

STATUS = {0: "GBF_OK", 1: "GBF_ERR_INVALID", 2: "GBF_ERR_OOM", 3: "GBF_ERR_CUDA",
          4: "GBF_ERR_TIMEOUT", 5: "GBF_ERR_OVERFLOW", 6: "GBF_ERR_BUSY", 7: "GBF_ERR_NOT_FOUND"}

LIB_PATH = _build.LIB


class GbfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class gbf_options(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("pull_divisor", ctypes.c_int32),
                ("heavy_cutoff", ctypes.c_int32), ("bucket_window", ctypes.c_int32),
                ("dense_wbfs", ctypes.c_int32), ("local_arcs", ctypes.c_int32),
                ("spin_cap_us", ctypes.c_int64), ("ctas", ctypes.c_int32),
                ("pull_serial", ctypes.c_int32), ("inject_wait", ctypes.c_int32),
                ("pull_stay", ctypes.c_int32)]


class gbf_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("push_rounds", ctypes.c_int64),
                ("pull_rounds", ctypes.c_int64), ("edges_scanned", ctypes.c_int64),
                ("vertices_expanded", ctypes.c_int64), ("vertices_reached", ctypes.c_int64),
                ("relaxations", ctypes.c_int64), ("bucket_inserts", ctypes.c_int64),
                ("refills", ctypes.c_int64), ("heavy_vertices", ctypes.c_int64),
                ("vertices_pulled", ctypes.c_int64), ("device_ns", ctypes.c_int64),
                ("grid_ctas", ctypes.c_int32),
                ("block", ctypes.c_int32), ("device_error", ctypes.c_int32),
                ("local_rounds", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class gbf_server_options(ctypes.Structure):
    _fields_ = [("bfs_engines", ctypes.c_int32), ("wbfs_engines", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("max_queue", ctypes.c_int32),
                ("hbm_budget", ctypes.c_size_t), ("kernel", gbf_options),
                ("min_batch", ctypes.c_int32), ("wbfs_share", ctypes.c_int32),
                ("always_batch", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class gbf_server_counters(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("pending", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("batched_queries", ctypes.c_uint64), ("free_slots", ctypes.c_uint64),
                ("engines", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class gbf_round_trace(ctypes.Structure):
    _fields_ = [("round", ctypes.c_int32), ("kind", ctypes.c_int32), ("frontier", ctypes.c_uint32),
                ("frontier_edges", ctypes.c_uint32), ("t_ns", ctypes.c_int64),
                ("t_mid_ns", ctypes.c_int64)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgbf.so is not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, U32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64
    S = ctypes.c_int
    sig = {
        "gbf_options_default": (S, [ctypes.POINTER(gbf_options)]),
        "gbf_last_error": (ctypes.c_size_t, [ctypes.c_char_p, ctypes.c_size_t]),
        "gbf_version": (ctypes.c_char_p, []),
        "gbf_graph_create": (S, [I32, P, P, P, ctypes.c_int, U32, P, ctypes.POINTER(P)]),
        "gbf_graph_destroy": (S, [P]),
        "gbf_graph_info": (S, [P, ctypes.POINTER(I32), ctypes.POINTER(U64), ctypes.POINTER(U32),
                               ctypes.POINTER(U64)]),
        "gbf_graph_device_bytes": (S, [P, ctypes.POINTER(ctypes.c_size_t)]),
        "gbf_bfs": (S, [P, I32, P, P, ctypes.c_int, ctypes.POINTER(gbf_options), P]),
        "gbf_bfs_host_batch": (S, [P, P, I32, P, P, ctypes.POINTER(gbf_options), P]),
        "gbf_wbfs": (S, [P, I32, P, ctypes.c_int, ctypes.POINTER(gbf_options), P]),
        "gbf_delta_stepping": (S, [P, I32, I32, P, ctypes.c_int, ctypes.POINTER(gbf_options), P]),
        "gbf_ldd": (S, [P, P, P, P, ctypes.c_int, ctypes.POINTER(gbf_options), P]),
        "gbf_connectivity": (S, [P, P, ctypes.c_int, ctypes.POINTER(gbf_options), P]),
        "gbf_bellman_ford": (S, [P, I32, P, ctypes.c_int, ctypes.POINTER(gbf_options), P]),
        "gbf_widest_path": (S, [P, I32, P, ctypes.c_int, ctypes.POINTER(gbf_options), P]),
        "gbf_betweenness": (S, [P, I32, P, ctypes.c_int, ctypes.POINTER(gbf_options), P]),
        "gbf_kcore": (S, [P, P, ctypes.c_int, ctypes.POINTER(gbf_options), P]),
        "gbf_wait": (S, [P, P, ctypes.POINTER(gbf_stats)]),
        "gbf_msbfs": (S, [P, P, I32, P, ctypes.c_int, ctypes.POINTER(gbf_options), P]),
        "gbf_mssp": (S, [P, P, I32, P, ctypes.c_int, ctypes.POINTER(gbf_options), P]),
        "gbf_server_options_default": (S, [ctypes.POINTER(gbf_server_options)]),
        "gbf_server_create": (S, [P, I32, ctypes.POINTER(gbf_server_options), ctypes.POINTER(P)]),
        "gbf_server_submit": (S, [P, I32, I32, I32, ctypes.POINTER(U64)]),
        "gbf_server_poll": (S, [P, U64, P, ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_double)]),
        "gbf_server_collect": (S, [P, P, P, P, I32, ctypes.POINTER(I32)]),
        "gbf_server_stats": (S, [P, ctypes.POINTER(gbf_server_counters)]),
        "gbf_server_destroy": (S, [P]),
        "gbf_autotune": (S, [P, I32, ctypes.POINTER(gbf_options)]),
        "gbf_trace": (S, [P, ctypes.POINTER(gbf_round_trace), I32, ctypes.POINTER(I32)]),
        "gbf_bfs_noalloc": (S, [I32, U32, P, P, I32, P, P, ctypes.POINTER(gbf_options), P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    _lib.gbf_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def _check(st: int, what: str) -> None:
    if st != 0:
        raise GbfError(st, f"{what}: {last_error()}")


def gbf_version() -> str:
    return _lib.gbf_version().decode()


def gbf_options_default(**overrides) -> gbf_options:
    o = gbf_options()
    _check(_lib.gbf_options_default(ctypes.byref(o)), "gbf_options_default")
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def _ptr(a):
    """(address, mem) of a numpy array (host) or a torch tensor (its device)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data, HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), (DEVICE if a.is_cuda else HOST)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def gbf_graph_create(n: int, off, tgt, w=None, validate: int = VALIDATE_BASIC, stream=None) -> int:
    """Make a CSR graph resident on the current device; returns the handle."""
    po, mem = _ptr(off)
    pt, mt = _ptr(tgt)
    pw, mw = _ptr(w)
    if (mt is not None and mt != mem) or (mw is not None and mw != mem):
        raise ValueError("off, tgt and w must all be host or all device buffers")
    h = ctypes.c_void_p()
    _check(_lib.gbf_graph_create(int(n), po, pt, pw, mem, validate, _stream(stream), ctypes.byref(h)),
           "gbf_graph_create")
    return h.value


def gbf_graph_destroy(h: int) -> None:
    _check(_lib.gbf_graph_destroy(h), "gbf_graph_destroy")


def gbf_graph_info(h: int) -> dict:
    n, m, wm, fp = ctypes.c_int32(), ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint64()
    _check(_lib.gbf_graph_info(h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(wm),
                               ctypes.byref(fp)), "gbf_graph_info")
    return {"n": n.value, "m": m.value, "w_max": wm.value, "fingerprint": fp.value}


def gbf_graph_device_bytes(h: int) -> int:
    b = ctypes.c_size_t()
    _check(_lib.gbf_graph_device_bytes(h, ctypes.byref(b)), "gbf_graph_device_bytes")
    return b.value


def _opt(opt):
    return None if opt is None else ctypes.byref(opt)


def gbf_bfs(h: int, src: int, dist, parent=None, opt: Optional[gbf_options] = None, stream=None) -> None:
    """BFS from src into dist (and parent): numpy arrays block; CUDA tensors are stream-ordered."""
    pd, mem = _ptr(dist)
    pp, mp = _ptr(parent)
    if mp is not None and mp != mem:
        raise ValueError("dist and parent must live in the same memory")
    _check(_lib.gbf_bfs(h, int(src), pd, pp, mem, _opt(opt), _stream(stream)), "gbf_bfs")


def _check_host_rows(name, a, k, n):
    """A C-contiguous host int32 array of k rows of n entries."""
    if not isinstance(a, np.ndarray) or a.dtype != np.int32 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"gbf_bfs_host_batch: {name} must be a contiguous int32 numpy array")
    if a.size != k * n:
        raise ValueError(f"gbf_bfs_host_batch: {name} holds {a.size} entries, needs {k} x {n}")


def gbf_bfs_host_batch(h: int, srcs, dist, parent=None, opt: Optional[gbf_options] = None,
                       stream=None) -> None:
    """BFS from each source into host rows dist[i] (and parent[i]), blocking;
    each row's read-back overlaps the next query (pinned arrays, e.g. from
    torch's pin_memory, let the copies run in the background)."""
    s = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    n = gbf_graph_info(h)["n"]
    _check_host_rows("dist", dist, int(s.size), n)
    if parent is not None:
        _check_host_rows("parent", parent, int(s.size), n)
    _check(_lib.gbf_bfs_host_batch(h, s.ctypes.data, int(s.size), dist.ctypes.data,
                                   None if parent is None else parent.ctypes.data, _opt(opt),
                                   _stream(stream)), "gbf_bfs_host_batch")


def gbf_wbfs(h: int, src: int, dist, opt: Optional[gbf_options] = None, stream=None) -> None:
    """Integral-weight SSSP from src into dist."""
    pd, mem = _ptr(dist)
    _check(_lib.gbf_wbfs(h, int(src), pd, mem, _opt(opt), _stream(stream)), "gbf_wbfs")


def gbf_delta_stepping(h: int, src: int, delta: int, dist, opt: Optional[gbf_options] = None,
                       stream=None) -> None:
    """Integral-weight SSSP from src into dist by Δ-stepping (delta a power of two)."""
    pd, mem = _ptr(dist)
    _check(_lib.gbf_delta_stepping(h, int(src), int(delta), pd, mem, _opt(opt), _stream(stream)),
           "gbf_delta_stepping")


def gbf_ldd(h: int, delta, cluster, rnd, opt: Optional[gbf_options] = None, stream=None) -> None:
    """Low-diameter decomposition with the given shifts (float64, one per
    vertex) into cluster (centres) and rnd (join rounds); all three in the
    same memory."""
    pd, md = _ptr(delta)
    pc, mc = _ptr(cluster)
    pr, mr = _ptr(rnd)
    if not (md == mc == mr):
        raise ValueError("delta, cluster and rnd must live in the same memory")
    _check(_lib.gbf_ldd(h, pd, pc, pr, mc, _opt(opt), _stream(stream)), "gbf_ldd")


def gbf_connectivity(h: int, label, opt: Optional[gbf_options] = None, stream=None) -> None:
    """Connected components into label (the smallest vertex id of each component)."""
    pl, mem = _ptr(label)
    _check(_lib.gbf_connectivity(h, pl, mem, _opt(opt), _stream(stream)), "gbf_connectivity")


def gbf_bellman_ford(h: int, src: int, dist, opt: Optional[gbf_options] = None,
                     stream=None) -> None:
    """General-weight SSSP from src by frontier Bellman-Ford rounds into dist."""
    pd, mem = _ptr(dist)
    _check(_lib.gbf_bellman_ford(h, int(src), pd, mem, _opt(opt), _stream(stream)),
           "gbf_bellman_ford")


def gbf_widest_path(h: int, src: int, width, opt: Optional[gbf_options] = None,
                    stream=None) -> None:
    """Single-source widest (bottleneck) path widths from src into width."""
    pd, mem = _ptr(width)
    _check(_lib.gbf_widest_path(h, int(src), pd, mem, _opt(opt), _stream(stream)),
           "gbf_widest_path")


def gbf_betweenness(h: int, src: int, dep, opt: Optional[gbf_options] = None,
                    stream=None) -> None:
    """Single-source betweenness dependencies from src into dep (float64)."""
    pd, mem = _ptr(dep)
    _check(_lib.gbf_betweenness(h, int(src), pd, mem, _opt(opt), _stream(stream)),
           "gbf_betweenness")


def gbf_kcore(h: int, core, opt: Optional[gbf_options] = None, stream=None) -> None:
    """Coreness of every vertex into core (int32)."""
    pd, mem = _ptr(core)
    _check(_lib.gbf_kcore(h, pd, mem, _opt(opt), _stream(stream)), "gbf_kcore")


def gbf_msbfs(h: int, srcs, dist, opt: Optional[gbf_options] = None, stream=None) -> None:
    """Multi-source BFS from k <= 64 sources into dist[k, n] (row i = source i)."""
    s = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    pd, mem = _ptr(dist)
    _check(_lib.gbf_msbfs(h, s.ctypes.data, int(s.size), pd, mem, _opt(opt), _stream(stream)),
           "gbf_msbfs")


def gbf_mssp(h: int, srcs, dist, opt: Optional[gbf_options] = None, stream=None) -> None:
    """Weighted shortest paths from k <= 8 sources into dist[k, n] (row i = source i)."""
    s = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    pd, mem = _ptr(dist)
    _check(_lib.gbf_mssp(h, s.ctypes.data, int(s.size), pd, mem, _opt(opt), _stream(stream)),
           "gbf_mssp")


TUNE_BFS, TUNE_MSBFS, TUNE_WBFS = 0, 1, 2


def gbf_autotune(h: int, kind: int = TUNE_BFS) -> gbf_options:
    """Time the knob grid on this graph and return the fastest options."""
    o = gbf_options()
    _check(_lib.gbf_autotune(h, int(kind), ctypes.byref(o)), "gbf_autotune")
    return o


def gbf_wait(h: int, stream=None) -> dict:
    """Synchronise and return the statistics of the last device-memory query."""
    s = gbf_stats()
    _check(_lib.gbf_wait(h, _stream(stream), ctypes.byref(s)), "gbf_wait")
    return s.as_dict()


def gbf_trace(h: int, cap: int = 1 << 16) -> list:
    """Per-round records (round, kind, frontier, frontier_edges, t_ns, t_mid_ns) of the last query."""
    buf = (gbf_round_trace * cap)()
    cnt = ctypes.c_int32()
    _check(_lib.gbf_trace(h, buf, cap, ctypes.byref(cnt)), "gbf_trace")
    return [(r.round, r.kind, r.frontier, r.frontier_edges, r.t_ns, r.t_mid_ns)
            for r in buf[:cnt.value]]


def _check_device_i32(name, t, count):
    """A contiguous CUDA tensor of 4-byte integers holding at least count entries."""
    if not hasattr(t, "is_cuda") or not t.is_cuda:
        raise ValueError(f"gbf_bfs_noalloc: {name} must be a CUDA tensor")
    if t.element_size() != 4 or t.dtype.is_floating_point:
        raise ValueError(f"gbf_bfs_noalloc: {name} must hold 32-bit integers")
    if t.numel() < count:
        raise ValueError(f"gbf_bfs_noalloc: {name} holds {t.numel()} entries, needs {count}")


def gbf_bfs_noalloc(n: int, m: int, off, tgt, src: int, dist, parent=None,
                    opt: Optional[gbf_options] = None, stream=None) -> None:
    """BFS on a caller-held device CSR with no device allocation (blocks).
    The buffers' lengths are checked here against n and m, since the C call
    cannot see them."""
    if 1 <= int(n) <= (1 << 20) and 0 <= int(m) <= (1 << 25):
        _check_device_i32("off", off, int(n) + 1)
        _check_device_i32("tgt", tgt, max(int(m), 1))
        _check_device_i32("dist", dist, int(n))
        if parent is not None:
            _check_device_i32("parent", parent, int(n))
    po, mo = _ptr(off)
    pt, mt = _ptr(tgt)
    pd, md = _ptr(dist)
    pp, mp = _ptr(parent)
    for mm in (mo, mt, md, mp):
        if mm is not None and mm != DEVICE:
            raise ValueError("gbf_bfs_noalloc takes device buffers only")
    _check(_lib.gbf_bfs_noalloc(int(n), int(m), po, pt, int(src), pd, pp, _opt(opt),
                                _stream(stream)), "gbf_bfs_noalloc")


QUERY_BFS, QUERY_WBFS = 0, 1


def gbf_server_options_default(**overrides) -> gbf_server_options:
    o = gbf_server_options()
    _check(_lib.gbf_server_options_default(ctypes.byref(o)), "gbf_server_options_default")
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def gbf_server_create(graphs: Sequence[int], opt: Optional[gbf_server_options] = None) -> int:
    arr = (ctypes.c_void_p * len(graphs))(*graphs)
    h = ctypes.c_void_p()
    _check(_lib.gbf_server_create(arr, len(graphs), None if opt is None else ctypes.byref(opt),
                                  ctypes.byref(h)), "gbf_server_create")
    return h.value


def gbf_server_submit(s: int, graph_idx: int, kind: int, src: int):
    """Returns the ticket, or None if the server is busy (GBF_ERR_BUSY)."""
    t = ctypes.c_uint64()
    st = _lib.gbf_server_submit(s, int(graph_idx), int(kind), int(src), ctypes.byref(t))
    if st == 6:
        return None
    _check(st, "gbf_server_submit")
    return t.value


def gbf_server_poll(s: int, ticket: int, dist=None):
    """Returns (done, latency_us); fills dist (numpy int32[n]) when done."""
    done = ctypes.c_int32()
    lat = ctypes.c_double()
    pd = None if dist is None else _ptr(dist)[0]
    _check(_lib.gbf_server_poll(s, ctypes.c_uint64(ticket), pd, ctypes.byref(done),
                                ctypes.byref(lat)), "gbf_server_poll")
    return bool(done.value), lat.value


def gbf_server_collect(s: int, cap: int = 65536):
    """Release finished queries without copying results: (tickets, latency_us, status)."""
    t = np.empty(cap, dtype=np.uint64)
    lat = np.empty(cap, dtype=np.float64)
    stt = np.empty(cap, dtype=np.int32)
    cnt = ctypes.c_int32()
    _check(_lib.gbf_server_collect(s, t.ctypes.data, lat.ctypes.data, stt.ctypes.data, cap,
                                   ctypes.byref(cnt)), "gbf_server_collect")
    k = cnt.value
    return t[:k], lat[:k], stt[:k]


def gbf_server_stats(s: int) -> dict:
    o = gbf_server_counters()
    _check(_lib.gbf_server_stats(s, ctypes.byref(o)), "gbf_server_stats")
    return o.as_dict()


def gbf_server_destroy(s: int) -> None:
    _check(_lib.gbf_server_destroy(s), "gbf_server_destroy")


class Graph:
    """Owning wrapper around a resident graph handle."""

    def __init__(self, csr=None, *, n=None, off=None, tgt=None, w=None,
                 validate: int = VALIDATE_BASIC, stream=None):
        if csr is not None:
            n, off, tgt, w = csr.n, csr.off, csr.tgt, csr.w
        off = np.ascontiguousarray(off, dtype=np.uint32) if isinstance(off, np.ndarray) else off
        tgt = np.ascontiguousarray(tgt, dtype=np.int32) if isinstance(tgt, np.ndarray) else tgt
        if isinstance(w, np.ndarray):
            w = np.ascontiguousarray(w, dtype=np.uint32)
        if isinstance(tgt, np.ndarray) and tgt.size == 0:
            tgt = np.zeros(1, dtype=np.int32)
            if w is not None:
                w = np.ones(1, dtype=np.uint32)
        self.h = gbf_graph_create(n, off, tgt, w, validate, stream)
        info = gbf_graph_info(self.h)
        self.n, self.m, self.w_max, self.fingerprint = info["n"], info["m"], info["w_max"], info["fingerprint"]

    def close(self):
        if getattr(self, "h", None):
            gbf_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bfs(self, src: int, parents: bool = True, opt=None):
        d = np.empty(self.n, dtype=np.int32)
        p = np.empty(self.n, dtype=np.int32) if parents else None
        gbf_bfs(self.h, src, d, p, opt)
        return d, p

    def msbfs(self, srcs, opt=None):
        d = np.empty((len(srcs), self.n), dtype=np.int32)
        gbf_msbfs(self.h, srcs, d, opt)
        return d

    def mssp(self, srcs, opt=None):
        d = np.empty((len(srcs), self.n), dtype=np.int32)
        gbf_mssp(self.h, srcs, d, opt)
        return d

    def wbfs(self, src: int, opt=None):
        d = np.empty(self.n, dtype=np.int32)
        gbf_wbfs(self.h, src, d, opt)
        return d

    def delta_stepping(self, src: int, delta: int, opt=None):
        d = np.empty(self.n, dtype=np.int32)
        gbf_delta_stepping(self.h, src, delta, d, opt)
        return d

    def connectivity(self, opt=None):
        lab = np.empty(self.n, dtype=np.int32)
        gbf_connectivity(self.h, lab, opt)
        return lab

    def ldd(self, delta, opt=None):
        d = np.ascontiguousarray(delta, dtype=np.float64)
        c = np.empty(self.n, dtype=np.int32)
        t = np.empty(self.n, dtype=np.int32)
        gbf_ldd(self.h, d, c, t, opt)
        return c, t

    def bellman_ford(self, src: int, opt=None):
        d = np.empty(self.n, dtype=np.int32)
        gbf_bellman_ford(self.h, src, d, opt)
        return d

    def widest_path(self, src: int, opt=None):
        d = np.empty(self.n, dtype=np.int32)
        gbf_widest_path(self.h, src, d, opt)
        return d

    def betweenness(self, src: int, opt=None):
        d = np.empty(self.n, dtype=np.float64)
        gbf_betweenness(self.h, src, d, opt)
        return d

    def kcore(self, opt=None):
        d = np.empty(self.n, dtype=np.int32)
        gbf_kcore(self.h, d, opt)
        return d

    def stats(self, stream=None) -> dict:
        return gbf_wait(self.h, stream)

    def device_bytes(self) -> int:
        return gbf_graph_device_bytes(self.h)
