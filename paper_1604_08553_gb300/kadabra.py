"""Thin Python binding of ``libkadabra.so`` (the C ABI in include/kadabra.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels (or, for computeDelta and omega, in the library's own host
code).  There is no CPU fallback: if the library cannot be loaded, every call
raises.  PyTorch is used only for device memory and streams (tensors whose
pointers are passed to the ``*_device`` / ``d_*`` arguments, and
``torch.cuda.current_stream()``).

Function names mirror the C ABI.
"""

from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import _build

_lock = threading.Lock()
_lib = None

OK = 0
ERR_ARG = 1
ERR_CSR = 2
ERR_OOM = 3
ERR_SIGMA_OVERFLOW = 4
ERR_CAPACITY = 5
ERR_TIMEOUT = 6
ERR_CUDA = 7
ERR_UNSUPPORTED = 8
ERR_INTERNAL = 9

STAT_NAMES = (
    "edges", "expanded", "new", "sigma_adds", "pi", "levels",
    "bt_scanned", "path_nodes", "sigma_lo", "sigma_hi", "dist",
)
NSTAT = len(STAT_NAMES)
FLAG_GLOBAL_TABLES = 1
FLAG_MEDIUM_TABLES = 2
FLAG_LARGE_SHARED_TABLES = 4
FLAG_WARP_TIER = 8
FLAG_ASYNC_SCAN = 16
FLAG_FRONTIER_SEGMENTS = 32
FLAG_COMPACT_TABLES = 64


class KadabraError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"kadabra status {status}: {msg}")
        self.status = status


class kadabra_config(C.Structure):
    _fields_ = [
        ("vd", C.c_int64), ("eps", C.c_double), ("check_interval", C.c_uint64),
        ("stream", C.c_void_p), ("ctas_per_sm", C.c_int32), ("warp_tier", C.c_int32), ("reserved", C.c_int32 * 6),
    ]


class kadabra_result(C.Structure):
    _fields_ = [
        ("tau", C.c_uint64), ("omega_cap", C.c_uint64), ("alpha", C.c_uint64), ("checks", C.c_uint64),
        ("vd", C.c_int64), ("omega", C.c_double), ("C", C.c_double), ("max_f", C.c_double),
        ("max_g", C.c_double), ("totals", C.c_int64 * NSTAT), ("check_interval", C.c_uint64),
        ("stopped_early", C.c_int32),
        ("status", C.c_int32), ("counts", C.c_void_p), ("btilde", C.c_void_p), ("d_counts", C.c_void_p),
        ("d_btilde", C.c_void_p), ("topk", C.c_void_p),
        ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
        ("ctas_per_sm", C.c_int32), ("warp_tier", C.c_int32),
    ]


def load_library():
    """Builds (if needed) and loads libkadabra.so; raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build_kadabra()
        if not os.path.exists(path):
            raise RuntimeError(f"libkadabra.so missing at {path}")
        lib = C.CDLL(path)
        p = C.c_void_p
        i32, i64, u32, u64, dbl = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
        st = C.c_int
        lib.kadabra_last_error.restype = C.c_char_p
        lib.kadabra_config_default.argtypes = [C.POINTER(kadabra_config)]
        lib.kadabra_omega.argtypes = [dbl, dbl, i64]
        lib.kadabra_omega.restype = dbl
        lib.kadabra_load_csr.argtypes = [i32, i64, p, p, C.c_int, p, p, C.POINTER(C.c_void_p)]
        lib.kadabra_load_csr.restype = st
        lib.kadabra_load_csr_device.argtypes = [i32, i64, p, p, C.c_int, p, p, C.POINTER(C.c_void_p)]
        lib.kadabra_load_csr_device.restype = st
        lib.kadabra_free_graph.argtypes = [p]
        lib.kadabra_graph_info.argtypes = [p, C.POINTER(i32), C.POINTER(i64), C.POINTER(C.c_int), C.POINTER(i64)]
        lib.kadabra_graph_info.restype = st
        lib.kadabra_graph_set_flags.argtypes = [p, u32]
        lib.kadabra_graph_set_flags.restype = st
        lib.kadabra_run.argtypes = [p, dbl, dbl, i32, u64, C.POINTER(kadabra_config), C.POINTER(kadabra_result)]
        lib.kadabra_run.restype = st
        lib.kadabra_sample_batch.argtypes = [p, u64, u32, u64, u64, p, p, p]
        lib.kadabra_sample_batch.restype = st
        lib.kadabra_sample_batch_noalloc.argtypes = [i32, i64, p, p, C.c_int, p, p, u64, u32, u64, u64, p, p, p]
        lib.kadabra_sample_batch_noalloc.restype = st
        lib.kadabra_sync_status.argtypes = [p, p]
        lib.kadabra_sync_status.restype = st
        lib.kadabra_sample_paths.argtypes = [p, u64, u32, u64, u32, p, p, p, i32, p, p]
        lib.kadabra_sample_paths.restype = st
        lib.kadabra_philox.argtypes = [u64, u32, u32, u64, u32, p]
        lib.kadabra_philox.restype = st
        lib.kadabra_check.argtypes = [i64, p, u64, dbl, p, p, dbl, C.POINTER(dbl), C.POINTER(dbl),
                                      C.POINTER(C.c_int)]
        lib.kadabra_check.restype = st
        lib.kadabra_compute_delta.argtypes = [i64, p, u64, dbl, dbl, dbl, dbl, p, p, C.POINTER(dbl)]
        lib.kadabra_compute_delta.restype = st
        pp = C.POINTER(C.c_void_p)
        lib.kadabra_load_batch.argtypes = [i32, p, p, p, p, p, p, p, C.POINTER(C.c_void_p)]
        lib.kadabra_load_batch.restype = st
        lib.kadabra_free_batch.argtypes = [p]
        lib.kadabra_batch_graph.argtypes = [p, i32, C.POINTER(C.c_void_p)]
        lib.kadabra_batch_graph.restype = st
        lib.kadabra_run_batch.argtypes = [p, p, p, p, C.POINTER(kadabra_config), p]
        lib.kadabra_run_batch.restype = st
        lib.kadabra_serve_configure.argtypes = [u64, i32]
        lib.kadabra_serve_configure.restype = st
        lib.kadabra_submit.argtypes = [p, dbl, dbl, i32, u64, C.POINTER(kadabra_config), C.POINTER(u64)]
        lib.kadabra_submit.restype = st
        lib.kadabra_poll.argtypes = [u64, i32, C.POINTER(i32), C.POINTER(kadabra_result)]
        lib.kadabra_poll.restype = st
        lib.kadabra_l2_read_probe.argtypes = [u64, i32, C.POINTER(dbl)]
        lib.kadabra_l2_read_probe.restype = st
        lib.kadabra_serve_shutdown.argtypes = []
        lib.kadabra_serve_shutdown.restype = None
        lib.kadabra_release_cached.argtypes = []
        lib.kadabra_release_cached.restype = None
        _lib = lib
        return lib


def _raise(status: int):
    if status != OK:
        msg = load_library().kadabra_last_error().decode(errors="replace")
        raise KadabraError(status, msg)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def config_default() -> kadabra_config:
    cfg = kadabra_config()
    load_library().kadabra_config_default(C.byref(cfg))
    return cfg


def kadabra_omega(lam: float, delta: float, vd: int) -> float:
    return float(load_library().kadabra_omega(lam, delta, vd))


class Graph:
    """Owns a kadabra_graph handle (device-resident CSR + sampler workspace)."""

    def __init__(self, handle: int, n: int, m: int, directed: bool, keepalive=None):
        self.handle = C.c_void_p(handle)
        self.n, self.m, self.directed = n, m, directed
        self._keepalive = keepalive

    @property
    def vd(self) -> int:
        vd = C.c_int64()
        _raise(load_library().kadabra_graph_info(self.handle, None, None, None, C.byref(vd)))
        return vd.value

    def set_flags(self, flags: int) -> None:
        _raise(load_library().kadabra_graph_set_flags(self.handle, flags))

    def free(self):
        if self.handle:
            load_library().kadabra_free_graph(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def kadabra_load_csr(g) -> Graph:
    """Copies a host CSR (an object with n, row_ptr, col, directed, rrow_ptr, rcol) to the device."""
    lib = load_library()
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(g.col, dtype=np.int32)
    rrp = np.ascontiguousarray(g.rrow_ptr, dtype=np.int32) if g.directed else None
    rci = np.ascontiguousarray(g.rcol, dtype=np.int32) if g.directed else None
    h = C.c_void_p()
    _raise(lib.kadabra_load_csr(int(g.n), int(ci.shape[0]), _ptr(rp), _ptr(ci), int(bool(g.directed)),
                                _ptr(rrp), _ptr(rci), C.byref(h)))
    return Graph(h.value, int(g.n), int(ci.shape[0]), bool(g.directed))


def kadabra_load_csr_device(n: int, row_ptr, col, directed: bool = False, rrow_ptr=None, rcol=None) -> Graph:
    """Wraps int32 CUDA tensors (not copied; kept alive by the returned Graph)."""
    lib = load_library()
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    h = C.c_void_p()
    _raise(lib.kadabra_load_csr_device(int(n), int(col.numel()), ptr(row_ptr), ptr(col), int(bool(directed)),
                                       ptr(rrow_ptr), ptr(rcol), C.byref(h)))
    return Graph(h.value, int(n), int(col.numel()), bool(directed), keepalive=(row_ptr, col, rrow_ptr, rcol))


@dataclass
class RunResult:
    tau: int
    check_interval: int
    omega_cap: int
    alpha: int
    checks: int
    vd: int
    omega: float
    C: float
    max_f: float
    max_g: float
    totals: np.ndarray
    stopped_early: bool
    counts: Optional[np.ndarray]
    btilde: Optional[np.ndarray]
    topk: Optional[np.ndarray] = None
    ctas_per_sm: int = 0
    warp_tier: int = 0


def kadabra_run(g: Graph, lam: float, delta: float, k: int = 0, seed: int = 0, *, vd: int = 0,
                eps: float = 0.001, check_interval: int = 1000, stream: Optional[int] = None,
                counts: Optional[np.ndarray] = None, btilde: Optional[np.ndarray] = None,
                d_counts=None, d_btilde=None, want_host: bool = True, ctas_per_sm: int = 0,
                warp_tier: int = 0) -> RunResult:
    """Runs KADABRA: all-nodes mode (k = 0), or the k most central nodes
    (k > 0; the ranking's k first nodes come back in `topk`).  Host outputs
    are numpy arrays (allocated here unless given); device outputs are
    optional CUDA tensors."""
    lib = load_library()
    cfg = config_default()
    cfg.vd = vd
    cfg.eps = eps
    cfg.check_interval = check_interval
    cfg.stream = stream
    cfg.ctas_per_sm = ctas_per_sm
    cfg.warp_tier = warp_tier
    res = kadabra_result()
    if want_host:
        if counts is None:
            counts = np.zeros(g.n, dtype=np.uint32)
        if btilde is None:
            btilde = np.zeros(g.n, dtype=np.float64)
        res.counts = counts.ctypes.data
        res.btilde = btilde.ctypes.data
    if d_counts is not None:
        res.d_counts = d_counts.data_ptr()
    if d_btilde is not None:
        res.d_btilde = d_btilde.data_ptr()
    topk = None
    if k > 0:
        topk = np.full(k, -1, dtype=np.int32)
        res.topk = topk.ctypes.data
    _raise(lib.kadabra_run(g.handle, lam, delta, k, seed, C.byref(cfg), C.byref(res)))
    if topk is not None:
        topk = topk[:min(k, g.n)]
    return RunResult(res.tau, res.check_interval, res.omega_cap, res.alpha, res.checks, res.vd, res.omega, res.C, res.max_f,
                     res.max_g, np.array(res.totals[:], dtype=np.int64), bool(res.stopped_early),
                     counts if want_host else None, btilde if want_host else None, topk, res.ctas_per_sm,
                     res.warp_tier)


def kadabra_serve_configure(budget_bytes: int = 0, max_active: int = 256) -> None:
    """Memory budget and slot count of the serving engine (before the first submit)."""
    _raise(load_library().kadabra_serve_configure(int(budget_bytes), int(max_active)))


def kadabra_submit(g: Graph, lam: float, delta: float, k: int = 0, seed: int = 0, *, vd: int = 0,
                   eps: float = 0.001, check_interval: int = 1000) -> int:
    """Queues a run on the serving engine; returns its job id at once."""
    lib = load_library()
    cfg = config_default()
    cfg.vd = vd
    cfg.eps = eps
    cfg.check_interval = check_interval
    job = C.c_uint64()
    _raise(lib.kadabra_submit(g.handle, lam, delta, k, seed, C.byref(cfg), C.byref(job)))
    return job.value


@dataclass
class ServedResult(RunResult):
    t_submit: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0


def kadabra_poll(job: int, n: int, k: int = 0, wait: bool = True) -> Optional[ServedResult]:
    """The job's result (collecting it), or None if it has not finished and
    wait is False.  n is the graph's node count, k the job's k."""
    lib = load_library()
    res = kadabra_result()
    counts = np.zeros(n, dtype=np.uint32)
    btilde = np.zeros(n, dtype=np.float64)
    res.counts = counts.ctypes.data
    res.btilde = btilde.ctypes.data
    topk = None
    if k > 0:
        topk = np.full(k, -1, dtype=np.int32)
        res.topk = topk.ctypes.data
    done = C.c_int32()
    _raise(lib.kadabra_poll(job, int(bool(wait)), C.byref(done), C.byref(res)))
    if not done.value:
        return None
    if topk is not None:
        topk = topk[:min(k, n)]
    return ServedResult(res.tau, res.check_interval, res.omega_cap, res.alpha, res.checks, res.vd, res.omega, res.C,
                        res.max_f, res.max_g, np.array(res.totals[:], dtype=np.int64), bool(res.stopped_early),
                        counts, btilde, topk, t_submit=res.t_submit, t_start=res.t_start, t_done=res.t_done)


def kadabra_l2_read_probe(nbytes: int = 32 << 20, reps: int = 50) -> float:
    """Read rate (GB/s) of an L2-resident buffer, for the L2 roofline."""
    out = C.c_double()
    _raise(load_library().kadabra_l2_read_probe(int(nbytes), int(reps), C.byref(out)))
    return out.value


def kadabra_serve_shutdown() -> None:
    load_library().kadabra_serve_shutdown()


def kadabra_release_cached() -> None:
    """Frees the sampler workspaces the library keeps for reuse after kadabra_free_graph."""
    load_library().kadabra_release_cached()


def kadabra_sample_batch(g: Graph, seed: int, domain: int, first_idx: int, count: int, d_counts,
                         d_totals=None, stream: Optional[int] = None) -> None:
    """Enqueues one sampler batch; d_counts (uint32/int32, n) and d_totals (int64, NSTAT) are CUDA tensors."""
    lib = load_library()
    _raise(lib.kadabra_sample_batch(g.handle, seed, domain, first_idx, count, C.c_void_p(d_counts.data_ptr()),
                                    None if d_totals is None else C.c_void_p(d_totals.data_ptr()), stream))


def kadabra_sample_batch_noalloc(n: int, row_ptr, col, seed: int, domain: int, first_idx: int, count: int,
                                 d_counts, d_totals=None, directed: bool = False, rrow_ptr=None, rcol=None,
                                 stream: Optional[int] = None) -> None:
    """The sampler batch without device allocation, from int32 CUDA tensors
    of a CSR (see include/kadabra.h for its limits).  Blocking."""
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    _raise(load_library().kadabra_sample_batch_noalloc(
        int(n), int(col.numel()), ptr(row_ptr), ptr(col), int(bool(directed)), ptr(rrow_ptr), ptr(rcol), seed,
        domain, first_idx, count, ptr(d_counts), ptr(d_totals), stream))


def kadabra_sync_status(g: Graph, stream: Optional[int] = None) -> None:
    _raise(load_library().kadabra_sync_status(g.handle, stream))


@dataclass
class Samples:
    st: np.ndarray
    path_len: np.ndarray
    paths: np.ndarray
    stats: np.ndarray
    status: np.ndarray

    def stat(self, name: str) -> np.ndarray:
        return self.stats[:, STAT_NAMES.index(name)]


def kadabra_sample_paths(g: Graph, seed: int, domain: int, first_idx: int, count: int,
                         max_len: int = 64, raise_on_error: bool = True):
    """Per-sample (s,t), paths, work counters and status.  With
    raise_on_error=False returns (Samples, status) instead of raising."""
    lib = load_library()
    st = np.zeros((count, 2), dtype=np.int32)
    pl = np.zeros(count, dtype=np.int32)
    paths = np.full((count, max_len), -1, dtype=np.int32)
    stats = np.zeros((count, NSTAT), dtype=np.int64)
    status = np.zeros(count, dtype=np.int32)
    rc = lib.kadabra_sample_paths(g.handle, seed, domain, first_idx, count, _ptr(st), _ptr(pl), _ptr(paths),
                                  max_len, _ptr(stats), _ptr(status))
    smp = Samples(st, pl, paths, stats, status)
    if not raise_on_error:
        return smp, rc
    _raise(rc)
    return smp


def kadabra_philox(seed: int, domain: int, j: int, first_idx: int, count: int) -> np.ndarray:
    out = np.zeros((count, 4), dtype=np.uint32)
    _raise(load_library().kadabra_philox(seed, domain, j, first_idx, count, _ptr(out)))
    return out


def kadabra_check(counts: np.ndarray, tau: int, omega: float, ln_inv_dl: np.ndarray, ln_inv_du: np.ndarray,
                  lam: float):
    c = np.ascontiguousarray(counts, dtype=np.uint32)
    L = np.ascontiguousarray(ln_inv_dl, dtype=np.float64)
    U = np.ascontiguousarray(ln_inv_du, dtype=np.float64)
    mf, mg, stop = C.c_double(), C.c_double(), C.c_int()
    _raise(load_library().kadabra_check(c.shape[0], _ptr(c), tau, omega, _ptr(L), _ptr(U), lam, C.byref(mf),
                                        C.byref(mg), C.byref(stop)))
    return bool(stop.value), mf.value, mg.value


def kadabra_compute_delta(count0: np.ndarray, alpha: int, omega: float, lam: float, delta: float, eps: float):
    c0 = np.ascontiguousarray(count0, dtype=np.uint32)
    n = c0.shape[0]
    dl = np.zeros(n, dtype=np.float64)
    du = np.zeros(n, dtype=np.float64)
    Cv = C.c_double()
    _raise(load_library().kadabra_compute_delta(n, _ptr(c0), alpha, omega, lam, delta, eps, _ptr(dl), _ptr(du),
                                                C.byref(Cv)))
    return Cv.value, dl, du


class Batch:
    """G graphs in one device arena, run together (kadabra_load_batch / kadabra_run_batch)."""

    def __init__(self, graphs):
        lib = load_library()
        G = len(graphs)
        self._keep = []
        arr = lambda t, vals: (t * G)(*vals)
        rp = [np.ascontiguousarray(g.row_ptr, dtype=np.int32) for g in graphs]
        ci = [np.ascontiguousarray(g.col, dtype=np.int32) for g in graphs]
        rrp = [np.ascontiguousarray(g.rrow_ptr, dtype=np.int32) if g.directed else None for g in graphs]
        rci = [np.ascontiguousarray(g.rcol, dtype=np.int32) if g.directed else None for g in graphs]
        self._keep = (rp, ci, rrp, rci)
        n = arr(C.c_int32, [int(g.n) for g in graphs])
        m = arr(C.c_int64, [int(c.shape[0]) for c in ci])
        d = arr(C.c_int, [int(bool(g.directed)) for g in graphs])
        ptrs = lambda xs: arr(C.c_void_p, [None if x is None else x.ctypes.data for x in xs])
        h = C.c_void_p()
        _raise(lib.kadabra_load_batch(G, n, m, ptrs(rp), ptrs(ci), d, ptrs(rrp), ptrs(rci), C.byref(h)))
        self.handle = h
        self.G = G
        self.n = [int(g.n) for g in graphs]
        self.views = []
        for i, g in enumerate(graphs):
            v = C.c_void_p()
            _raise(lib.kadabra_batch_graph(h, i, C.byref(v)))
            gv = Graph(v.value, int(g.n), int(ci[i].shape[0]), bool(g.directed))
            gv.free = lambda: None  # released with the batch
            self.views.append(gv)

    def run(self, lam, delta, seed, *, check_interval: int = 0, eps: float = 0.001,
            stream: Optional[int] = None, d_counts=None, d_btilde=None, want_host: bool = True):
        """KADABRA on every graph; lam/delta/seed are sequences of length G.
        Host outputs are numpy arrays allocated here (want_host); d_counts /
        d_btilde are optional sequences of G CUDA tensors (n_i int32 / float64)
        that receive the results on the device."""
        lib = load_library()
        G = self.G
        cfg = config_default()
        cfg.eps = eps
        cfg.check_interval = check_interval
        cfg.stream = stream
        res = (kadabra_result * G)()
        counts = [np.zeros(n, dtype=np.uint32) for n in self.n] if want_host else [None] * G
        btilde = [np.zeros(n, dtype=np.float64) for n in self.n] if want_host else [None] * G
        for i in range(G):
            if want_host:
                res[i].counts = counts[i].ctypes.data
                res[i].btilde = btilde[i].ctypes.data
            if d_counts is not None:
                res[i].d_counts = d_counts[i].data_ptr()
            if d_btilde is not None:
                res[i].d_btilde = d_btilde[i].data_ptr()
        L = (C.c_double * G)(*lam)
        D = (C.c_double * G)(*delta)
        S = (C.c_uint64 * G)(*seed)
        _raise(lib.kadabra_run_batch(self.handle, L, D, S, C.byref(cfg), res))
        return [RunResult(r.tau, r.check_interval, r.omega_cap, r.alpha, r.checks, r.vd, r.omega, r.C, r.max_f,
                          r.max_g, np.array(r.totals[:], dtype=np.int64), bool(r.stopped_early), counts[i],
                          btilde[i]) for i, r in enumerate(res)]

    def free(self):
        if self.handle:
            load_library().kadabra_free_batch(self.handle)
            self.handle = C.c_void_p()
            self.views = []

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
