"""KADABRA oracle: Python binding of the plain single-threaded C++ oracle.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The oracle shares no code
with the CUDA path (``paper_1604_08553_gb300``) and neither imports the other;
both consume graphs from the input generators.

Function-by-function citations (Borassi & Natale, KADABRA):
  * ``sample_paths`` / ``sample_fixed_pair`` -- Sec. 4 balanced bidirectional
    BFS, candidate-edge choice and backtracking; Sec. 2 hit variables.
  * ``omega``            -- Alg. 1 first line (omega with c = 0.5).
  * ``vd_bound``         -- the vertex-diameter bound omega needs (Alg. 1,
    Sec. 2), from the condensation into strongly connected components.
  * ``compute_delta``    -- Alg. 2 and App. D.
  * ``f_and_g`` / ``check_stop`` -- Thm. 2 (f, g) and the all-nodes rule.
  * ``run``              -- Alg. 1 with the stop test every K samples.
  * ``brandes``          -- exact normalised betweenness (Sec. 2 definition).
  * ``enumerate_paths``  -- brute force over all shortest paths (tests only).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kadabra_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_ARG = 1
ERR_SIGMA_OVERFLOW = 4
ERR_CAPACITY = 5
ERR_INTERNAL = 99

# per-sample work counters, in the order the C++ side writes them
STAT_NAMES = (
    "edges", "expanded", "new", "sigma_adds", "pi", "levels",
    "bt_scanned", "path_nodes", "sigma_lo", "sigma_hi", "dist",
)


def build(force: bool = False) -> str:
    """Compiles the oracle (plain g++, FP contraction off) into oracle/liboracle.so."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


class orc_result(C.Structure):
    _fields_ = [
        ("tau", C.c_uint64), ("omega_cap", C.c_uint64), ("alpha", C.c_uint64),
        ("checks", C.c_uint64), ("vd", C.c_int64), ("omega", C.c_double),
        ("C", C.c_double), ("max_f", C.c_double), ("max_g", C.c_double),
        ("edges_warm", C.c_int64), ("edges_main", C.c_int64),
        ("stopped_early", C.c_int32), ("status", C.c_int32),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        p = C.c_void_p
        i64, u64, u32, i32, dbl = C.c_int64, C.c_uint64, C.c_uint32, C.c_int32, C.c_double
        graph = [i64, p, p, C.c_int, p, p]
        lib.orc_philox.argtypes = [u64, u32, u64, u32, p]
        lib.orc_philox_raw.argtypes = [u32, u32, p, p]
        lib.orc_philox_many.argtypes = [u64, u32, u32, u64, i64, p]
        lib.orc_scale128.argtypes = [p, u64]
        lib.orc_scale128.restype = u64
        lib.orc_stat_count.restype = C.c_int
        lib.orc_sample_paths.argtypes = graph + [u64, u32, u64, i64, p, p, p, i32, p, p]
        lib.orc_sample_fixed_pair.argtypes = graph + [i32, i32, u64, u32, u64, i64, p, p, i32, p]
        lib.orc_accumulate.argtypes = graph + [u64, u32, u64, i64, p, p]
        lib.orc_omega.argtypes = [dbl, dbl, i64]
        lib.orc_omega.restype = dbl
        lib.orc_vd_bound.argtypes = graph
        lib.orc_vd_bound.restype = i64
        lib.orc_compute_delta.argtypes = [i64, p, u64, dbl, dbl, dbl, dbl, p, p]
        lib.orc_compute_delta.restype = dbl
        lib.orc_f_and_g.argtypes = [u32, u64, dbl, dbl, dbl, p, p]
        lib.orc_check_stop.argtypes = [i64, p, u64, dbl, p, p, dbl, p, p]
        lib.orc_run.argtypes = graph + [dbl, dbl, u64, u64, i64, dbl, p, p, p, p, C.POINTER(orc_result)]
        lib.orc_run_topk.argtypes = graph + [dbl, dbl, u64, u64, i64, dbl, i64, p, p, p, p, p, p, p, p,
                                             C.POINTER(orc_result)]
        lib.orc_compute_delta_lv.argtypes = [i64, p, u64, dbl, p, p, dbl, dbl, p, p]
        lib.orc_compute_delta_lv.restype = dbl
        lib.orc_topk_lambdas.argtypes = [i64, p, u64, i64, dbl, p, p]
        lib.orc_check_stop_topk.argtypes = [i64, p, u64, dbl, p, p, dbl, i64, p, p, p]
        lib.orc_brandes.argtypes = graph + [p]
        lib.orc_enumerate_paths.argtypes = graph + [i32, i32, i64, i32, p]
        lib.orc_enumerate_paths.restype = i64
        assert lib.orc_stat_count() == len(STAT_NAMES)
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _gargs(g):
    """Marshals a graph object with n/row_ptr/col/directed/rrow_ptr/rcol."""
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(g.col, dtype=np.int32)
    if g.directed:
        rrp = np.ascontiguousarray(g.rrow_ptr, dtype=np.int32)
        rci = np.ascontiguousarray(g.rcol, dtype=np.int32)
    else:
        rrp, rci = rp, ci
    keep = (rp, ci, rrp, rci)
    return keep, [int(g.n), _ptr(rp), _ptr(ci), int(bool(g.directed)), _ptr(rrp), _ptr(rci)]


def philox(seed: int, domain: int, idx: int, j: int) -> np.ndarray:
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox(seed, domain, idx, j, _ptr(out))
    return out


def philox_many(seed: int, domain: int, j: int, first: int, count: int) -> np.ndarray:
    out = np.zeros((count, 4), dtype=np.uint32)
    _load().orc_philox_many(seed, domain, j, first, count, _ptr(out))
    return out


def philox_raw(key0: int, key1: int, ctr) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox_raw(key0, key1, _ptr(c), _ptr(out))
    return out


def scale128(words, S: int) -> int:
    w = np.asarray(words, dtype=np.uint32)
    return int(_load().orc_scale128(_ptr(w), S))


@dataclass
class Samples:
    st: np.ndarray        # (count, 2) int32
    path_len: np.ndarray  # (count,) int32
    paths: np.ndarray     # (count, max_len) int32, -1 padded
    stats: np.ndarray     # (count, len(STAT_NAMES)) int64
    status: np.ndarray    # (count,) int32

    def stat(self, name: str) -> np.ndarray:
        return self.stats[:, STAT_NAMES.index(name)]

    def sigma_st(self) -> np.ndarray:
        return (self.stat("sigma_hi").astype(np.uint64) << np.uint64(32)) | self.stat("sigma_lo").astype(np.uint64)


def sample_paths(g, seed: int, domain: int, first_idx: int, count: int, max_len: int = 64) -> Samples:
    keep, ga = _gargs(g)
    st = np.zeros((count, 2), dtype=np.int32)
    pl = np.zeros(count, dtype=np.int32)
    paths = np.full((count, max_len), -1, dtype=np.int32)
    stats = np.zeros((count, len(STAT_NAMES)), dtype=np.int64)
    status = np.zeros(count, dtype=np.int32)
    _load().orc_sample_paths(*ga, seed, domain, first_idx, count, _ptr(st), _ptr(pl), _ptr(paths),
                             max_len, _ptr(stats), _ptr(status))
    del keep
    return Samples(st, pl, paths, stats, status)


def sample_fixed_pair(g, s: int, t: int, seed: int, count: int, first_idx: int = 0,
                      domain: int = 0, max_len: int = 64):
    keep, ga = _gargs(g)
    pl = np.zeros(count, dtype=np.int32)
    paths = np.full((count, max_len), -1, dtype=np.int32)
    stats = np.zeros((count, len(STAT_NAMES)), dtype=np.int64)
    rc = _load().orc_sample_fixed_pair(*ga, s, t, seed, domain, first_idx, count, _ptr(pl), _ptr(paths),
                                       max_len, _ptr(stats))
    del keep
    return rc, pl, paths, stats


def accumulate(g, seed: int, domain: int, first_idx: int, count: int):
    keep, ga = _gargs(g)
    counts = np.zeros(g.n, dtype=np.uint32)
    totals = np.zeros(len(STAT_NAMES), dtype=np.int64)
    rc = _load().orc_accumulate(*ga, seed, domain, first_idx, count, _ptr(counts), _ptr(totals))
    del keep
    return rc, counts, totals


def omega(lam: float, delta: float, vd: int) -> float:
    return float(_load().orc_omega(lam, delta, vd))


def vd_bound(g) -> int:
    """Upper bound on the vertex diameter (the most nodes on a shortest path)
    from the condensation into strongly connected components; omega's VD
    (Alg. 1, Sec. 2)."""
    keep, ga = _gargs(g)
    r = int(_load().orc_vd_bound(*ga))
    del keep
    return r


def compute_delta(count0: np.ndarray, alpha: int, omega_: float, lam: float, delta: float, eps: float):
    c0 = np.ascontiguousarray(count0, dtype=np.uint32)
    n = c0.shape[0]
    dl = np.zeros(n, dtype=np.float64)
    du = np.zeros(n, dtype=np.float64)
    Cval = _load().orc_compute_delta(n, _ptr(c0), alpha, omega_, lam, delta, eps, _ptr(dl), _ptr(du))
    return float(Cval), dl, du


def f_and_g(count: int, tau: int, omega_: float, lnL: float, lnU: float):
    f = C.c_double()
    g = C.c_double()
    _load().orc_f_and_g(count, tau, omega_, lnL, lnU, C.byref(f), C.byref(g))
    return f.value, g.value


def check_stop(counts: np.ndarray, tau: int, omega_: float, lnL: np.ndarray, lnU: np.ndarray, lam: float):
    c = np.ascontiguousarray(counts, dtype=np.uint32)
    L = np.ascontiguousarray(lnL, dtype=np.float64)
    U = np.ascontiguousarray(lnU, dtype=np.float64)
    mf = C.c_double()
    mg = C.c_double()
    stop = _load().orc_check_stop(c.shape[0], _ptr(c), tau, omega_, _ptr(L), _ptr(U), lam,
                                  C.byref(mf), C.byref(mg))
    return bool(stop), mf.value, mg.value


def compute_delta_lv(count0: np.ndarray, alpha: int, omega_: float, lam_l: np.ndarray, lam_u: np.ndarray,
                     delta: float, eps: float):
    """Alg. 2 with per-node error targets lambda_L(v), lambda_U(v)."""
    c0 = np.ascontiguousarray(count0, dtype=np.uint32)
    ll = np.ascontiguousarray(lam_l, dtype=np.float64)
    lu = np.ascontiguousarray(lam_u, dtype=np.float64)
    n = c0.shape[0]
    dl = np.zeros(n, dtype=np.float64)
    du = np.zeros(n, dtype=np.float64)
    Cval = _load().orc_compute_delta_lv(n, _ptr(c0), alpha, omega_, _ptr(ll), _ptr(lu), delta, eps, _ptr(dl),
                                        _ptr(du))
    return float(Cval), dl, du


def topk_lambdas(count_pre: np.ndarray, alpha_pre: int, k: int, lam: float):
    """Sec. 5 error targets (lambda_L, lambda_U) for the top-k stop test."""
    c = np.ascontiguousarray(count_pre, dtype=np.uint32)
    n = c.shape[0]
    ll = np.zeros(n, dtype=np.float64)
    lu = np.zeros(n, dtype=np.float64)
    _load().orc_topk_lambdas(n, _ptr(c), alpha_pre, k, lam, _ptr(ll), _ptr(lu))
    return ll, lu


def check_stop_topk(counts: np.ndarray, tau: int, omega_: float, lnL: np.ndarray, lnU: np.ndarray, lam: float,
                    k: int):
    """Alg. 3: (stop, top-k ids, max f, max g)."""
    c = np.ascontiguousarray(counts, dtype=np.uint32)
    L = np.ascontiguousarray(lnL, dtype=np.float64)
    U = np.ascontiguousarray(lnU, dtype=np.float64)
    n = c.shape[0]
    top = np.full(min(k, n), -1, dtype=np.int32)
    mf = C.c_double()
    mg = C.c_double()
    stop = _load().orc_check_stop_topk(n, _ptr(c), tau, omega_, _ptr(L), _ptr(U), lam, k, _ptr(top),
                                       C.byref(mf), C.byref(mg))
    return bool(stop), top, mf.value, mg.value


@dataclass
class RunResult:
    res: orc_result
    counts: np.ndarray
    count0: np.ndarray
    ln_inv_dl: np.ndarray
    ln_inv_du: np.ndarray
    topk: np.ndarray = None
    count_pre: np.ndarray = None
    lam_l: np.ndarray = None
    lam_u: np.ndarray = None

    def __getattr__(self, k):
        return getattr(self.res, k)


def run(g, lam: float, delta: float, seed: int, K: int, vd: int = 0, eps: float = 0.001) -> RunResult:
    keep, ga = _gargs(g)
    n = int(g.n)
    counts = np.zeros(n, dtype=np.uint32)
    count0 = np.zeros(n, dtype=np.uint32)
    dl = np.zeros(n, dtype=np.float64)
    du = np.zeros(n, dtype=np.float64)
    res = orc_result()
    _load().orc_run(*ga, lam, delta, seed, K, vd, eps, _ptr(counts), _ptr(count0), _ptr(dl), _ptr(du),
                    C.byref(res))
    del keep
    return RunResult(res, counts, count0, dl, du)


def run_topk(g, lam: float, delta: float, k: int, seed: int, K: int, vd: int = 0, eps: float = 0.001) -> RunResult:
    """Alg. 1 in top-k mode (Sec. 5 targets, Alg. 2, Alg. 3 every K samples)."""
    keep, ga = _gargs(g)
    n = int(g.n)
    counts = np.zeros(n, dtype=np.uint32)
    count0 = np.zeros(n, dtype=np.uint32)
    count_pre = np.zeros(n, dtype=np.uint32)
    dl = np.zeros(n, dtype=np.float64)
    du = np.zeros(n, dtype=np.float64)
    ll = np.zeros(n, dtype=np.float64)
    lu = np.zeros(n, dtype=np.float64)
    top = np.full(min(k, n), -1, dtype=np.int32)
    res = orc_result()
    _load().orc_run_topk(*ga, lam, delta, seed, K, vd, eps, k, _ptr(counts), _ptr(count0), _ptr(dl), _ptr(du),
                         _ptr(top), _ptr(count_pre), _ptr(ll), _ptr(lu), C.byref(res))
    del keep
    return RunResult(res, counts, count0, dl, du, top, count_pre, ll, lu)


def brandes(g) -> np.ndarray:
    keep, ga = _gargs(g)
    bc = np.zeros(g.n, dtype=np.float64)
    rc = _load().orc_brandes(*ga, _ptr(bc))
    del keep
    if rc != OK:
        raise ValueError(f"orc_brandes failed: {rc}")
    return bc


def enumerate_paths(g, s: int, t: int, max_paths: int = 100000, max_len: int = 64) -> np.ndarray:
    keep, ga = _gargs(g)
    paths = np.full((max_paths, max_len), -1, dtype=np.int32)
    k = int(_load().orc_enumerate_paths(*ga, s, t, max_paths, max_len, _ptr(paths)))
    del keep
    if k < 0:
        raise ValueError("too many paths or too long")
    return paths[:k]
