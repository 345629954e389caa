"""Seeded synthetic input graphs (input side only; no part of the method).

Both the CUDA path and the oracle consume these graphs; this module holds
none of the method's arithmetic.  Large families (Erdos-Renyi, Chung-Lu,
Barabasi-Albert, R-MAT) come from ``csrc/graphgen.cpp``; the small closed-form
families (paths, stars, cycles, grids, hypercubes, complete graphs) used by
tests are built here with numpy.

Every graph is an int32 CSR with sorted, duplicate-free rows and no
self-loops; directed graphs also carry the reverse CSR (in-arcs), which the
backward search of the bidirectional BFS reads (paper Sec. 4).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "graphgen.cpp")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


@dataclass
class CSRGraph:
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    directed: bool = False
    rrow_ptr: Optional[np.ndarray] = None
    rcol: Optional[np.ndarray] = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def in_row_ptr(self) -> np.ndarray:
        return self.rrow_ptr if self.directed else self.row_ptr

    def in_col(self) -> np.ndarray:
        return self.rcol if self.directed else self.col

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def build(force: bool = False) -> str:
    """Compiles csrc/graphgen.cpp into the package directory."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        p = C.c_void_p
        lib.gg_erdos_renyi.argtypes = [C.c_int64, C.c_double, C.c_uint64, C.c_int]
        lib.gg_erdos_renyi.restype = p
        lib.gg_chung_lu.argtypes = [C.c_int64, C.c_double, C.c_double, C.c_double, C.c_uint64, C.c_int]
        lib.gg_chung_lu.restype = p
        lib.gg_barabasi_albert.argtypes = [C.c_int64, C.c_int32, C.c_uint64]
        lib.gg_barabasi_albert.restype = p
        lib.gg_rmat.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_uint64]
        lib.gg_rmat.restype = p
        for f in ("gg_num_nodes", "gg_num_arcs"):
            getattr(lib, f).argtypes = [p]
            getattr(lib, f).restype = C.c_int64
        lib.gg_is_directed.argtypes = [p]
        lib.gg_copy.argtypes = [p, p, p, p, p]
        lib.gg_free.argtypes = [p]
        _lib = lib
    return _lib


def _take(h, name: str, meta: dict) -> CSRGraph:
    lib = _load()
    if not h:
        raise ValueError(f"graph generator rejected its arguments: {name} {meta}")
    try:
        n = int(lib.gg_num_nodes(h))
        m = int(lib.gg_num_arcs(h))
        directed = bool(lib.gg_is_directed(h))
        rp = np.empty(n + 1, dtype=np.int32)
        col = np.empty(m, dtype=np.int32)
        rrp = np.empty(n + 1, dtype=np.int32) if directed else None
        rcol = np.empty(m, dtype=np.int32) if directed else None
        f = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)
        lib.gg_copy(h, f(rp), f(col), f(rrp), f(rcol))
    finally:
        lib.gg_free(h)
    return CSRGraph(n, rp, col, directed, rrp, rcol, name, meta)


def erdos_renyi(n: int, avg_deg: float, seed: int, lcc: bool = True) -> CSRGraph:
    meta = dict(n=n, avg_deg=avg_deg, seed=seed, lcc=lcc)
    return _take(_load().gg_erdos_renyi(n, avg_deg, seed, int(lcc)), "erdos_renyi", meta)


def chung_lu(n: int, beta: float, mean_deg: float, max_deg: float, seed: int, lcc: bool = True) -> CSRGraph:
    meta = dict(n=n, beta=beta, mean_deg=mean_deg, max_deg=max_deg, seed=seed, lcc=lcc)
    return _take(_load().gg_chung_lu(n, beta, mean_deg, max_deg, seed, int(lcc)), "chung_lu", meta)


def barabasi_albert(n: int, m: int, seed: int) -> CSRGraph:
    meta = dict(n=n, m=m, seed=seed)
    return _take(_load().gg_barabasi_albert(n, m, seed), "barabasi_albert", meta)


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int) -> CSRGraph:
    meta = dict(scale=scale, edge_factor=edge_factor, a=a, b=b, c=c, seed=seed)
    return _take(_load().gg_rmat(scale, edge_factor, a, b, c, seed), "rmat", meta)


# ---------------------------------------------------------------- small graphs
def from_edges(n: int, edges, directed: bool = False, name: str = "") -> CSRGraph:
    """CSR from an edge list (pairs); undirected edges are symmetrised."""
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    if not directed:
        e = np.concatenate([e, e[:, ::-1]], axis=0)
    key = np.unique(e[:, 0] * n + e[:, 1]) if e.size else np.zeros(0, dtype=np.int64)
    src, dst = key // n, key % n
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    col = dst.astype(np.int32)
    g = CSRGraph(n, rp, col, directed, name=name)
    if directed:
        rkey = np.unique(dst * n + src) if key.size else np.zeros(0, dtype=np.int64)
        rs, rd = rkey // n, rkey % n
        rrp = np.zeros(n + 1, dtype=np.int64)
        np.add.at(rrp, rs + 1, 1)
        g.rrow_ptr = np.cumsum(rrp).astype(np.int32)
        g.rcol = rd.astype(np.int32)
    return g


def path_graph(n: int) -> CSRGraph:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], name=f"path{n}")


def star_graph(n: int) -> CSRGraph:
    """Centre 0 and n-1 leaves."""
    return from_edges(n, [(0, i) for i in range(1, n)], name=f"star{n}")


def cycle_graph(n: int) -> CSRGraph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], name=f"cycle{n}")


def complete_graph(n: int) -> CSRGraph:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], name=f"K{n}")


def grid_graph(rows: int, cols: int) -> CSRGraph:
    """rows x cols lattice; node id = r*cols + c."""
    e = []
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            if c + 1 < cols:
                e.append((v, v + 1))
            if r + 1 < rows:
                e.append((v, v + cols))
    return from_edges(rows * cols, e, name=f"grid{rows}x{cols}")


def hypercube_graph(d: int) -> CSRGraph:
    n = 1 << d
    return from_edges(n, [(v, v ^ (1 << b)) for v in range(n) for b in range(d) if v < v ^ (1 << b)],
                      name=f"Q{d}")


def directed_cycle(n: int) -> CSRGraph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], directed=True, name=f"dcycle{n}")
