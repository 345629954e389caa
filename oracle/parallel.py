"""Process-pool driver for the oracle (TEST INFRASTRUCTURE ONLY).

Runs the single-threaded oracle sampler over disjoint sample-index ranges in
separate processes and sums the integer hit counts, which gives the same
result as one sequential pass (counts are order-independent sums).  Workers
are started with the 'spawn' method, so a parent that already holds a CUDA
context is safe.
"""

from __future__ import annotations

import multiprocessing as mp
import os
import shutil
import tempfile

import numpy as np

_G = None


class _Graph:
    def __init__(self, d):
        self.n = int(np.load(os.path.join(d, "n.npy")))
        self.directed = bool(np.load(os.path.join(d, "directed.npy")))
        self.row_ptr = np.load(os.path.join(d, "row_ptr.npy"), mmap_mode="r")
        self.col = np.load(os.path.join(d, "col.npy"), mmap_mode="r")
        self.rrow_ptr = np.load(os.path.join(d, "rrow_ptr.npy"), mmap_mode="r") if self.directed else None
        self.rcol = np.load(os.path.join(d, "rcol.npy"), mmap_mode="r") if self.directed else None


def _init(d):
    global _G
    g = _Graph(d)
    # materialise once per worker (the oracle wants contiguous int32 arrays)
    g.row_ptr = np.ascontiguousarray(g.row_ptr)
    g.col = np.ascontiguousarray(g.col)
    if g.directed:
        g.rrow_ptr = np.ascontiguousarray(g.rrow_ptr)
        g.rcol = np.ascontiguousarray(g.rcol)
    _G = g


def _work(args):
    import oracle
    key, seed, domain, first, count = args
    rc, counts, totals = oracle.accumulate(_G, seed, domain, first, count)
    return key, rc, counts, totals


def accumulate_ranges(g, seed: int, domain: int, ranges, processes: int | None = None, chunk: int = 2000,
                      timing: dict | None = None):
    """Returns [(counts, totals)] for each (first, count) in ranges.  If
    timing is a dict, timing["work_s"] gets the wall time of the sampling
    alone (workers started and warmed up before the clock starts) and
    timing["processes"] the worker count."""
    processes = processes or max(1, min(os.cpu_count() or 1, 64))
    d = tempfile.mkdtemp(prefix="orc_graph_")
    try:
        np.save(os.path.join(d, "n.npy"), np.int64(g.n))
        np.save(os.path.join(d, "directed.npy"), np.bool_(g.directed))
        np.save(os.path.join(d, "row_ptr.npy"), np.asarray(g.row_ptr, dtype=np.int32))
        np.save(os.path.join(d, "col.npy"), np.asarray(g.col, dtype=np.int32))
        if g.directed:
            np.save(os.path.join(d, "rrow_ptr.npy"), np.asarray(g.rrow_ptr, dtype=np.int32))
            np.save(os.path.join(d, "rcol.npy"), np.asarray(g.rcol, dtype=np.int32))
        tasks = []
        for key, (first, count) in enumerate(ranges):
            for a in range(first, first + count, chunk):
                tasks.append((key, seed, domain, a, min(chunk, first + count - a)))
        out = [[np.zeros(g.n, dtype=np.uint64), np.zeros(11, dtype=np.int64)] for _ in ranges]
        ctx = mp.get_context("spawn")
        with ctx.Pool(processes, initializer=_init, initargs=(d,)) as pool:
            if timing is not None:
                import time
                # one tiny task per worker: start-up and imports before the clock
                pool.map(_work, [(0, seed, domain, 0, 1)] * processes, chunksize=1)
                t0 = time.perf_counter()
            for key, rc, counts, totals in pool.imap_unordered(_work, tasks):
                if rc != 0:
                    raise RuntimeError(f"oracle status {rc}")
                out[key][0] += counts
                out[key][1] += totals
            if timing is not None:
                timing["work_s"] = time.perf_counter() - t0
                timing["processes"] = processes
        return [(c.astype(np.uint32), t) for c, t in out]
    finally:
        shutil.rmtree(d, ignore_errors=True)
