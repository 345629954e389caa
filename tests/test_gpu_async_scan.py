"""Variants of the level scans against the oracle (GPU only): 16-byte loads
along long row stretches (KADABRA_FLAG_ASYNC_SCAN; taken by itself for graphs
whose CSR exceeds the L2; the star, Barabasi-Albert, R-MAT and Chung-Lu
graphs have rows long enough, with heads at every 16-byte misalignment) and frontiers scanned in segments (KADABRA_FLAG_FRONTIER_SEGMENTS:
64-node segments; by itself only for frontiers beyond the frontier array, 1024 nodes or 512 in the compact
tier-S layout).
Per-sample pairs, paths, work counters and statuses bit-exact, whole runs
identical.  The R-MAT scale-24 tests cover the automatic choice on a graph
beyond the L2."""

import numpy as np
import pytest

from conftest import random_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1604_08553_gb300 import kadabra
    kadabra.load_library()
    return kadabra


def _same_samples(a, b, tag):
    assert np.array_equal(a.status, b.status), tag
    ok = a.status == 0
    assert np.array_equal(a.st[ok], b.st[ok]), tag
    assert np.array_equal(a.path_len[ok], b.path_len[ok]), tag
    assert np.array_equal(a.paths[ok], b.paths[ok]), tag
    bad = np.nonzero((a.stats[ok] != b.stats[ok]).any(axis=1))[0]
    assert bad.size == 0, (tag, bad[:5], a.stats[ok][bad[:3]], b.stats[ok][bad[:3]])


GRAPHS = [
    ("path50", lambda gg: gg.path_graph(50)),
    ("star300", lambda gg: gg.star_graph(300)),
    ("cycle600", lambda gg: gg.cycle_graph(600)),
    ("grid12", lambda gg: gg.grid_graph(12, 12)),
    ("Q6", lambda gg: gg.hypercube_graph(6)),
    ("K2", lambda gg: gg.complete_graph(2)),
    ("dcycle50", lambda gg: gg.directed_cycle(50)),
    ("drand300", lambda gg: random_graph(gg, 300, 0.012, 7, directed=True)),
    ("rand_disconnected", lambda gg: random_graph(gg, 400, 0.004, 8)),
    ("ba3000", lambda gg: gg.barabasi_albert(3000, 3, 9)),
    ("rmat12", lambda gg: gg.rmat(12, 8, 0.57, 0.19, 0.19, 10)),
    ("cl20k", lambda gg: gg.chung_lu(20000, 2.5, 12.0, 800.0, 4)),
]


@pytest.mark.parametrize("name,make", GRAPHS, ids=[s[0] for s in GRAPHS])
def test_async_scan_sample_paths_match_oracle(kd, orc, gg, name, make):
    g = make(gg)
    ref = orc.sample_paths(g, 51, 0, 0, 3000, max_len=700)
    for flag, tag in ((kd.FLAG_ASYNC_SCAN, "vector"),
                      (kd.FLAG_ASYNC_SCAN | kd.FLAG_LARGE_SHARED_TABLES, "vector, tier B first")):
        G = kd.kadabra_load_csr(g)
        try:
            G.set_flags(flag)
            got, rc = kd.kadabra_sample_paths(G, 51, 0, 0, 3000, max_len=700, raise_on_error=False)
        finally:
            G.free()
        assert rc == 0, (name, tag, rc)
        _same_samples(got, ref, (name, tag))


def test_async_scan_power_law_ranges(kd, orc, chung_lu_1m):
    ref = orc.sample_paths(chung_lu_1m, 4, 1, 70_000, 1500)
    G = kd.kadabra_load_csr(chung_lu_1m)
    try:
        G.set_flags(kd.FLAG_ASYNC_SCAN)
        got = kd.kadabra_sample_paths(G, 4, 1, 70_000, 1500)
    finally:
        G.free()
    _same_samples(got, ref, "chung-lu ring")


@pytest.mark.parametrize("name,make,lam,k", [
    ("er2000", lambda gg: gg.erdos_renyi(2000, 8.0, 1), 0.01, 0),
    ("cl20k_topk", lambda gg: gg.chung_lu(20000, 2.5, 12.0, 800.0, 4), 0.01, 10),
    ("drand", lambda gg: random_graph(gg, 400, 0.01, 9, directed=True), 0.02, 0),
], ids=["er2000", "cl20k_topk", "drand"])
def test_async_scan_runs_identical(kd, gg, name, make, lam, k):
    g = make(gg)
    out = []
    for flag in (0, kd.FLAG_ASYNC_SCAN):
        G = kd.kadabra_load_csr(g)
        try:
            G.set_flags(flag)
            out.append(kd.kadabra_run(G, lam, 0.1, k, 7, check_interval=1000))
        finally:
            G.free()
    a, b = out
    assert (a.tau, a.checks, a.C, a.max_f, a.max_g) == (b.tau, b.checks, b.C, b.max_f, b.max_g), name
    assert np.array_equal(a.counts, b.counts) and np.array_equal(a.totals, b.totals), name
    if k:
        assert np.array_equal(a.topk, b.topk), name


@pytest.mark.parametrize("name,make", GRAPHS, ids=[s[0] for s in GRAPHS])
def test_frontier_segments_match_oracle(kd, orc, gg, name, make):
    """Every frontier of more than 64 nodes scanned in segments, in tier S and
    (all samples started there) in tier B, with either scan."""
    g = make(gg)
    ref = orc.sample_paths(g, 61, 0, 0, 2000, max_len=700)
    for flag, tag in ((kd.FLAG_FRONTIER_SEGMENTS, "segments"),
                      (kd.FLAG_FRONTIER_SEGMENTS | kd.FLAG_ASYNC_SCAN, "segments, vector"),
                      (kd.FLAG_FRONTIER_SEGMENTS | kd.FLAG_LARGE_SHARED_TABLES, "segments, tier B")):
        G = kd.kadabra_load_csr(g)
        try:
            G.set_flags(flag)
            got, rc = kd.kadabra_sample_paths(G, 61, 0, 0, 2000, max_len=700, raise_on_error=False)
        finally:
            G.free()
        assert rc == 0, (name, tag, rc)
        _same_samples(got, ref, (name, tag))


def test_frontier_segments_power_law(kd, orc, chung_lu_1m):
    ref = orc.sample_paths(chung_lu_1m, 5, 0, 90_000, 1500)
    G = kd.kadabra_load_csr(chung_lu_1m)
    try:
        G.set_flags(kd.FLAG_FRONTIER_SEGMENTS | kd.FLAG_LARGE_SHARED_TABLES)
        got = kd.kadabra_sample_paths(G, 5, 0, 90_000, 1500)
    finally:
        G.free()
    _same_samples(got, ref, "chung-lu segments, tier B")


def test_vector_scan_in_deferred_tiers(kd, orc, gg, chung_lu_1m):
    """The scan for graphs beyond the L2 in the tiers after tier S: deep
    searches (a path and a cycle, beyond tier S's levels: tiers B, M and L)
    and the power-law graph's large samples (tier B); per-sample results as
    the oracle's."""
    for name, g, count, ml in (("path1500", gg.path_graph(1500), 300, 1600),
                               ("cycle2001", gg.cycle_graph(2001), 300, 1100)):
        ref = orc.sample_paths(g, 3, 0, 0, count, max_len=ml)
        G = kd.kadabra_load_csr(g)
        try:
            G.set_flags(kd.FLAG_ASYNC_SCAN)
            got = kd.kadabra_sample_paths(G, 3, 0, 0, count, max_len=ml)
        finally:
            G.free()
        _same_samples(got, ref, name)
    ref = orc.sample_paths(chung_lu_1m, 9, 0, 40_000, 3000)
    G = kd.kadabra_load_csr(chung_lu_1m)
    try:
        G.set_flags(kd.FLAG_ASYNC_SCAN)
        got = kd.kadabra_sample_paths(G, 9, 0, 40_000, 3000)
    finally:
        G.free()
    _same_samples(got, ref, "chung-lu, deferred samples")
