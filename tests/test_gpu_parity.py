"""CUDA path against the oracle, through the C ABI (GPU only).

Integer results (pairs, paths, hit counts, tau, work counters, statuses) must
be bit-exact; the FP64 stop test (max f, max g) and computeDelta must be
bit-exact too, because both sides evaluate the same expression trees with
IEEE-exact operations and no contraction.
"""

import math

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


def assert_samples_equal(a, b, tag=""):
    assert np.array_equal(a.status, b.status), tag
    ok = a.status == 0
    assert np.array_equal(a.st[ok], b.st[ok]), tag
    assert np.array_equal(a.path_len[ok], b.path_len[ok]), tag
    assert np.array_equal(a.paths[ok], b.paths[ok]), tag
    bad = np.nonzero((a.stats[ok] != b.stats[ok]).any(axis=1))[0]
    assert bad.size == 0, (tag, bad[:5], a.stats[ok][bad[:3]], b.stats[ok][bad[:3]])


def compare_paths(kd, orc, g, seed, domain, first, count, max_len=64, tag=""):
    G = kd.kadabra_load_csr(g)
    try:
        got = kd.kadabra_sample_paths(G, seed, domain, first, count, max_len=max_len)
    finally:
        G.free()
    ref = orc.sample_paths(g, seed, domain, first, count, max_len=max_len)
    assert np.all(ref.status == 0)
    assert_samples_equal(got, ref, tag)
    return got


# ------------------------------------------------------------------ RNG
def test_philox_device_matches_oracle(kd, orc):
    for seed, dom, j, first in ((1, 0, 0, 0), (0xDEADBEEFCAFEF00D, 1, 3, 2**32 - 1000), (2**64 - 1, 0, 7, 12345)):
        n = 1_000_000 if j == 0 else 100_000
        assert np.array_equal(kd.kadabra_philox(seed, dom, j, first, n), orc.philox_many(seed, dom, j, first, n))


# ------------------------------------------------------------------ sampler
def test_sample_paths_er2000(kd, orc, er2000):
    compare_paths(kd, orc, er2000, 1, 0, 0, 5000, tag="main")
    compare_paths(kd, orc, er2000, 1, 1, 0, 2000, tag="warm-up")
    compare_paths(kd, orc, er2000, 0xABCDEF0123456789, 0, 2**32 - 700, 1500, tag="idx crosses 2^32")


SMALL = [
    ("path50", lambda gg: gg.path_graph(50)),
    ("star30", lambda gg: gg.star_graph(30)),
    ("cycle41", lambda gg: gg.cycle_graph(41)),
    ("cycle200", lambda gg: gg.cycle_graph(200)),
    ("grid12", lambda gg: gg.grid_graph(12, 12)),
    ("Q6", lambda gg: gg.hypercube_graph(6)),
    ("K20", lambda gg: gg.complete_graph(20)),
    ("K2", lambda gg: gg.complete_graph(2)),
    ("dcycle50", lambda gg: gg.directed_cycle(50)),
    ("drand300", lambda gg: random_graph(gg, 300, 0.012, 7, directed=True)),
    ("rand_disconnected", lambda gg: random_graph(gg, 400, 0.004, 8)),
    ("ba3000", lambda gg: gg.barabasi_albert(3000, 3, 9)),
    ("rmat12", lambda gg: gg.rmat(12, 8, 0.57, 0.19, 0.19, 10)),
    ("er_nolcc", lambda gg: gg.erdos_renyi(3000, 1.5, 11, lcc=False)),
]


@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
def test_sample_paths_small_graphs(kd, orc, gg, name, make):
    g = make(gg)
    compare_paths(kd, orc, g, 17, 0, 0, 3000, max_len=256, tag=name)
    compare_paths(kd, orc, g, 18, 1, 100, 700, max_len=256, tag=name + "/warm")


@pytest.mark.slow
def test_sample_paths_chung_lu_full_size(kd, orc, chung_lu_1m):
    """Full-size power-law graph (n = 10^6): per-sample parity on sampled index
    ranges of both RNG domains, including samples deferred to the
    global-memory tables (visited sets beyond shared memory)."""
    got = compare_paths(kd, orc, chung_lu_1m, 1, 0, 123_456, 2500, tag="main")
    compare_paths(kd, orc, chung_lu_1m, 1, 1, 0, 800, tag="warm-up")


def test_sigma_overflow_is_reported_per_sample(kd, orc, gg):
    """A chain of 80 diamonds: pairs 64+ diamonds apart have 2^64+ shortest paths."""
    k = 80
    edges = []
    for i in range(k):
        a, b, c, d = 3 * i, 3 * i + 1, 3 * i + 2, 3 * i + 3
        edges += [(a, b), (a, c), (b, d), (c, d)]
    g = gg.from_edges(3 * k + 1, edges)
    G = kd.kadabra_load_csr(g)
    try:
        got, rc = kd.kadabra_sample_paths(G, 5, 0, 0, 3000, max_len=256, raise_on_error=False)
    finally:
        G.free()
    ref = orc.sample_paths(g, 5, 0, 0, 3000, max_len=256)
    assert rc == kd.ERR_SIGMA_OVERFLOW
    assert (ref.status == 4).sum() > 10
    assert_samples_equal(got, ref, "diamonds")


def test_deep_searches_use_global_tables(kd, orc, gg):
    """Distances far beyond the shared-memory level limit (254 per side):
    such samples are deferred to the global-memory tables."""
    compare_paths(kd, orc, gg.path_graph(1500), 1, 0, 0, 300, max_len=1600, tag="path1500")
    compare_paths(kd, orc, gg.cycle_graph(2001), 2, 0, 0, 300, max_len=1100, tag="cycle2001")


def compare_paths_global(kd, orc, g, seed, domain, first, count, max_len=64, tag="", flag=None):
    G = kd.kadabra_load_csr(g)
    try:
        G.set_flags(kd.FLAG_GLOBAL_TABLES if flag is None else flag)
        got = kd.kadabra_sample_paths(G, seed, domain, first, count, max_len=max_len)
    finally:
        G.free()
    ref = orc.sample_paths(g, seed, domain, first, count, max_len=max_len)
    assert_samples_equal(got, ref, tag)


@pytest.mark.parametrize("name,make", [s for s in SMALL if s[0] in ("Q6", "drand300", "ba3000", "rmat12", "star30")],
                         ids=["Q6", "drand300", "ba3000", "rmat12", "star30"])
def test_global_tables_match_oracle(kd, orc, gg, name, make):
    g = make(gg)
    compare_paths_global(kd, orc, g, 23, 0, 0, 1500, max_len=256, tag=name)
    compare_paths_global(kd, orc, g, 26, 0, 0, 1500, max_len=256, tag=name + "/medium", flag=kd.FLAG_MEDIUM_TABLES)
    compare_paths_global(kd, orc, g, 29, 0, 0, 1500, max_len=256, tag=name + "/large-shared",
                         flag=kd.FLAG_LARGE_SHARED_TABLES)


def test_global_tables_er_and_power_law(kd, orc, er2000, chung_lu_1m):
    compare_paths_global(kd, orc, er2000, 24, 0, 0, 3000, tag="er2000")
    compare_paths_global(kd, orc, chung_lu_1m, 25, 0, 777, 400, tag="chung-lu")
    compare_paths_global(kd, orc, er2000, 27, 1, 0, 3000, tag="er2000/medium", flag=kd.FLAG_MEDIUM_TABLES)
    compare_paths_global(kd, orc, chung_lu_1m, 28, 0, 5000, 1500, tag="chung-lu/medium",
                         flag=kd.FLAG_MEDIUM_TABLES)
    compare_paths_global(kd, orc, chung_lu_1m, 30, 0, 9000, 1500, tag="chung-lu/large-shared",
                         flag=kd.FLAG_LARGE_SHARED_TABLES)


def test_searched_rows_match_oracle(kd, orc, gg):
    """A dense Barabasi-Albert graph (n = 2000, 30 arcs per new node) with the
    scan for graphs beyond the L2 forced on: frontier rows that are long next
    to a small other frontier are searched for that frontier's nodes instead
    of scanned, and levels that searched rows without a touch are scanned
    again to insert.  Every table tier; with 64-node frontier segments a
    segment takes two searched rows at most, so levels with more scan the
    rest.  The default scan (no searches) gives the same samples."""
    g = gg.barabasi_albert(2000, 30, 3)
    compare_paths(kd, orc, g, 41, 0, 0, 3000, tag="ba2000x30")
    for flag, tag in ((0, "searched rows"), (kd.FLAG_LARGE_SHARED_TABLES, "large-shared"),
                      (kd.FLAG_MEDIUM_TABLES, "medium"), (kd.FLAG_GLOBAL_TABLES, "global"),
                      (kd.FLAG_FRONTIER_SEGMENTS, "segments")):
        compare_paths_global(kd, orc, g, 42, 0, 0, 1500, tag="ba2000x30/" + tag, flag=flag | kd.FLAG_ASYNC_SCAN)


@pytest.mark.parametrize("name,make", [s for s in SMALL if s[0] in ("Q6", "drand300", "ba3000", "rmat12", "star30", "cycle200")],
                         ids=["Q6", "drand300", "ba3000", "rmat12", "star30", "cycle200"])
def test_compact_tier_s_chain_matches_oracle(kd, orc, gg, name, make):
    """Tier S in the compact layout (lists of 2048 nodes, 38 levels per side):
    per-sample results as the oracle's (the cycle's long searches and the
    power-law graphs' large ones move on to tier B)."""
    g = make(gg)
    compare_paths_global(kd, orc, g, 43, 0, 0, 2000, max_len=256, tag=name + "/compact", flag=kd.FLAG_COMPACT_TABLES)


def test_compact_tier_s_chain_power_law(kd, orc, gg, chung_lu_1m):
    compare_paths_global(kd, orc, chung_lu_1m, 44, 0, 20_000, 3000, tag="chung-lu/compact", flag=kd.FLAG_COMPACT_TABLES)
    compare_paths_global(kd, orc, gg.path_graph(300), 45, 0, 0, 500, max_len=320, tag="path300/compact",
                         flag=kd.FLAG_COMPACT_TABLES)


def test_run_with_forced_tiers_matches_plain(kd, er2000):
    """Whole runs give identical results whichever table tier holds the samples."""
    out = []
    for flag in (0, kd.FLAG_LARGE_SHARED_TABLES, kd.FLAG_MEDIUM_TABLES, kd.FLAG_GLOBAL_TABLES):
        G = kd.kadabra_load_csr(er2000)
        try:
            G.set_flags(flag)
            r = kd.kadabra_run(G, 0.02, 0.1, 0, 9, check_interval=500)
        finally:
            G.free()
        out.append(r)
    for r in out[1:]:
        assert r.tau == out[0].tau and np.array_equal(r.counts, out[0].counts)
        assert np.array_equal(r.totals, out[0].totals)


def test_sample_batch_ragged_and_order_independent(kd, orc, er2000):
    import torch
    G = kd.kadabra_load_csr(er2000)
    try:
        c1 = torch.zeros(er2000.n, dtype=torch.int32, device="cuda")
        t1 = torch.zeros(kd.NSTAT, dtype=torch.int64, device="cuda")
        first = 0
        for sz in (1, 7, 0, 1000, 4097, 33):
            kd.kadabra_sample_batch(G, 3, 0, first, sz, c1, t1)
            first += sz
        kd.kadabra_sync_status(G)
        c2 = torch.zeros_like(c1)
        t2 = torch.zeros_like(t1)
        kd.kadabra_sample_batch(G, 3, 0, 0, first, c2, t2)
        kd.kadabra_sync_status(G)
    finally:
        G.free()
    assert torch.equal(c1, c2) and torch.equal(t1, t2)
    rc, ref, tot = orc.accumulate(er2000, 3, 0, 0, first)
    assert np.array_equal(c1.cpu().numpy().astype(np.uint32), ref)
    t = t1.cpu().numpy()
    for k in (0, 1, 2, 3, 4, 5, 6, 7):
        assert t[k] == tot[k], k


def test_load_csr_device_tensors(kd, orc, er2000):
    import torch
    rp = torch.from_numpy(er2000.row_ptr).cuda()
    ci = torch.from_numpy(er2000.col).cuda()
    G = kd.kadabra_load_csr_device(er2000.n, rp, ci)
    try:
        got = kd.kadabra_sample_paths(G, 2, 0, 0, 500)
        assert G.vd == orc.vd_bound(er2000)
    finally:
        G.free()
    assert_samples_equal(got, orc.sample_paths(er2000, 2, 0, 0, 500), "device csr")


def test_invalid_csr_rejected(kd, gg):
    CSR = gg.CSRGraph
    i32 = lambda a: np.array(a, dtype=np.int32)
    cases = {
        # path 0-1-2 with row 1 stored out of order
        "unsorted": CSR(3, i32([0, 1, 3, 4]), i32([1, 2, 0, 1])),
        "self-loop": CSR(3, i32([0, 2, 3, 4]), i32([0, 1, 0, 1])),
        "id out of range": CSR(3, i32([0, 1, 3, 4]), i32([1, 0, 7, 1])),
        "asymmetric": CSR(3, i32([0, 1, 2, 2]), i32([1, 2])),
        # every arc u -> v with u < v has its mirror, but 2 -> 0 has none
        "asymmetric descending": CSR(3, i32([0, 1, 2, 3]), i32([1, 0, 0])),
        "duplicate": CSR(3, i32([0, 2, 3, 4]), i32([1, 1, 0, 1])),
    }
    # a large symmetric graph with one arc v -> u (v > u) removed
    er = gg.erdos_renyi(2000, 8.0, 1)
    v = er.n - 1
    a0, a1 = int(er.row_ptr[v]), int(er.row_ptr[v + 1])
    assert int(er.col[a0]) < v
    col = np.delete(er.col, a0)
    rp = er.row_ptr.copy()
    rp[v + 1:] -= 1
    cases["asymmetric large"] = CSR(er.n, rp, col)
    for name, b in cases.items():
        with pytest.raises(kd.KadabraError) as e:
            kd.kadabra_load_csr(b)
        assert e.value.status == kd.ERR_CSR, name
    d = gg.from_edges(4, [(0, 1), (1, 2), (2, 3)], directed=True)
    d.rcol = d.rcol.copy()
    d.rcol[0] = 3  # reverse CSR no longer mirrors the forward CSR
    with pytest.raises(kd.KadabraError) as e:
        kd.kadabra_load_csr(d)
    assert e.value.status == kd.ERR_CSR


def test_vd_with_hub_rows_matches_oracle(kd, orc, gg):
    """The VD bound's root and BFS on graphs whose rows exceed the BFS's
    per-warp chunk (hubs of degree > 1024, split into work items), directed
    graphs with and without reciprocal arcs (undirected degree = out + in -
    reciprocal), and a graph with empty rows."""
    rng = np.random.default_rng(5)
    n = 6000
    arcs = {(0, v) for v in range(1, n)} | {(v, 0) for v in range(1, n, 3)}  # hub 0, partly reciprocal
    arcs |= {(int(a), int(b)) for a, b in rng.integers(1, n, size=(8000, 2)) if a != b}
    cases = [
        ("star5000", gg.star_graph(5000)),
        ("ba20000", gg.barabasi_albert(20000, 5, 3)),
        ("rmat14", gg.rmat(14, 16, 0.57, 0.19, 0.19, 2)),
        ("directed hub", gg.from_edges(n, sorted(arcs), directed=True)),
        ("isolated nodes", gg.from_edges(50, [(1, 2), (2, 3), (10, 11)])),
    ]
    for name, g in cases:
        G = kd.kadabra_load_csr(g)
        try:
            assert G.vd == orc.vd_bound(g), name
        finally:
            G.free()


def _scc_chain(gg, k, size, seed):
    """k directed cycles of `size` nodes in a chain (an arc from each cycle to
    the next) plus random arcs forward along the chain: components with two or
    more nodes that become ready at different levels of the condensation."""
    rng = np.random.default_rng(seed)
    e = set()
    for c in range(k):
        b = c * size
        e |= {(b + i, b + (i + 1) % size) for i in range(size)}
        if c + 1 < k:
            e.add((b + int(rng.integers(size)), b + size + int(rng.integers(size))))
    for _ in range(3 * k):
        a, b = sorted(rng.integers(0, k * size, size=2))
        if a // size < b // size:
            e.add((int(a), int(b)))
    return gg.from_edges(k * size, sorted(e), directed=True, name=f"scc_chain{k}x{size}")


def test_vd_bound_condensation_matches_oracle(kd, orc, gg):
    """Graphs whose root component is not the whole graph, so the bound comes
    from the condensation: directed graphs with many components (trimmed
    singletons, components found by colour propagation, components ready at
    different levels), the chain with a hub whose undirected-eccentricity
    rule under-counts, and undirected graphs with several components.  The
    GPU bound equals the oracle's and bounds every shortest path."""
    import networkx as nx
    from test_oracle_pins import hub_sink_graph, _true_vd
    cases = [random_graph(gg, n, p, seed, directed=True)
             for (n, p, seed) in ((30, 0.05, 2), (60, 0.02, 5), (200, 0.012, 7), (400, 0.004, 8), (300, 0.02, 9))]
    cases += [hub_sink_graph(gg, 40), gg.directed_cycle(11), _scc_chain(gg, 12, 5, 3), _scc_chain(gg, 40, 3, 4),
              gg.from_edges(10, [(i, i + 1) for i in range(9)], directed=True, name="dpath10"),
              gg.from_edges(25, [(i, i + 1) for i in range(4)] + [(i, i + 1) for i in range(5, 24)], name="p5+p20"),
              random_graph(gg, 300, 0.006, 11), gg.rmat(12, 16, 0.57, 0.19, 0.19, 1),
              gg.rmat(16, 8, 0.57, 0.19, 0.19, 3)]
    for g in cases:
        G = kd.kadabra_load_csr(g)
        try:
            got = G.vd
        finally:
            G.free()
        assert got == orc.vd_bound(g), g.name
        if g.n <= 400:
            assert got >= _true_vd(g), g.name


def test_graph_memory_reused_across_loads(kd, orc, gg):
    """Graph buffers come from a pool that keeps freed memory: loading and
    freeing the same graph again does not grow the device's used memory,
    results stay the oracle's, and releasing the cached memory returns it."""
    import torch
    g = gg.barabasi_albert(50000, 6, 11)
    ref = orc.sample_paths(g, 8, 0, 0, 1000)
    used = []
    for _ in range(4):
        G = kd.kadabra_load_csr(g)
        try:
            got = kd.kadabra_sample_paths(G, 8, 0, 0, 1000)
        finally:
            G.free()
        assert_samples_equal(got, ref, "pooled load")
        torch.cuda.synchronize()
        free_b, total_b = torch.cuda.mem_get_info()
        used.append(total_b - free_b)
    assert max(used[1:]) <= used[0] + (8 << 20), used
    kd.kadabra_release_cached()
    free_b, total_b = torch.cuda.mem_get_info()
    assert total_b - free_b <= used[-1], (total_b - free_b, used)


def test_workspace_reuse_across_graph_objects(kd, orc, gg, er2000):
    """A freed graph object's sampler workspace serves the next one that fits
    in it: results stay identical to the oracle, an error left in the
    workspace does not reach the next owner, and releasing the kept
    workspaces changes nothing."""
    import torch
    big = gg.barabasi_albert(20000, 5, 3)
    G = kd.kadabra_load_csr(big)
    kd.kadabra_run(G, 0.02, 0.1, 0, 5, check_interval=1000)
    G.free()
    G = kd.kadabra_load_csr(er2000)  # smaller: takes the kept workspace
    try:
        got = kd.kadabra_sample_paths(G, 3, 0, 0, 2000)
        r1 = kd.kadabra_run(G, 0.02, 0.1, 0, 9, check_interval=500)
    finally:
        G.free()
    assert_samples_equal(got, orc.sample_paths(er2000, 3, 0, 0, 2000), "reused workspace")
    ref = orc.run(er2000, 0.02, 0.1, 9, 500)
    assert r1.tau == ref.tau and np.array_equal(r1.counts, ref.counts)
    # a sigma overflow left unread in the workspace (no status sync before the free)
    k = 80
    edges = []
    for i in range(k):
        a, b, c, d = 3 * i, 3 * i + 1, 3 * i + 2, 3 * i + 3
        edges += [(a, b), (a, c), (b, d), (c, d)]
    dia = gg.from_edges(3 * k + 1, edges)
    G = kd.kadabra_load_csr(dia)
    c = torch.zeros(dia.n, dtype=torch.int32, device="cuda")
    t = torch.zeros(kd.NSTAT, dtype=torch.int64, device="cuda")
    kd.kadabra_sample_batch(G, 5, 0, 0, 3000, c, t)
    G.free()
    G = kd.kadabra_load_csr(er2000)
    try:
        r2 = kd.kadabra_run(G, 0.02, 0.1, 0, 9, check_interval=500)
    finally:
        G.free()
    assert r2.tau == r1.tau and np.array_equal(r2.counts, r1.counts)
    kd.kadabra_release_cached()
    G = kd.kadabra_load_csr(er2000)
    try:
        r3 = kd.kadabra_run(G, 0.02, 0.1, 0, 9, check_interval=500)
    finally:
        G.free()
    assert r3.tau == r1.tau and np.array_equal(r3.counts, r1.counts)


# ------------------------------------------------------------------ stop test
def test_check_kernel_matches_oracle(kd, orc):
    rng = np.random.default_rng(12)
    for trial in range(8):
        n = int(rng.integers(1, 300_000))
        tau = int(rng.integers(1, 500_000))
        omega = float(tau) * float(rng.uniform(1.0, 30.0))
        counts = rng.integers(0, max(1, tau // int(rng.integers(1, 1000))), size=n).astype(np.uint32)
        counts[rng.random(n) < 0.3] = 0
        c0 = rng.poisson(0.4, n).astype(np.uint32)
        _, L, U = orc.compute_delta(c0, 500, omega, 0.01, 0.1, 0.001)
        lam = float(rng.choice([0.002, 0.01, 0.05, 0.5]))
        a = kd.kadabra_check(counts, tau, omega, L, U, lam)
        b = orc.check_stop(counts, tau, omega, L, U, lam)
        assert a == b, (trial, a, b)


# ------------------------------------------------------------------ full runs
def _run_pair(kd, orc, g, lam, delta, seed, K, vd=0):
    G = kd.kadabra_load_csr(g)
    try:
        got = kd.kadabra_run(G, lam, delta, 0, seed, vd=vd, check_interval=K)
    finally:
        G.free()
    ref = orc.run(g, lam, delta, seed=seed, K=K, vd=vd)
    assert ref.status == 0
    for f in ("tau", "omega_cap", "alpha", "checks", "vd", "omega", "C", "max_f", "max_g"):
        assert getattr(got, f) == getattr(ref, f), (f, getattr(got, f), getattr(ref, f))
    assert got.stopped_early == bool(ref.stopped_early)
    assert np.array_equal(got.counts, ref.counts)
    assert got.totals[0] == ref.edges_warm + ref.edges_main
    assert np.array_equal(got.btilde, ref.counts / float(ref.tau))
    return got, ref


def test_run_matches_oracle_er2000(kd, orc, er2000):
    for seed in (1, 2):
        got, ref = _run_pair(kd, orc, er2000, 0.01, 0.1, seed, 1000)
        assert got.checks >= 1


@pytest.mark.parametrize("name,make,lam,K", [
    ("star40", lambda gg: gg.star_graph(40), 0.05, 100),
    ("grid8", lambda gg: gg.grid_graph(8, 8), 0.03, 250),
    ("drand200", lambda gg: random_graph(gg, 200, 0.03, 13, directed=True), 0.05, 128),
    ("K12", lambda gg: gg.complete_graph(12), 0.05, 100),
    ("ba2000", lambda gg: gg.barabasi_albert(2000, 4, 14), 0.02, 1000),
])
def test_run_matches_oracle_small(kd, orc, gg, name, make, lam, K):
    got, ref = _run_pair(kd, orc, make(gg), lam, 0.1, 21, K)
    if name == "K12":
        assert got.counts.sum() == 0


def test_run_rejects_bad_args(kd, er2000):
    G = kd.kadabra_load_csr(er2000)
    try:
        for k in (-1, 257):  # top-k mode takes 1 <= k <= 256
            with pytest.raises(kd.KadabraError) as e:
                kd.kadabra_run(G, 0.01, 0.1, k, 1)
            assert e.value.status == kd.ERR_ARG
        for lam, delta in ((0.0, 0.1), (0.01, 1.0), (-1.0, 0.1)):
            with pytest.raises(kd.KadabraError):
                kd.kadabra_run(G, lam, delta, 0, 1)
    finally:
        G.free()


@pytest.mark.slow
def test_run_chung_lu_full_size_matches_oracle(kd, orc, chung_lu_1m):
    """The benchmark configuration (n = 10^6, lambda = 0.005, delta = 0.1,
    K = 2^16): warm-up counts, C, every stop decision, the final tau and the
    final hit counts, with the oracle run over index ranges in a process pool."""
    from oracle.parallel import accumulate_ranges
    g = chung_lu_1m
    lam, delta, K, seed = 0.005, 0.1, 1 << 16, 1
    G = kd.kadabra_load_csr(g)
    try:
        got = kd.kadabra_run(G, lam, delta, 0, seed, check_interval=K)
        vd_gpu = G.vd
    finally:
        G.free()
    assert vd_gpu == orc.vd_bound(g) == got.vd
    assert got.omega == orc.omega(lam, delta, got.vd)
    assert got.alpha == max(1, math.floor(got.omega / 100))
    bounds = list(range(0, got.tau, K)) + [got.tau]
    ranges = [(0, got.alpha)] + [(a, b - a) for a, b in zip(bounds[:-1], bounds[1:])]
    res = accumulate_ranges(g, seed, 1, ranges[:1]) + accumulate_ranges(g, seed, 0, ranges[1:])
    count0 = res[0][0]
    C, L, U = orc.compute_delta(count0, got.alpha, got.omega, lam, delta, 0.001)
    assert C == got.C
    counts = np.zeros(g.n, dtype=np.uint32)
    for i, (cnt, _) in enumerate(res[1:]):
        counts += cnt
        tau_i = bounds[i + 1]
        stop, mf, mg = orc.check_stop(counts, tau_i, got.omega, L, U, lam)
        last = i == len(res) - 2
        if not last:
            assert not stop, tau_i
        elif got.stopped_early:
            assert stop
    assert np.array_equal(got.counts, counts)
    assert (got.max_f, got.max_g) == (mf, mg)
    edges = sum(t[0] for _, t in res)
    assert got.totals[0] == edges
