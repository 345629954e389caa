"""The one-warp-per-sample tier (tier W) against the oracle and against the
block tiers (GPU only).  With KADABRA_FLAG_WARP_TIER every sample starts in
tier W's small table and moves on to the block tiers only if its search
outgrows it; per-sample pairs, paths, work counters and statuses must be
bit-exact with the oracle either way, and whole runs, batches and served
jobs must not depend on the tier."""

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


def _paths_warp(kd, orc, g, seed, domain, first, count, max_len=256, tag="", expect_rc=0):
    G = kd.kadabra_load_csr(g)
    try:
        G.set_flags(kd.FLAG_WARP_TIER)
        got, rc = kd.kadabra_sample_paths(G, seed, domain, first, count, max_len=max_len, raise_on_error=False)
    finally:
        G.free()
    ref = orc.sample_paths(g, seed, domain, first, count, max_len=max_len)
    assert rc == expect_rc, (tag, rc)
    _same_samples(got, ref, tag)
    return got


def _bipartite(gg, a, b):
    """Complete bipartite K_{a,b}: two nodes on the same side are joined by
    one shortest path through each node of the other side, so their search
    meets on up to max(a, b) candidate edges at once."""
    e = [(i, a + j) for i in range(a) for j in range(b)]
    return gg.from_edges(a + b, e, name=f"K{a},{b}")


GRAPHS = [
    ("path50", lambda gg: gg.path_graph(50)),
    ("star30", lambda gg: gg.star_graph(30)),
    ("cycle41", lambda gg: gg.cycle_graph(41)),
    ("cycle600", lambda gg: gg.cycle_graph(600)),    # distances beyond the 256-node lists
    ("grid12", lambda gg: gg.grid_graph(12, 12)),
    ("Q6", lambda gg: gg.hypercube_graph(6)),
    ("K20", lambda gg: gg.complete_graph(20)),
    ("K2", lambda gg: gg.complete_graph(2)),
    ("K60_70", lambda gg: _bipartite(gg, 60, 70)),
    ("K150_160", lambda gg: _bipartite(gg, 150, 160)),  # > 128 candidate edges: handed on
    ("dcycle50", lambda gg: gg.directed_cycle(50)),
    ("drand300", lambda gg: random_graph(gg, 300, 0.012, 7, directed=True)),
    ("rand_disconnected", lambda gg: random_graph(gg, 400, 0.004, 8)),
    ("ba3000", lambda gg: gg.barabasi_albert(3000, 3, 9)),
    ("rmat12", lambda gg: gg.rmat(12, 8, 0.57, 0.19, 0.19, 10)),
    ("er_nolcc", lambda gg: gg.erdos_renyi(3000, 1.5, 11, lcc=False)),
    ("cl20k", lambda gg: gg.chung_lu(20000, 2.5, 12.0, 800.0, 4)),
]


@pytest.mark.parametrize("name,make", GRAPHS, ids=[s[0] for s in GRAPHS])
def test_warp_tier_sample_paths_match_oracle(kd, orc, gg, name, make):
    g = make(gg)
    _paths_warp(kd, orc, g, 41, 0, 0, 3000, max_len=700, tag=name)
    _paths_warp(kd, orc, g, 42, 1, 2**32 - 300, 700, max_len=700, tag=name + "/warm")


def test_warp_tier_er2000_and_power_law(kd, orc, er2000, chung_lu_1m):
    _paths_warp(kd, orc, er2000, 1, 0, 0, 5000, max_len=64, tag="er2000")
    _paths_warp(kd, orc, chung_lu_1m, 3, 0, 40_000, 2000, max_len=64, tag="chung-lu")


def test_warp_tier_sigma_overflow(kd, orc, gg):
    """A chain of 80 diamonds (sigma up to 2^80): samples whose sigma outgrows
    the packed field move on; those beyond 64 bits are reported per sample."""
    k = 80
    edges = []
    for i in range(k):
        a, b, c, d = 3 * i, 3 * i + 1, 3 * i + 2, 3 * i + 3
        edges += [(a, b), (a, c), (b, d), (c, d)]
    g = gg.from_edges(3 * k + 1, edges)
    got = _paths_warp(kd, orc, g, 5, 0, 0, 3000, max_len=256, tag="diamonds", expect_rc=kd.ERR_SIGMA_OVERFLOW)
    assert (got.status == 4).sum() > 10


def test_warp_tier_sample_batch(kd, orc, er2000, gg):
    """Hit counts and work totals of sample batches, flag on and off."""
    import torch
    for g in (er2000, gg.barabasi_albert(3000, 3, 9), gg.path_graph(400)):
        res = []
        for flag in (0, kd.FLAG_WARP_TIER):
            G = kd.kadabra_load_csr(g)
            try:
                G.set_flags(flag)
                c = torch.zeros(g.n, dtype=torch.int32, device="cuda")
                t = torch.zeros(kd.NSTAT, dtype=torch.int64, device="cuda")
                first = 0
                for sz in (1, 31, 4097, 0, 2000):
                    kd.kadabra_sample_batch(G, 8, 0, first, sz, c, t)
                    first += sz
                kd.kadabra_sync_status(G)
            finally:
                G.free()
            res.append((c.cpu().numpy().astype(np.uint32), t.cpu().numpy()))
        assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1]), g.name
        rc, ref, tot = orc.accumulate(g, 8, 0, 0, first)
        assert rc == 0 and np.array_equal(res[1][0], ref)
        for q in range(8):
            assert res[1][1][q] == tot[q], (g.name, q)


RUNS = [
    ("er2000", lambda gg: gg.erdos_renyi(2000, 8.0, 1), 0.01, 0),
    ("cl20k", lambda gg: gg.chung_lu(20000, 2.5, 12.0, 800.0, 4), 0.01, 0),
    ("path300", lambda gg: gg.path_graph(300), 0.03, 0),
    ("K150_160", lambda gg: _bipartite(gg, 150, 160), 0.02, 0),
    ("drand_topk", lambda gg: random_graph(gg, 400, 0.01, 9, directed=True), 0.02, 5),
    ("ba3000_topk", lambda gg: gg.barabasi_albert(3000, 3, 1), 0.02, 10),
]


@pytest.mark.parametrize("name,make,lam,k", RUNS, ids=[r[0] for r in RUNS])
def test_warp_tier_runs_identical(kd, orc, gg, name, make, lam, k):
    g = make(gg)
    G = kd.kadabra_load_csr(g)
    try:
        off = kd.kadabra_run(G, lam, 0.1, k, 3, check_interval=1000, warp_tier=-1)
        on = kd.kadabra_run(G, lam, 0.1, k, 3, check_interval=1000, warp_tier=1)
        on4 = kd.kadabra_run(G, lam, 0.1, k, 3, check_interval=1000, warp_tier=1, ctas_per_sm=5)
        auto = kd.kadabra_run(G, lam, 0.1, k, 3, check_interval=1000)
        with pytest.raises(kd.KadabraError):
            kd.kadabra_run(G, lam, 0.1, k, 3, warp_tier=2)
    finally:
        G.free()
    assert (off.warp_tier, on.warp_tier, on4.warp_tier, on4.ctas_per_sm) == (0, 1, 1, 5)
    assert auto.warp_tier in (0, 1) and auto.ctas_per_sm in (4, 5)
    for r in (on, on4, auto):
        assert (r.tau, r.checks, r.C, r.max_f, r.max_g) == (off.tau, off.checks, off.C, off.max_f, off.max_g), name
        assert np.array_equal(r.counts, off.counts) and np.array_equal(r.totals, off.totals), name
        if k:
            assert np.array_equal(r.topk, off.topk), name
    ref = orc.run_topk(g, lam, 0.1, k, 3, 1000) if k else orc.run(g, lam, 0.1, 3, 1000)
    assert on.tau == ref.tau and np.array_equal(on.counts, ref.counts)


def test_warp_tier_batch_and_serving(kd, gg):
    """A batch whose views carry the flag, and served jobs on such graphs,
    equal plain runs without it."""
    graphs = [gg.barabasi_albert(3000, 3, 1), gg.path_graph(300), random_graph(gg, 400, 0.01, 9, directed=True),
              gg.erdos_renyi(2000, 8.0, 1)]
    G = len(graphs)
    lam, delta, seed = [0.02] * G, [0.1] * G, [21 + i for i in range(G)]
    B = kd.Batch(graphs)
    try:
        plain = B.run(lam, delta, seed)
        for v in B.views:
            v.set_flags(kd.FLAG_WARP_TIER)
        warp = B.run(lam, delta, seed)
        for a, b in zip(plain, warp):
            assert a.tau == b.tau and np.array_equal(a.counts, b.counts) and np.array_equal(a.totals, b.totals)
    finally:
        B.free()
    handles = [kd.kadabra_load_csr(g) for g in graphs]
    try:
        for h in handles:
            h.set_flags(kd.FLAG_WARP_TIER)
        ids = [kd.kadabra_submit(handles[i], lam[i], delta[i], 0, seed[i], check_interval=plain[i].check_interval)
               for i in range(G)]
        served = [kd.kadabra_poll(j, graphs[i].n, 0, wait=True) for i, j in enumerate(ids)]
        for a, b in zip(plain, served):
            assert a.tau == b.tau and np.array_equal(a.counts, b.counts) and np.array_equal(a.totals, b.totals)
    finally:
        kd.kadabra_serve_shutdown()
        for h in handles:
            h.free()
