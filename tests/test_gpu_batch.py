"""Batched multi-graph runs against plain per-graph runs and the oracle (GPU only).

A batch samples every unfinished graph's next batch of samples in one launch
per round; each graph's result must be bit-identical to kadabra_run on that
graph alone with the same lambda, delta, seed and check interval, and to the
oracle.
"""

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


def _same(a, b, tag):
    for f in ("tau", "check_interval", "omega_cap", "alpha", "checks", "vd", "omega", "C", "max_f", "max_g",
              "stopped_early"):
        assert getattr(a, f) == getattr(b, f), (tag, f, getattr(a, f), getattr(b, f))
    assert np.array_equal(a.counts, b.counts), tag
    assert np.array_equal(a.totals, b.totals), tag
    assert np.array_equal(a.btilde, b.btilde), tag


def _uneven(gg):
    return [
        gg.barabasi_albert(3000, 3, 1),
        gg.erdos_renyi(5000, 6.0, 2),
        gg.rmat(11, 8, 0.57, 0.19, 0.19, 3),          # directed, many disconnected pairs
        gg.star_graph(400),
        gg.chung_lu(20000, 2.5, 12.0, 800.0, 4),
        gg.barabasi_albert(20000, 5, 5),
        gg.path_graph(700),                            # deep searches: n-sized tables
        random_graph(gg, 300, 0.02, 6, directed=True),
    ]


def test_batch_matches_plain_runs(kd, gg):
    graphs = _uneven(gg)
    G = len(graphs)
    lam = [0.03, 0.02, 0.05, 0.04, 0.02, 0.025, 0.05, 0.05]
    delta = [0.1] * G
    seed = [11 + i for i in range(G)]
    B = kd.Batch(graphs)
    try:
        got = B.run(lam, delta, seed)
        for i, g in enumerate(graphs):
            ref = kd.kadabra_run(B.views[i], lam[i], delta[i], 0, seed[i], check_interval=got[i].check_interval)
            _same(got[i], ref, g.name)
        # a second run on the same batch reuses the workspace and gives the same results
        again = B.run(lam, delta, seed)
        for i in range(G):
            _same(again[i], got[i], "repeat")
    finally:
        B.free()


def test_batch_matches_oracle(kd, orc, gg):
    graphs = [gg.erdos_renyi(2000, 8.0, 1), gg.barabasi_albert(1500, 4, 7), gg.star_graph(60)]
    lam, delta, seed = [0.02, 0.03, 0.05], [0.1, 0.1, 0.1], [5, 6, 7]
    B = kd.Batch(graphs)
    try:
        got = B.run(lam, delta, seed)
    finally:
        B.free()
    for i, g in enumerate(graphs):
        r = orc.run(g, lam[i], delta[i], seed=seed[i], K=got[i].check_interval)
        assert r.status == 0
        assert (got[i].tau, got[i].C, got[i].max_f, got[i].max_g) == (r.tau, r.C, r.max_f, r.max_g), g.name
        assert np.array_equal(got[i].counts, r.counts), g.name


def test_auto_check_interval(kd, er2000):
    G = kd.kadabra_load_csr(er2000)
    try:
        r = kd.kadabra_run(G, 0.01, 0.1, 0, 3, check_interval=0)
    finally:
        G.free()
    assert r.check_interval == max(1024, int(np.ceil(r.omega / 32)))


def test_batch_repeated_mixed_depths_match_plain(kd, gg):
    """Many batched launches mixing deep searches (a path, a sparse directed
    graph: some samples reach the shared-memory depth limit and move to the
    global tables) with shallow ones.  Every run must equal the plain runs
    of its graphs; a block whose warps ever left a sample at different
    barriers would corrupt later samples of that block."""
    graphs = [gg.barabasi_albert(3000, 3, 1), gg.path_graph(300), random_graph(gg, 400, 0.01, 9, directed=True),
              gg.erdos_renyi(2000, 8.0, 1)]
    G = len(graphs)
    B = kd.Batch(graphs)
    plain = {}
    try:
        for it in range(25):
            seeds = [it * 10 + i for i in range(G)]
            got = B.run([0.02] * G, [0.1] * G, seeds)
            for i in (1, 2):  # the deep graphs, against plain runs
                ref = plain.get((i, seeds[i]))
                if ref is None:
                    ref = kd.kadabra_run(B.views[i], 0.02, 0.1, 0, seeds[i], check_interval=got[i].check_interval)
                    plain[(i, seeds[i])] = ref
                assert got[i].tau == ref.tau and np.array_equal(got[i].counts, ref.counts), (it, i)
    finally:
        B.free()


@pytest.mark.slow
def test_batched_workload_largest_graphs_match_oracle(kd, orc):
    """The 64-graph uneven Barabasi-Albert workload of the benchmark, run as
    one batch; each of its 8 largest graphs (n up to 2 * 10^6) must equal the
    oracle's run replayed over index ranges (same K)."""
    import bench
    from replay import replay_run
    graphs = bench.make_batched_graphs()
    b = bench.BATCHED
    G = len(graphs)
    seeds = [7 + i for i in range(G)]
    B = kd.Batch(graphs)
    try:
        got = B.run([b["lam"]] * G, [b["delta"]] * G, seeds)
        for i in range(G):
            assert got[i].vd == B.views[i].vd
    finally:
        B.free()
    for i in sorted(range(G), key=lambda i: -graphs[i].n)[:8]:
        assert got[i].vd == orc.vd_bound(graphs[i])
        replay_run(orc, graphs[i], got[i], b["lam"], b["delta"], got[i].check_interval, seeds[i])
