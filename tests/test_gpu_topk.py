"""Top-k mode (Sec. 5 targets, Alg. 2 with per-node targets, Alg. 3) on the
GPU against the oracle: tau, the number of stop tests, C, max f, max g, the
per-node counts and the returned ranking must be identical."""

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


def _compare(kd, orc, g, lam, delta, k, seed, K, tag):
    G = kd.kadabra_load_csr(g)
    try:
        got = kd.kadabra_run(G, lam, delta, k, seed, check_interval=K)
    finally:
        G.free()
    ref = orc.run_topk(g, lam, delta, k, seed, K)
    assert ref.status == 0, tag
    assert got.alpha == ref.alpha and got.omega == ref.omega and got.vd == ref.vd, tag
    assert got.C == ref.C, (tag, got.C, ref.C)
    assert (got.tau, got.checks, got.stopped_early) == (ref.tau, ref.checks, bool(ref.stopped_early)), tag
    assert np.array_equal(got.counts, ref.counts), tag
    assert np.array_equal(got.topk, ref.topk), (tag, got.topk, ref.topk)
    assert (got.max_f, got.max_g) == (ref.max_f, ref.max_g), tag
    # the ranking is the order of the final counts (ties by id)
    order = sorted(range(g.n), key=lambda v: (-int(got.counts[v]), v))
    assert list(got.topk) == order[:min(k, g.n)], tag
    return got


CASES = [
    ("ba300_k5", lambda gg: gg.barabasi_albert(300, 3, 1), 0.02, 5, 1000),
    ("ba300_k1", lambda gg: gg.barabasi_albert(300, 3, 2), 0.02, 1, 1000),
    ("er2000_k10", lambda gg: gg.erdos_renyi(2000, 8.0, 1), 0.01, 10, 1000),
    ("er2000_k50", lambda gg: gg.erdos_renyi(2000, 8.0, 1), 0.01, 50, 2000),
    ("cl20k_k10", lambda gg: gg.chung_lu(20000, 2.5, 12.0, 800.0, 4), 0.01, 10, 4096),
    ("rmat12_k10", lambda gg: gg.rmat(12, 8, 0.57, 0.19, 0.19, 3), 0.01, 10, 2048),
    ("star_k3", lambda gg: gg.star_graph(200), 0.02, 3, 500),
    ("path_k4", lambda gg: gg.path_graph(300), 0.03, 4, 500),
    ("dir_random_k7", lambda gg: random_graph(gg, 400, 0.01, 9, directed=True), 0.02, 7, 700),
    ("k_above_n", lambda gg: gg.complete_graph(6), 0.05, 10, 200),
    ("k256", lambda gg: gg.barabasi_albert(5000, 4, 3), 0.02, 256, 3000),
]


@pytest.mark.parametrize("name,make,lam,k,K", CASES, ids=[c[0] for c in CASES])
def test_topk_run_matches_oracle(kd, orc, gg, name, make, lam, k, K):
    g = make(gg)
    _compare(kd, orc, g, lam, 0.1, k, seed=17, K=K, tag=name)


def test_topk_two_seeds_and_rerun(kd, orc, gg):
    """Same graph object, two seeds, then the first seed again (buffers reused)."""
    g = gg.barabasi_albert(3000, 5, 8)
    G = kd.kadabra_load_csr(g)
    try:
        a = kd.kadabra_run(G, 0.01, 0.1, 10, 5, check_interval=2000)
        b = kd.kadabra_run(G, 0.01, 0.1, 10, 6, check_interval=2000)
        c = kd.kadabra_run(G, 0.01, 0.1, 10, 5, check_interval=2000)
        d = kd.kadabra_run(G, 0.01, 0.1, 0, 5, check_interval=2000)  # all-nodes mode in between
        e = kd.kadabra_run(G, 0.01, 0.1, 10, 5, check_interval=2000)
    finally:
        G.free()
    assert np.array_equal(a.counts, c.counts) and np.array_equal(a.topk, c.topk) and a.tau == c.tau
    assert np.array_equal(a.counts, e.counts) and a.tau == e.tau
    ref = orc.run_topk(g, 0.01, 0.1, 10, 6, 2000)
    assert b.tau == ref.tau and np.array_equal(b.counts, ref.counts) and np.array_equal(b.topk, ref.topk)
    ref0 = orc.run(g, 0.01, 0.1, 5, 2000)
    assert d.tau == ref0.tau and np.array_equal(d.counts, ref0.counts)


def test_topk_rejects_bad_k(kd, gg):
    g = gg.barabasi_albert(100, 2, 1)
    G = kd.kadabra_load_csr(g)
    try:
        with pytest.raises(kd.KadabraError):
            kd.kadabra_run(G, 0.05, 0.1, 257, 1)
        with pytest.raises(kd.KadabraError):
            kd.kadabra_run(G, 0.05, 0.1, -1, 1)
    finally:
        G.free()
