"""Serving (continuous batching): jobs submitted together, admitted as memory
and slots allow and sampled in shared launches, give the same results as
kadabra_run alone and as the oracle (GPU only)."""

import time

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
    yield kadabra
    kadabra.kadabra_serve_shutdown()


@pytest.fixture(scope="module")
def loaded(kd, gg):
    graphs = {
        "ba3000": gg.barabasi_albert(3000, 3, 1),
        "er2000": gg.erdos_renyi(2000, 8.0, 1),
        "cl20k": gg.chung_lu(20000, 2.5, 12.0, 800.0, 4),
        "rmat12": gg.rmat(12, 8, 0.57, 0.19, 0.19, 3),
        "path300": gg.path_graph(300),
        "drand": random_graph(gg, 400, 0.01, 9, directed=True),
    }
    handles = {k: kd.kadabra_load_csr(g) for k, g in graphs.items()}
    yield graphs, handles
    for h in handles.values():
        h.free()


# (graph, lambda, k, seed, K)
JOBS = [
    ("ba3000", 0.02, 0, 1, 1000), ("er2000", 0.01, 10, 2, 1000), ("cl20k", 0.01, 0, 3, 0),
    ("rmat12", 0.02, 5, 4, 2048), ("path300", 0.03, 0, 5, 500), ("drand", 0.02, 3, 6, 700),
    ("cl20k", 0.01, 50, 7, 0), ("ba3000", 0.02, 0, 8, 1000), ("ba3000", 0.02, 0, 1, 1000),
    ("er2000", 0.02, 0, 9, 0), ("rmat12", 0.01, 0, 10, 4096), ("er2000", 0.01, 1, 11, 1000),
]


def _same(a, b, tag):
    assert (a.tau, a.checks, a.alpha, a.omega, a.C, a.max_f, a.max_g, a.stopped_early, a.check_interval) == \
        (b.tau, b.checks, b.alpha, b.omega, b.C, b.max_f, b.max_g, b.stopped_early, b.check_interval), tag
    assert np.array_equal(a.counts, b.counts), tag
    assert np.array_equal(a.btilde, b.btilde), tag
    assert np.array_equal(a.totals, b.totals), tag
    if a.topk is not None or b.topk is not None:
        assert np.array_equal(a.topk, b.topk), tag


def _serve_all(kd, graphs, handles, jobs):
    ids = [kd.kadabra_submit(handles[gname], lam, 0.1, k, seed, check_interval=K) for gname, lam, k, seed, K in jobs]
    out = []
    for jid, (gname, lam, k, seed, K) in zip(ids, jobs):
        out.append(kd.kadabra_poll(jid, graphs[gname].n, k, wait=True))
    return out


def test_served_equals_alone(kd, loaded):
    graphs, handles = loaded
    served = _serve_all(kd, graphs, handles, JOBS)
    for (gname, lam, k, seed, K), r in zip(JOBS, served):
        alone = kd.kadabra_run(handles[gname], lam, 0.1, k, seed, check_interval=K)
        _same(r, alone, (gname, lam, k, seed))
        assert r.t_submit <= r.t_start <= r.t_done


def test_served_matches_oracle(kd, orc, loaded):
    graphs, handles = loaded
    pick = [JOBS[1], JOBS[2], JOBS[3], JOBS[5]]
    served = _serve_all(kd, graphs, handles, pick)
    for (gname, lam, k, seed, K), r in zip(pick, served):
        g = graphs[gname]
        Kx = K if K else r.check_interval
        ref = orc.run_topk(g, lam, 0.1, k, seed, Kx) if k else orc.run(g, lam, 0.1, seed, Kx)
        assert (r.tau, r.checks, r.C, r.max_f, r.max_g) == (ref.tau, ref.checks, ref.C, ref.max_f, ref.max_g)
        assert np.array_equal(r.counts, ref.counts)
        if k:
            assert np.array_equal(r.topk, ref.topk)


def test_tight_budget_admits_one_at_a_time(kd, loaded):
    """A budget below any job's state: jobs run one after another (each alone
    when nothing else is active) and results do not change."""
    graphs, handles = loaded
    kd.kadabra_serve_shutdown()
    kd.kadabra_serve_configure(1, 2)
    try:
        served = _serve_all(kd, graphs, handles, JOBS[:6])
        starts = sorted((r.t_start, r.t_done) for r in served)
        for (s0, d0), (s1, d1) in zip(starts, starts[1:]):
            assert s1 >= d0 - 1e-3  # admitted only after the previous one finished
        for (gname, lam, k, seed, K), r in zip(JOBS[:6], served):
            alone = kd.kadabra_run(handles[gname], lam, 0.1, k, seed, check_interval=K)
            _same(r, alone, (gname, "tight"))
    finally:
        kd.kadabra_serve_shutdown()
        kd.kadabra_serve_configure(0, 256)


def test_poll_without_wait_and_unknown_job(kd, loaded):
    graphs, handles = loaded
    jid = kd.kadabra_submit(handles["cl20k"], 0.005, 0.1, 0, 99, check_interval=0)
    r = None
    t0 = time.time()
    while r is None and time.time() - t0 < 60:
        r = kd.kadabra_poll(jid, graphs["cl20k"].n, 0, wait=False)
        if r is None:
            time.sleep(0.001)
    assert r is not None and r.tau > 0
    with pytest.raises(kd.KadabraError):
        kd.kadabra_poll(jid, graphs["cl20k"].n, 0, wait=False)
