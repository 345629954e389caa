"""The R-MAT scale-24 benchmark graph (directed, 2^24 ids, about 2.6 * 10^8
arcs, forward and reverse CSR) at full size: the VD bound against the
oracle's, per-sample parity with the oracle on sampled index ranges of both
RNG domains, and full runs in all-nodes and top-k mode (lambda = 0.0025,
delta = 0.1, K = 2^16) replayed by the oracle over index ranges: C, every
stop decision, tau, the hit counts, max f, max g and the ranking (GPU only,
slow)."""

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def kd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1604_08553_gb300 import kadabra
    kadabra.load_library()
    return kadabra


@pytest.fixture(scope="module")
def rmat24(gg):
    return gg.rmat(24, 16, 0.57, 0.19, 0.19, 1)


@pytest.fixture(scope="module")
def G(kd, rmat24):
    h = kd.kadabra_load_csr(rmat24)
    yield h
    h.free()


@pytest.mark.parametrize("domain,first,count", [(0, 123_456, 300), (1, 0, 150)])
def test_rmat24_samples_match_oracle(kd, orc, rmat24, G, domain, first, count):
    got = kd.kadabra_sample_paths(G, 1, domain, first, count, max_len=64)
    ref = orc.sample_paths(rmat24, 1, domain, first, count, max_len=64)
    assert np.array_equal(got.status, ref.status)
    ok = ref.status == 0
    assert np.array_equal(got.st[ok], ref.st[ok])
    assert np.array_equal(got.path_len[ok], ref.path_len[ok])
    assert np.array_equal(got.paths[ok], ref.paths[ok])
    assert np.array_equal(got.stats[ok], ref.stats[ok])


def test_rmat24_vd_bound_matches_oracle(orc, rmat24, G):
    assert G.vd == orc.vd_bound(rmat24)


def test_rmat24_run_matches_oracle(kd, orc, rmat24, G):
    from replay import replay_run
    K = 1 << 16
    got = kd.kadabra_run(G, 0.0025, 0.1, 0, 1, check_interval=K)
    assert got.vd == G.vd
    replay_run(orc, rmat24, got, 0.0025, 0.1, K, 1)


def test_rmat24_topk_run_matches_oracle(kd, orc, rmat24, G):
    from replay import replay_run
    K = 1 << 16
    got = kd.kadabra_run(G, 0.0025, 0.1, 10, 1, check_interval=K)
    replay_run(orc, rmat24, got, 0.0025, 0.1, K, 1, k=10)


def test_rmat24_topk_run_ranking(kd, rmat24, G):
    K = 1 << 16
    r = kd.kadabra_run(G, 0.0025, 0.1, 10, 1, check_interval=K)
    assert r.tau % K == 0 or r.tau == r.omega_cap
    order = np.lexsort((np.arange(rmat24.n), -r.counts.astype(np.int64)))[:10]
    assert list(r.topk) == list(order)
    assert r.counts[r.topk[-1]] >= np.delete(r.counts, r.topk).max()
