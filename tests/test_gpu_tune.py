"""The shared-memory tier's two table sizes (chosen per graph by the
autotuner, or forced) give identical runs (GPU only)."""

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


@pytest.mark.parametrize("name,make,lam,k", [
    ("er2000", lambda gg: gg.erdos_renyi(2000, 8.0, 1), 0.01, 0),
    ("cl20k", lambda gg: gg.chung_lu(20000, 2.5, 12.0, 800.0, 4), 0.01, 0),
    ("path300", lambda gg: gg.path_graph(300), 0.03, 0),
    ("drand", lambda gg: random_graph(gg, 400, 0.01, 9, directed=True), 0.02, 5),
], ids=["er2000", "cl20k", "path300", "drand_topk"])
def test_tier_variants_give_identical_runs(kd, gg, name, make, lam, k):
    g = make(gg)
    G = kd.kadabra_load_csr(g)
    try:
        auto = kd.kadabra_run(G, lam, 0.1, k, 3, check_interval=1000)
        again = kd.kadabra_run(G, lam, 0.1, k, 3, check_interval=1000)  # cached choice
        forced = [kd.kadabra_run(G, lam, 0.1, k, 3, check_interval=1000, ctas_per_sm=c) for c in (4, 5)]
        # every setup by itself: both layouts, with and without tier W
        forced += [kd.kadabra_run(G, lam, 0.1, k, 3, check_interval=1000, ctas_per_sm=c, warp_tier=wt)
                   for c in (4, 5) for wt in (-1, 1)]
        with pytest.raises(kd.KadabraError):
            kd.kadabra_run(G, lam, 0.1, k, 3, ctas_per_sm=7)
    finally:
        G.free()
    assert auto.ctas_per_sm in (4, 5) and again.ctas_per_sm == auto.ctas_per_sm
    assert [r.ctas_per_sm for r in forced] == [4, 5, 4, 4, 5, 5]
    assert [r.warp_tier for r in forced[2:]] == [0, 1, 0, 1]
    for r in [again] + forced:
        assert r.tau == auto.tau and r.checks == auto.checks and r.C == auto.C
        assert np.array_equal(r.counts, auto.counts) and (r.max_f, r.max_g) == (auto.max_f, auto.max_g)
        assert np.array_equal(r.totals, auto.totals)
        if k:
            assert np.array_equal(r.topk, auto.topk)
