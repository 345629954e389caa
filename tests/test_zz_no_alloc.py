"""The sampler batch without device allocation (GPU only).

kadabra_sample_batch_noalloc is for callers that cannot allocate device
memory: code whose device memory belongs to another allocator, or code that
must not call cudaMalloc/cudaFree after start-up.  It keeps its scratch in one
file-scope device array shared by all calls.  This test checks, through the C
ABI, that it gives the same hit counts and work counters as
kadabra_sample_batch on two calls in a row (the second call sees the scratch
the first one left behind), and that it rejects batches beyond its limit.

This file is collected last so that a failure here cannot hide others.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1604_08553_gb300 import kadabra
    kadabra.load_library()
    return kadabra


def _reference(kd, g, seed, domain, first, count):
    import torch
    G = kd.kadabra_load_csr(g)
    try:
        c = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        t = torch.zeros(kd.NSTAT, dtype=torch.int64, device="cuda")
        kd.kadabra_sample_batch(G, seed, domain, first, count, c, t)
        kd.kadabra_sync_status(G)
    finally:
        G.free()
    return c.cpu().numpy(), t.cpu().numpy()


def _noalloc(kd, g, seed, domain, first, count):
    import torch
    rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr)).cuda()
    ci = torch.from_numpy(np.ascontiguousarray(g.col)).cuda()
    rrp = torch.from_numpy(np.ascontiguousarray(g.rrow_ptr)).cuda() if g.directed else None
    rci = torch.from_numpy(np.ascontiguousarray(g.rcol)).cuda() if g.directed else None
    c = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    t = torch.zeros(kd.NSTAT, dtype=torch.int64, device="cuda")
    kd.kadabra_sample_batch_noalloc(g.n, rp, ci, seed, domain, first, count, c, t, directed=g.directed,
                                    rrow_ptr=rrp, rcol=rci)
    return c.cpu().numpy(), t.cpu().numpy()


def test_noalloc_matches_sample_batch_twice(kd, gg):
    # the Chung-Lu graph and the path send samples on to the global-memory
    # tier of the call (larger or deeper searches than the shared tables hold;
    # on a path equal costs expand the s side, so its search runs up to 899
    # levels deep)
    graphs = [gg.erdos_renyi(2000, 8.0, 1), gg.rmat(12, 8, 0.57, 0.19, 0.19, 10),
              gg.chung_lu(100_000, 2.5, 16.0, 2_000.0, 3), gg.path_graph(900)]
    for g in graphs:
        calls = [(1, 0, 0, 20_000), (2, 1, 777, 20_000)]  # two calls in a row on the shared scratch
        for seed, domain, first, count in calls:
            c_new, t_new = _noalloc(kd, g, seed, domain, first, count)
            c_ref, t_ref = _reference(kd, g, seed, domain, first, count)
            assert np.array_equal(c_new, c_ref), (g.name, seed)
            assert np.array_equal(t_new, t_ref), (g.name, seed)
            assert c_new.sum() > 0


def test_noalloc_rejects_oversized_batches(kd, gg):
    import torch
    g = gg.erdos_renyi(2000, 8.0, 1)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col).cuda()
    c = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(kd.KadabraError) as e:
        kd.kadabra_sample_batch_noalloc(g.n, rp, ci, 1, 0, 0, 65537, c)
    assert e.value.status == kd.ERR_CAPACITY
    assert int(c.sum().item()) == 0


def test_noalloc_capacity_error_then_recovers(kd, gg):
    """A batch whose samples outgrow every table of the call (a path of 6000
    nodes: s-side searches deeper than the 1022 levels of the largest one)
    is refused with KADABRA_ERR_CAPACITY; the next call, on an ordinary graph,
    starts from a cleared scratch header and equals kadabra_sample_batch
    again."""
    path = gg.path_graph(6000)
    with pytest.raises(kd.KadabraError) as e:
        _noalloc(kd, path, 3, 0, 0, 4096)
    assert e.value.status == kd.ERR_CAPACITY
    g = gg.erdos_renyi(2000, 8.0, 1)
    c_new, t_new = _noalloc(kd, g, 4, 0, 0, 8192)
    c_ref, t_ref = _reference(kd, g, 4, 0, 0, 8192)
    assert np.array_equal(c_new, c_ref)
    assert np.array_equal(t_new, t_ref)


def test_noalloc_without_totals(kd, gg):
    """d_totals may be NULL: the hit counts are the same."""
    import torch
    g = gg.rmat(12, 8, 0.57, 0.19, 0.19, 10)
    rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr)).cuda()
    ci = torch.from_numpy(np.ascontiguousarray(g.col)).cuda()
    rrp = torch.from_numpy(np.ascontiguousarray(g.rrow_ptr)).cuda()
    rci = torch.from_numpy(np.ascontiguousarray(g.rcol)).cuda()
    c = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    kd.kadabra_sample_batch_noalloc(g.n, rp, ci, 5, 0, 100, 20_000, c, None, directed=True, rrow_ptr=rrp, rcol=rci)
    c_ref, _ = _reference(kd, g, 5, 0, 100, 20_000)
    assert np.array_equal(c.cpu().numpy(), c_ref)
