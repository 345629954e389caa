"""Replays a run of the CUDA path with the oracle (test infrastructure).

The oracle's sampler runs over the run's sample-index ranges in a process
pool (oracle.parallel), and its own computeDelta, Sec. 5 targets and stop
tests are applied in the run's schedule: the warm-up (and in top-k mode the
preliminary estimate) of alpha samples, then batches of K main-loop samples
with a stop test after each, until the test holds or ceil(omega) samples.
Every value that the oracle's sequential run would produce is checked
against the GPU run: omega, alpha, C, each stop decision, tau, the hit
counts, max f, max g, the ranking (top-k) and the scanned-edge total.
"""

import math

import numpy as np


def replay_run(orc, g, got, lam, delta, K, seed, k=0, eps=0.001):
    from oracle.parallel import accumulate_ranges
    assert got.omega == orc.omega(lam, delta, got.vd)
    assert got.alpha == max(1, math.floor(got.omega / 100))
    assert got.omega_cap == math.ceil(got.omega)
    edges = 0
    warm = accumulate_ranges(g, seed, 1, [(0, got.alpha)])
    count0 = warm[0][0]
    edges += int(warm[0][1][0])
    if k:
        pre = accumulate_ranges(g, seed, 2, [(0, got.alpha)])
        edges += int(pre[0][1][0])
        ll, lu = orc.topk_lambdas(pre[0][0], got.alpha, k, lam)
        C, L, U = orc.compute_delta_lv(count0, got.alpha, got.omega, ll, lu, delta, eps)
    else:
        C, L, U = orc.compute_delta(count0, got.alpha, got.omega, lam, delta, eps)
    assert C == got.C
    bounds = list(range(0, got.tau, K)) + [got.tau]
    res = accumulate_ranges(g, seed, 0, [(a, b - a) for a, b in zip(bounds[:-1], bounds[1:])])
    counts = np.zeros(g.n, dtype=np.uint32)
    top = None
    tests = 0
    for i, (cnt, tot) in enumerate(res):
        counts += cnt
        edges += int(tot[0])
        tau_i = bounds[i + 1]
        last = i == len(res) - 1
        if k:
            stop, top, mf, mg = orc.check_stop_topk(counts, tau_i, got.omega, L, U, lam, k)
        else:
            stop, mf, mg = orc.check_stop(counts, tau_i, got.omega, L, U, lam)
        if tau_i < got.omega_cap:
            tests += 1
            if not last:
                assert not stop, tau_i
            else:
                assert stop == got.stopped_early, tau_i
    assert tests == got.checks
    assert np.array_equal(got.counts, counts)
    assert (got.max_f, got.max_g) == (mf, mg)
    assert int(got.totals[0]) == edges
    if k:
        assert list(got.topk) == list(top)
    return counts
