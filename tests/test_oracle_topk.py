"""Pins of the oracle's top-k mode (Sec. 5, Alg. 2 with per-node targets,
Alg. 3) against hand-derived values, closed forms, special cases and the
ranking guarantee of Sec. 5.  CPU only."""

import math

import numpy as np
import pytest

from conftest import random_graph


# ------------------------------------------------------------------ Alg. 2, per-node targets
def test_compute_delta_lv_reduces_to_all_nodes(orc):
    """lambda_L = lambda_U = lambda everywhere is the all-nodes computeDelta."""
    rng = np.random.default_rng(11)
    n, alpha, lam, delta, eps = 2000, 300, 0.01, 0.1, 0.001
    omega = orc.omega(lam, delta, 17)
    count0 = rng.poisson(0.4, size=n).astype(np.uint32)
    C0, dl0, du0 = orc.compute_delta(count0, alpha, omega, lam, delta, eps)
    lamv = np.full(n, lam)
    C1, dl1, du1 = orc.compute_delta_lv(count0, alpha, omega, lamv, lamv, delta, eps)
    assert C0 == C1 and np.array_equal(dl0, dl1) and np.array_equal(du0, du1)


def test_compute_delta_lv_two_targets_root(orc):
    """N nodes with the same warm-up count, lambda_U = 2 lambda_L: with
    x = exp(-C/c_L) the condition is N (x + x^4) = delta/2 - eps*delta, a
    quartic solved here by numpy's polynomial roots; the bisection must land
    on that root (App. D)."""
    n, N, c0, alpha = 400, 25, 7, 250
    lam, delta, eps = 0.01, 0.1, 0.001
    omega = orc.omega(lam, delta, 13)
    count0 = np.zeros(n, dtype=np.uint32)
    count0[3::11][:N] = c0
    lamL = np.full(n, lam)
    lamU = np.full(n, 2 * lam)
    C, dl, du = orc.compute_delta_lv(count0, alpha, omega, lamL, lamU, delta, eps)
    cL = 2 * (c0 / alpha) * omega / lam**2
    target = delta / 2 - eps * delta
    roots = np.roots([N, 0, 0, N, -target])
    x = [r.real for r in roots if abs(r.imag) < 1e-12 and 0 < r.real < 1]
    assert len(x) == 1
    assert C == pytest.approx(-cL * math.log(x[0]), rel=1e-10)
    # lambda_U larger -> c_U smaller -> delta_U smaller -> ln(1/delta_U) larger
    hit = count0 > 0
    assert np.all(du[hit] > dl[hit])
    d = np.exp(-dl) + np.exp(-du)
    assert d.sum() <= delta / 2 * (1 + 1e-12)


# ------------------------------------------------------------------ Sec. 5 targets
def test_topk_lambdas_worked_example(orc):
    """Sec. 5 rules applied by hand.  alpha = 1000, k = 3, lambda = 0.02;
    b~ by id = .1 .39 .5 .01 .4 .2 .05 .04 .03 .02, so the ranking is
    v1..v10 = ids 2 4 1 5 0 6 7 8 9 3.
      top-k:   v1: U = 1 (nothing above), L = (.5-.4)/2 = .05
               v2: U = .05, L = (.4-.39)/2 = .005
               v3: U = .005, L = (.39-.2)/2 = .095
      others:  L = 1, U = b~(v3) - L(v3) - b~ = .295 - b~
      small gaps (< 2 lambda = .04): only v2-v3 (.01): both get .02 / .02."""
    cnt = np.array([100, 390, 500, 10, 400, 200, 50, 40, 30, 20], dtype=np.uint32)
    L, U = orc.topk_lambdas(cnt, 1000, 3, 0.02)
    expL = [1, 0.02, 0.05, 1, 0.02, 1, 1, 1, 1, 1]
    expU = [0.195, 0.02, 1, 0.285, 0.02, 0.095, 0.245, 0.255, 0.265, 0.275]
    assert L == pytest.approx(expL, rel=1e-12)
    assert U == pytest.approx(expU, rel=1e-12)


def test_topk_lambdas_clamp_example(orc):
    """k = 1, lambda = .02, b~ by id = .489 .5 .1 .49 0: v1 = id 1,
    L(v1) = (.5-.49)/2 = .005; others U = .5 - .005 - b~ (.005, .006, .395,
    .495 for ids 3, 0, 2, 4); the gap v1-v2 is small, so ids 1 and 3 get
    .02 / .02; id 0's U = .006 < lambda is raised to .02."""
    cnt = np.array([489, 500, 100, 490, 0], dtype=np.uint32)
    L, U = orc.topk_lambdas(cnt, 1000, 1, 0.02)
    assert L == pytest.approx([1, 0.02, 1, 0.02, 1], rel=1e-12)
    assert U == pytest.approx([0.02, 0.02, 0.395, 0.02, 0.495], rel=1e-12)


def test_topk_lambdas_intervals_meet(orc):
    """The Sec. 5 targets place adjacent intervals of well separated top-k
    nodes edge to edge (at the midpoint of the gap), and the upper ends of
    the other nodes at the lower end of v_k; none is below lambda."""
    rng = np.random.default_rng(12)
    for trial in range(20):
        n, alpha, lam = 60, 5000, 0.005
        cnt = rng.integers(0, 2500, size=n).astype(np.uint32)
        k = int(rng.integers(1, 8))
        L, U = orc.topk_lambdas(cnt, alpha, k, lam)
        assert np.all(L >= lam) and np.all(U >= lam)
        order = sorted(range(n), key=lambda v: (-int(cnt[v]), v))
        b = cnt.astype(np.float64) / alpha
        gap = [b[order[i]] - b[order[i + 1]] for i in range(n - 1)]
        for i in range(k - 1):  # 0-based pair (i, i+1) inside the top k
            near = [j for j in (i - 1, i, i + 1) if 0 <= j < n - 1 and j < k]
            if all(gap[j] >= 2 * lam for j in near):
                u, w = order[i], order[i + 1]
                assert b[u] - L[u] == pytest.approx(b[w] + U[w], abs=1e-12)
        vk = order[k - 1]
        if gap[k - 1] >= 2 * lam and (k < 2 or gap[k - 2] >= 2 * lam):
            for i in range(k, n):
                v = order[i]
                if U[v] > lam and not (i == k and gap[k - 1] < 2 * lam):
                    assert b[v] + U[v] == pytest.approx(b[vk] - L[vk], abs=1e-12)


# ------------------------------------------------------------------ Alg. 3
def test_check_stop_topk_implied_by_all_nodes(orc):
    """If every node has f, g <= lambda, no node is loose and Alg. 3 stops;
    the top-k list is the ranking by count (ties by id)."""
    rng = np.random.default_rng(13)
    for trial in range(30):
        n = int(rng.integers(5, 80))
        counts = rng.integers(0, 40, size=n).astype(np.uint32)
        L = rng.uniform(5, 15, size=n)
        U = rng.uniform(5, 15, size=n)
        tau = int(rng.choice([1000, 10**6, 10**8]))
        omega = 2e6
        k = int(rng.integers(1, n + 3))
        stop_all, mf, mg = orc.check_stop(counts, tau, omega, L, U, 0.01)
        stop_k, top, mf2, mg2 = orc.check_stop_topk(counts, tau, omega, L, U, 0.01, k)
        assert (mf, mg) == (mf2, mg2)
        if stop_all:
            assert stop_k
        exp = sorted(range(n), key=lambda v: (-int(counts[v]), v))[:min(k, n)]
        assert list(top) == exp


def test_check_stop_topk_separation(orc):
    """Every node loose (lambda tiny): Alg. 3 stops exactly when v_1's
    interval [b~ - f, b~ + g] lies above every other node's (k = 1), and for
    k = 2 also when v_1 and v_2 are separated from each other."""
    tau, omega, lam = 10000, 20000.0, 1e-6
    Lv = np.full(4, 0.05)

    def iv(c):
        f, g = orc.f_and_g(int(c), tau, omega, 0.05, 0.05)
        return c / tau - f, c / tau + g

    far = np.array([5000, 1000, 900, 0], dtype=np.uint32)
    near = np.array([5000, 4990, 900, 0], dtype=np.uint32)
    for counts in (far, near):
        lo1 = iv(counts[0])[0]
        sep1 = all(lo1 >= iv(c)[1] for c in counts[1:])
        stop, top, _, _ = orc.check_stop_topk(counts, tau, omega, Lv, Lv, lam, 1)
        assert stop == sep1 and list(top) == [0]
    assert orc.check_stop_topk(far, tau, omega, Lv, Lv, lam, 1)[0]
    assert not orc.check_stop_topk(near, tau, omega, Lv, Lv, lam, 1)[0]
    # k = 2: far has v1 > v2 > {v3, v4} separated only if 1000 vs 900 separate
    lo2 = iv(1000)[0]
    sep = lo2 >= iv(900)[1] and iv(5000)[0] >= iv(1000)[1]
    assert orc.check_stop_topk(far, tau, omega, Lv, Lv, lam, 2)[0] == sep


# ------------------------------------------------------------------ guarantee
@pytest.mark.slow
def test_topk_ranking_guarantee_over_seeds(orc, gg):
    """Sec. 5 / Thm. 1: with probability >= 1 - delta, for every node v_i of
    the returned top k and every node v_j ranked below it, bc(v_j) <=
    bc(v_i) + 2 lambda (pairs are ordered correctly or almost even).  Exact
    Brandes on small graphs, one-sided binomial test on the failure rate."""
    from scipy.stats import binomtest
    graphs = [gg.barabasi_albert(40, 2, 51), random_graph(gg, 30, 0.12, 52), gg.star_graph(20),
              random_graph(gg, 28, 0.12, 53, directed=True), gg.grid_graph(5, 5)]
    delta = 0.1
    fails = trials = 0
    for lam, k, seeds in ((0.05, 3, 60), (0.02, 5, 20)):
        for g in graphs:
            bc = orc.brandes(g)
            for seed in range(seeds):
                r = orc.run_topk(g, lam, delta, k, seed=7000 + seed, K=100)
                assert r.status == 0
                order = sorted(range(g.n), key=lambda v: (-int(r.counts[v]), v))
                assert list(r.topk) == order[:min(k, g.n)]
                bad = False
                for i in range(min(k, g.n)):
                    below = [order[j] for j in range(i + 1, g.n)]
                    if below and bc[below].max() > bc[order[i]] + 2 * lam + 1e-12:
                        bad = True
                fails += int(bad)
                trials += 1
    assert binomtest(fails, trials, delta, alternative="greater").pvalue > 1e-3
    assert fails / trials <= delta
