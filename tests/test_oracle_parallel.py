"""The oracle's process-pool driver (the multi-core CPU baseline) gives the
same hit counts and work counters as one sequential pass over the same
sample indices (CPU only): counts are order-independent integer sums."""

import numpy as np


def test_parallel_ranges_equal_sequential(orc, gg):
    from oracle.parallel import accumulate_ranges
    g = gg.barabasi_albert(1500, 3, 4)
    seed, first, count = 9, 123, 3000
    rc, ref_counts, ref_tot = orc.accumulate(g, seed, 0, first, count)
    assert rc == 0
    timing = {}
    [(counts, tot)] = accumulate_ranges(g, seed, 0, [(first, count)], processes=2, chunk=700, timing=timing)
    assert np.array_equal(counts, ref_counts)
    assert np.array_equal(tot, ref_tot)
    assert timing["processes"] == 2 and timing["work_s"] > 0


def test_parallel_several_ranges_and_domains(orc, gg):
    from oracle.parallel import accumulate_ranges
    g = gg.erdos_renyi(800, 6.0, 3)
    ranges = [(0, 500), (2**32 - 200, 400)]
    got = accumulate_ranges(g, 4, 1, ranges, processes=2, chunk=150)
    for (first, count), (counts, tot) in zip(ranges, got):
        rc, ref_counts, ref_tot = orc.accumulate(g, 4, 1, first, count)
        assert rc == 0
        assert np.array_equal(counts, ref_counts) and np.array_equal(tot, ref_tot)
