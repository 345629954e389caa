"""Parity cases run against the KADABRA_CHECKED build of the library (test
infrastructure; run in a child process by test_gpu_checked.py, since one
process loads one build).  Every table tier, the one-warp tier, the
16-byte-load scans and the segmented frontier scans are forced in turn on
undirected and directed graphs; per-sample results must equal the oracle's
and no index check may fail (a failure makes the call return
KADABRA_ERR_INTERNAL naming the check)."""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main(lib_path):
    from paper_1604_08553_gb300 import _build
    _build.build_kadabra = lambda *a, **k: lib_path
    from paper_1604_08553_gb300 import kadabra as kd, graphgen as gg
    import oracle as orc
    from conftest import random_graph
    assert kd.load_library()._name == lib_path
    kb = gg.from_edges(310, [(i, 150 + j) for i in range(150) for j in range(160)], name="K150,160")
    graphs = [gg.erdos_renyi(2000, 8.0, 1), random_graph(gg, 400, 0.01, 9, directed=True),
              gg.rmat(12, 16, 0.57, 0.19, 0.19, 1), gg.chung_lu(20000, 2.5, 12.0, 800.0, 4), kb,
              gg.path_graph(700)]
    flags = [0, kd.FLAG_LARGE_SHARED_TABLES, kd.FLAG_MEDIUM_TABLES, kd.FLAG_GLOBAL_TABLES, kd.FLAG_WARP_TIER,
             kd.FLAG_ASYNC_SCAN, kd.FLAG_FRONTIER_SEGMENTS]
    cases = 0
    for g in graphs:
        ref = orc.sample_paths(g, 3, 0, 100, 600, max_len=800)
        for f in flags:
            G = kd.kadabra_load_csr(g)
            try:
                G.set_flags(f)
                got = kd.kadabra_sample_paths(G, 3, 0, 100, 600, max_len=800)
            finally:
                G.free()
            assert np.array_equal(got.status, ref.status), (g.name, f)
            ok = ref.status == 0
            for a, b in ((got.st, ref.st), (got.paths, ref.paths), (got.stats, ref.stats)):
                assert np.array_equal(a[ok], b[ok]), (g.name, f)
            cases += 1
    # whole runs (device-driven loop) and a batch
    er = graphs[0]
    G = kd.kadabra_load_csr(er)
    try:
        r = kd.kadabra_run(G, 0.01, 0.1, 0, 2, check_interval=1000)
    finally:
        G.free()
    o = orc.run(er, 0.01, 0.1, seed=2, K=1000)
    assert r.tau == o.tau and np.array_equal(r.counts, o.counts)
    B = kd.Batch(graphs[:4])
    try:
        rb = B.run([0.03] * 4, [0.1] * 4, [5, 6, 7, 8])
        for i in range(4):
            rp = kd.kadabra_run(B.views[i], 0.03, 0.1, 0, 5 + i, check_interval=rb[i].check_interval)
            assert rb[i].tau == rp.tau and np.array_equal(rb[i].counts, rp.counts)
    finally:
        B.free()
    print(f"checked build: {cases} forced-tier cases, a run and a batch equal to the oracle and plain runs")


if __name__ == "__main__":
    main(sys.argv[1])
