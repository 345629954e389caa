"""Benchmark of the KADABRA adaptive sampling loop on one GB300.

One step = one full run of the hot path (warm-up sampling, computeDelta, then
sample batches of K with the FP64 stop test after each, until the stop rule
holds or ceil(omega) samples) on one graph.  Workloads (--workload):

    chung_lu_1m (default): Chung-Lu power-law graph, n = 10^6, beta = 2.5,
        mean degree 16, max expected degree 10^4, largest component, int32
        CSR; lambda = 0.005, delta = 0.1, stop test every 2^16 samples.
    erdos_renyi_2k: G(n = 2000, mean degree 8), largest component;
        lambda = 0.01, delta = 0.1, stop test every 1000 samples.
    rmat_24: directed R-MAT, scale 24, edge factor 16, (a, b, c) = (0.57,
        0.19, 0.19), self-loops and duplicate arcs removed, all 2^24 ids kept,
        forward and reverse CSR; all-nodes mode at lambda = 0.0025,
        delta = 0.1, stop test every 2^16 samples.
    rmat_24_topk: the same graph in top-k mode (Sec. 5, Alg. 3), k = 10.
    rmat_22: the scale-22 graph of the same recipe (for profiler captures).
    batched: 64 Barabasi-Albert graphs of uneven sizes, one batched run
        against the same graphs run one at a time (results on the device).
    serving: 2000 Poisson-arriving jobs on 16 graphs through the serving
        engine; latency percentiles and jobs/s.
    edge_exponent: edges scanned per sample as a power of m on graphs of
        growing size (a diagnostic of the Sec. 4 theorem, no timing).

Prints ONE JSON line (rank 0).  `value` is sampled paths per second over the
whole run (warm-up + main loop) with the graph resident on the device;
`e2e` repeats the measurement through the C ABI with host buffers (upload of
the CSR from pinned host memory, run, copy of counts and b~ into pinned host
memory) inside the timed region.  `roofline` relates the sampler batch's
algorithmic bytes to the measured HBM peak, `roofline_l2` (graphs whose CSR
fits in L2) to the measured L2 read rate, with the same work counted in 32 B
sectors beside it; `cpu_baseline` times the oracle on the host's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "paths/sec & time-to-(lambda,delta) per graph, batched vs plain on GPU; % HBM roofline"
# Single-graph workloads.  `sampler_dram_bytes`: DRAM bytes (read + write) of
# one sampler batch of K samples, summed over its launches, from an ncu capture
# summarised under profiles/ (None until captured for the current kernels).
WORKLOADS = {
    "chung_lu_1m": dict(family="chung_lu", n=1_000_000, beta=2.5, mean_deg=16.0, max_deg=10_000.0, graph_seed=1,
                        lcc=True, lam=0.005, delta=0.1, check_interval=1 << 16,
                        sampler_dram_bytes=99_782_571 + 23_815_338 + 64_768),
    "erdos_renyi_2k": dict(family="erdos_renyi", n=2000, mean_deg=8.0, graph_seed=1, lcc=True, lam=0.01,
                           delta=0.1, check_interval=1000, sampler_dram_bytes=None),
    "rmat_24": dict(family="rmat", scale=24, edge_factor=16, a=0.57, b=0.19, c=0.19, graph_seed=1, lam=0.0025,
                    delta=0.1, check_interval=1 << 16, sampler_dram_bytes=None),
    # the scale-22 graph of the same recipe: the size the ncu counters are captured at
    "rmat_22": dict(family="rmat", scale=22, edge_factor=16, a=0.57, b=0.19, c=0.19, graph_seed=1, lam=0.0025,
                    delta=0.1, check_interval=1 << 16,
                    sampler_dram_bytes=632_693_077 + 149_157_888 + 65_792),
    "rmat_24_topk": dict(family="rmat", scale=24, edge_factor=16, a=0.57, b=0.19, c=0.19, graph_seed=1, lam=0.0025,
                         delta=0.1, check_interval=1 << 16, sampler_dram_bytes=None, k=10),
}
WORKLOAD = WORKLOADS["chung_lu_1m"]
L2_FLUSH_BYTES = 512 << 20


def make_graph():
    from paper_1604_08553_gb300 import graphgen
    w = WORKLOAD
    if w["family"] == "chung_lu":
        return graphgen.chung_lu(w["n"], w["beta"], w["mean_deg"], w["max_deg"], w["graph_seed"], lcc=w["lcc"])
    if w["family"] == "erdos_renyi":
        return graphgen.erdos_renyi(w["n"], w["mean_deg"], w["graph_seed"], lcc=w["lcc"])
    return graphgen.rmat(w["scale"], w["edge_factor"], w["a"], w["b"], w["c"], w["graph_seed"])


def workload_name():
    w = WORKLOAD
    tail = f"lambda={w['lam']} delta={w['delta']} K={w['check_interval']}"
    if w.get("k"):
        tail = f"top-k k={w['k']}; " + tail
    if w["family"] == "chung_lu":
        return (f"chung_lu n={w['n']} beta={w['beta']} mean_deg={w['mean_deg']:g} max_deg={w['max_deg']:g} "
                f"lcc; {tail}")
    if w["family"] == "erdos_renyi":
        return f"erdos_renyi n={w['n']} mean_deg={w['mean_deg']:g} lcc; {tail}"
    return (f"rmat scale={w['scale']} edge_factor={w['edge_factor']} a={w['a']} b={w['b']} c={w['c']} directed, "
            f"all ids; {tail}")


def workload_config(g, extra=None):
    w = WORKLOAD
    cfg = {
        "workload": workload_name(),
        "nodes": int(g.n), "arcs": int(g.m), "directed": bool(g.directed), "lambda": w["lam"],
        "delta": w["delta"], "check_interval": w["check_interval"], "graph_seed": w["graph_seed"],
        "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB write)",
    }
    if extra:
        cfg.update(extra)
    return cfg


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        """Starts sampling every 20 ms (every 200 ms if that yields nothing)
        and returns once the first sample has arrived, so that the sampler is
        running before the timed region opens."""
        for interval in ("20", "200"):
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                     "--format=csv,noheader,nounits", "-lms", interval],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except (FileNotFoundError, OSError):
                self.proc = None
                return
            self.lines = []
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 3.0:
                time.sleep(0.01)
            if self.lines:
                return
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=5)
        self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax = float(p[1])
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# What the algorithmic bytes count (reported beside each roofline)
BYTES_BASIS = ("work counters of the paper's search: every arc of each expanded row and every adjacency position "
               "up to each backtracking pick; the kernel reads fewer (bisected backtracking steps, and on graphs "
               "beyond L2 long touching-level rows searched instead of scanned)")


def algorithmic_bytes(totals, hits):
    """Bytes the sampler must touch (per batch): 8 B per expanded node (two
    offsets), 4 B per scanned arc (adjacency) + 4 B per scanned arc (visited
    probe), 12 B per node kept in a level (state + sigma), 8 B per sigma
    addition, 4 B per hit-counter update, 4 B per adjacency entry read while
    backtracking."""
    t = totals
    return (8 * t[1] + 8 * t[0] + 12 * t[2] + 8 * t[3] + 4 * hits + 4 * t[6])


def sector_bytes(totals, hits):
    """The same work at the granularity of 32 B sectors of L2 and DRAM: the
    two offsets of an expanded node share one sector; its row's arcs are read
    contiguously (4 B each plus about one partial sector per row); a hit
    counter update moves one sector; backtracking reads one offset sector and
    one partial row sector per path node plus 4 B per scanned position.  The
    visited-set probes, level lists and sigma updates of the shared-memory
    tiers cost no L2 or DRAM bytes."""
    t = totals
    return 64 * t[1] + 4 * t[0] + 32 * hits + 4 * t[6] + 64 * t[7]


def step_spread(times, results):
    """Per final tau (the check schedule fixes a few values of tau, and the
    step time follows it): the median step time and the slowest step over
    that median."""
    by = {}
    for t, r in zip(times, results):
        by.setdefault(int(r.tau), []).append(1e3 * t)
    med = {tau: statistics.median(v) for tau, v in by.items()}
    return {"step_ms_median_by_tau": {str(k): round(v, 3) for k, v in sorted(med.items())},
            "step_max_over_median": round(max(max(v) / med[k] for k, v in by.items()), 3)}


def replica_seed(rank: int, step: int) -> int:
    """Seed of a timed step on a rank: replicas sample different paths."""
    return 1 + step + 7919 * rank


def reduce_replicas(dist, seconds: float, paths: float, device: str):
    """Whole-job figures of independent replicas, one per rank: the slowest
    rank's time and the paths of all ranks.  Every rank calls it; dist is
    torch.distributed (any backend) or None for a single process."""
    if dist is None:
        return float(seconds), float(paths)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    p = torch.tensor([float(paths)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t[0]), float(p[0])


def run_launches(r, w):
    """Kernels one run launches.  All-nodes mode: the warm-up batch, the
    warm-up count compaction (3), the main loop's rounds (CUDA graph), the
    final test and b~.  Top-k mode: the preliminary + warm-up
    batch, the preliminary selection (2), the compaction (3), the fill and
    scatter of ln(1/delta) (2), the main-loop batches, three kernels per
    Alg. 3 test (checks + the final one) and b~."""
    rounds = -(-int(r.tau) // w["check_interval"])
    spb = sampler_launches_per_batch(r)
    # the first main-loop batch shares the warm-up's launch; a final full test
    # runs only when no test held (a test that held gave the maxima)
    final = 0 if r.stopped_early else 1
    if w.get("k"):
        return spb * rounds + 2 + 3 + 2 + 3 * int(r.checks) + 3 * final + 1
    # one-graph all-nodes runs with more than 4 possible rounds test the first
    # round from the host and loop on the device from the second: a setup
    # kernel, then per round the sampler batch and the stop test (whose last
    # block closes the round); shorter runs take host rounds (batch, then a
    # test if tau < cap)
    cap_rounds = -(-int(r.omega_cap) // w["check_interval"])
    if cap_rounds > 4:
        loop = 1 + (spb + 1) * (rounds - 1) if rounds > 1 else 0
        return spb + 3 + 1 + loop + final + 1
    return spb * rounds + 3 + int(r.checks) + final + 1


def sampler_launches_per_batch(r=None):
    """Kernels of one sampler batch: the shared-memory tier and the two
    escalation tiers (which exit at once when nothing was queued to them),
    plus the one-warp-per-sample tier in front when the run used it."""
    return 3 + (1 if r is not None and getattr(r, "warp_tier", 0) else 0)


def cpu_baseline(g, seconds_cap=20.0):
    """The oracle (single-threaded, as it stands) on a bounded sample of the
    same workload: the first main-loop samples of seed 1."""
    import oracle
    w = WORKLOAD
    count = 0
    t0 = time.perf_counter()
    chunk = 1000
    first = 0
    while time.perf_counter() - t0 < seconds_cap * 0.5 and count < 50_000:
        rc, _, _ = oracle.accumulate(g, 1, 0, first, chunk)
        if rc != 0:
            raise RuntimeError(f"oracle status {rc}")
        first += chunk
        count += chunk
    dt = time.perf_counter() - t0
    return {"value": count / dt, "unit": "paths/s", "cores": 1, "kind": "oracle",
            "sample": f"main-loop samples 0..{count - 1} (seed 1) of the {workload_name()} workload, "
                      f"single-threaded oracle, {dt:.1f} s"}


def cpu_baseline_multicore(g, rate_single: float, seconds: float = 3.0):
    """The oracle's sampler over disjoint sample-index ranges on all host
    cores (process pool started with spawn; counts are order-independent
    sums, so the result equals one sequential pass), timed without the pool's
    start-up."""
    from oracle.parallel import accumulate_ranges
    procs = max(1, os.cpu_count() or 1)
    total = max(procs * 200, int(rate_single * seconds) * procs)
    timing = {}
    accumulate_ranges(g, 1, 0, [(0, total)], processes=procs, chunk=max(200, total // (4 * procs)), timing=timing)
    return {"value": total / timing["work_s"], "unit": "paths/s", "cores": timing["processes"], "kind": "oracle",
            "sample": f"main-loop samples 0..{total - 1} (seed 1) of the {workload_name()} workload, oracle over "
                      f"disjoint index ranges in {timing['processes']} processes, {timing['work_s']:.1f} s"}


def l2_read_peak_gbs():
    """Read rate of an L2-resident 32 MB buffer, re-read 50 times in one
    launch with L2-only loads (kadabra_l2_read_probe): the L2 roofline's
    denominator."""
    from paper_1604_08553_gb300 import kadabra as kd
    return max(kd.kadabra_l2_read_probe(32 << 20, 50) for _ in range(3))


def run_reference(args, rank, world):
    """The oracle on the host cores (the reference arm for this paper-only tier)."""
    g = make_graph()
    import oracle
    per_step = 3000
    for i in range(args.warmup):
        oracle.accumulate(g, 100 + i, 0, 0, 300)
    t0 = time.perf_counter()
    for i in range(args.steps):
        rc, _, _ = oracle.accumulate(g, 1, 0, i * per_step, per_step)
        assert rc == 0
    dt = time.perf_counter() - t0
    value = args.steps * per_step / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64+f64",
        "data": "synthetic",
        "config": workload_config(g, {"sample": f"{per_step} main-loop samples per step"}),
        "cpu_baseline": {"value": value, "unit": "paths/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} main-loop samples per step, single-threaded oracle"},
        "e2e": {"value": value, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def sampler_only(kd, G, g, launches):
    """Times `launches` sampler batches of K main-loop samples (the dominant
    kernel), after one untimed run that autotunes the sampler setup the
    batches then use.  The batches sit in the NVTX range "sampler_batches"
    (for profiler captures)."""
    import torch
    K = WORKLOAD["check_interval"]
    d_counts = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    d_tot = torch.zeros(kd.NSTAT, dtype=torch.int64, device="cuda")
    r = kd.kadabra_run(G, WORKLOAD["lam"], WORKLOAD["delta"], WORKLOAD.get("k", 0), 1,
                       check_interval=K, want_host=False, d_counts=d_counts)
    torch.cuda.synchronize()
    d_counts.zero_()
    out = []
    torch.cuda.nvtx.range_push("sampler_batches")
    for i in range(launches):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        kd.kadabra_sample_batch(G, 1, 0, i * K, K, d_counts, d_tot)
        ev1.record()
        ev1.synchronize()
        kd.kadabra_sync_status(G)
        out.append(ev0.elapsed_time(ev1))
    torch.cuda.nvtx.range_pop()
    tot = d_tot.cpu().numpy()
    print(json.dumps({"sampler_ms": out, "samples": K * launches, "edges": int(tot[0]),
                      "bt_scanned": int(tot[6]), "ctas_per_sm": int(r.ctas_per_sm), "warp_tier": int(r.warp_tier),
                      "workload": workload_config(g)["workload"]}), flush=True)


BATCHED = dict(graphs=64, n_lo=10_000, n_hi=2_000_000, m_lo=4, m_hi=16, lam=0.01, delta=0.1, seed=2024)


def make_batched_graphs():
    """64 Barabasi-Albert graphs: n log-uniform in [10^4, 2*10^6], attachment m
    uniform in {4..16}, one seed per graph (generated in parallel threads)."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_1604_08553_gb300 import graphgen
    b = BATCHED
    rng = np.random.default_rng(b["seed"])
    ns = np.exp(rng.uniform(np.log(b["n_lo"]), np.log(b["n_hi"]), b["graphs"])).astype(np.int64)
    ms = rng.integers(b["m_lo"], b["m_hi"] + 1, b["graphs"])
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        return list(ex.map(lambda i: graphgen.barabasi_albert(int(ns[i]), int(ms[i]), b["seed"] + 1 + i),
                           range(b["graphs"])))


def batched_vs_plain(kd, graphs, warmup: int, steps: int):
    """Time-to-(lambda, delta) of the uneven multi-graph workload: one batched
    run (all graphs per launch) against the same graphs run one at a time on
    the same device arena, results on the device in both arms and compared
    after each timed pair (identical per graph: tau and counts)."""
    import torch
    b = BATCHED
    G = len(graphs)
    B = kd.Batch(graphs)
    lam, delta = [b["lam"]] * G, [b["delta"]] * G
    stream = torch.cuda.current_stream()
    dc_b = [torch.zeros(g.n, dtype=torch.int32, device="cuda") for g in graphs]
    db_b = [torch.zeros(g.n, dtype=torch.float64, device="cuda") for g in graphs]
    dc_p = [torch.zeros(g.n, dtype=torch.int32, device="cuda") for g in graphs]
    db_p = [torch.zeros(g.n, dtype=torch.float64, device="cuda") for g in graphs]

    def batched(seed0):
        return B.run(lam, delta, [seed0 + i for i in range(G)], stream=stream.cuda_stream, d_counts=dc_b,
                     d_btilde=db_b, want_host=False)

    def plain(seed0):
        return [kd.kadabra_run(B.views[i], lam[i], delta[i], 0, seed0 + i, check_interval=0,
                               stream=stream.cuda_stream, d_counts=dc_p[i], d_btilde=db_p[i], want_host=False)
                for i in range(G)]

    for i in range(warmup):
        batched(100 * (i + 1))
        plain(100 * (i + 1))
    tb, tp, paths, same = [], [], 0, True
    for i in range(steps):
        seed0 = 7 + 1000 * i
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rb = batched(seed0)
        torch.cuda.synchronize()
        tb.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        rp = plain(seed0)
        torch.cuda.synchronize()
        tp.append(time.perf_counter() - t0)
        for q, (x, y) in enumerate(zip(rb, rp)):
            same = same and x.tau == y.tau and bool(torch.equal(dc_b[q], dc_p[q]))
        paths += sum(r.alpha + r.tau for r in rb)
    B.free()
    return {"graphs": G, "nodes": int(sum(g.n for g in graphs)), "arcs": int(sum(g.m for g in graphs)),
            "time_to_lambda_delta_batched_ms": [round(1e3 * t, 2) for t in tb],
            "time_to_lambda_delta_plain_ms": [round(1e3 * t, 2) for t in tp],
            "batched_speedup": sum(tp) / sum(tb), "paths_per_s_batched": paths / sum(tb),
            "identical_results": same}


def batched_workload_name():
    b = BATCHED
    return (f"batched: {b['graphs']} Barabasi-Albert graphs, n log-uniform in [{b['n_lo']}, {b['n_hi']}], "
            f"m uniform in {{{b['m_lo']}..{b['m_hi']}}}; lambda={b['lam']} delta={b['delta']}; "
            "check interval max(1024, ceil(omega/32))")


def run_batched(args, kd, rank, world):
    """The batched workload alone: one JSON line whose value is the batched
    arm's paths/s."""
    graphs = make_batched_graphs()
    r = batched_vs_plain(kd, graphs, args.warmup, args.steps)
    if not r["identical_results"]:
        raise RuntimeError("batched and plain runs differ")
    if rank == 0:
        tb = r["time_to_lambda_delta_batched_ms"]
        line = {
            "metric": METRIC, "value": r["paths_per_s_batched"], "unit": "paths/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(tb) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
            "config": {
                "workload": batched_workload_name(),
                "nodes": r["nodes"], "arcs": r["arcs"],
                "time_to_lambda_delta_batched_ms": tb,
                "time_to_lambda_delta_plain_ms": r["time_to_lambda_delta_plain_ms"],
                "batched_speedup": r["batched_speedup"],
                "results": "identical per graph (tau, counts) in batched and plain runs; results kept on the device",
            },
        }
        print(json.dumps(line), flush=True)


def rmat24_roofline(kd, launches: int = 4):
    """The HBM-bound configuration's sampler roofline: R-MAT scale 24 (forward
    and reverse CSR, 2.2 GB, beyond L2), batches of 2^16 main-loop samples
    timed with CUDA events on the launching stream, algorithmic bytes from
    the work counters, against the measured HBM copy rate."""
    import torch
    global WORKLOAD
    saved = WORKLOAD
    WORKLOAD = WORKLOADS["rmat_24"]
    try:
        g = make_graph()
        G = kd.kadabra_load_csr(g)
        K = WORKLOAD["check_interval"]
        stream = torch.cuda.current_stream()
        d_counts = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        d_tot = torch.zeros(kd.NSTAT, dtype=torch.int64, device="cuda")
        ts, bs = [], []
        for i in range(launches + 1):
            d_counts.zero_()
            d_tot.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            kd.kadabra_sample_batch(G, 1, 0, i * K, K, d_counts, d_tot, stream=stream.cuda_stream)
            ev1.record(stream)
            ev1.synchronize()
            kd.kadabra_sync_status(G, stream.cuda_stream)
            if i == 0:
                continue
            ts.append(ev0.elapsed_time(ev1) / 1e3)
            bs.append(algorithmic_bytes(d_tot.cpu().numpy(), int(d_counts.sum().item())))
        G.free()
        peak, src = peaks()
        t, by = sum(ts) / len(ts), sum(bs) / len(bs)
        return {"workload": workload_name(), "nodes": int(g.n), "arcs": int(g.m), "bound": "hbm",
                "achieved": by / t / 1e9, "peak": peak, "unit": "GB/s", "frac": by / t / 1e9 / peak,
                "traffic": WORKLOAD["sampler_dram_bytes"], "bytes_per_launch": by, "launch_ms": 1e3 * t,
                "samples_per_launch": K, "paths_per_s": K / t, "peak_source": src, "bytes_basis": BYTES_BASIS}
    finally:
        WORKLOAD = saved


SERVING = dict(jobs=2000, rate=50.0, graphs=16, n_lo=2_000, n_hi=4_000_000, lams=(0.02, 0.01, 0.005), delta=0.1,
               seed=77)


def make_serving_pool():
    """Graph pool of the serving workload: Erdos-Renyi (mean degree 8),
    Chung-Lu (beta 2.5, mean degree 16) and Barabasi-Albert (m in {4..16})
    in turn, n log-uniform in [2*10^3, 4*10^6], one seed per graph."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_1604_08553_gb300 import graphgen
    b = SERVING
    rng = np.random.default_rng(b["seed"])
    ns = np.exp(rng.uniform(np.log(b["n_lo"]), np.log(b["n_hi"]), b["graphs"])).astype(np.int64)
    ms = rng.integers(4, 17, b["graphs"])

    def make(i):
        n, sd = int(ns[i]), b["seed"] + 1 + i
        if i % 3 == 0:
            return graphgen.erdos_renyi(n, 8.0, sd)
        if i % 3 == 1:
            return graphgen.chung_lu(n, 2.5, 16.0, float(min(10_000, max(50, n // 20))), sd)
        return graphgen.barabasi_albert(n, int(ms[i]), sd)

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        return list(ex.map(make, range(b["graphs"])))


def run_serving(args, kd, rank, world):
    """Poisson arrivals of KADABRA jobs (all-nodes, or top-k with k in
    {10, 50}; lambda in {0.02, 0.01, 0.005}; delta = 0.1) on a pool of
    device-resident graphs, served by the continuous-batching engine.
    Latency = result ready - submitted (the engine's clock)."""
    import threading
    b = SERVING
    njobs = args.serve_jobs or b["jobs"]
    graphs = make_serving_pool()
    handles = [kd.kadabra_load_csr(g) for g in graphs]
    rng = np.random.default_rng(b["seed"] + 1000)
    gap = rng.exponential(1.0 / b["rate"], njobs)
    spec = []
    for i in range(njobs):
        gi = int(rng.integers(0, len(graphs)))
        mode = rng.random()
        k = 0 if mode < 0.5 else (10 if mode < 0.75 else 50)
        lam = float(b["lams"][int(rng.integers(0, len(b["lams"])))])
        spec.append((gi, lam, k, 1 + i))
    # warm-up: a few jobs through the engine (first launches, allocations)
    for i in range(max(3, args.warmup)):
        gi, lam, k, seed = spec[i % njobs]
        jid = kd.kadabra_submit(handles[gi], lam, b["delta"], k, 10_000 + seed, check_interval=0)
        kd.kadabra_poll(jid, graphs[gi].n, k, wait=True)
    results = [None] * njobs
    ids = [None] * njobs
    submitted = threading.Semaphore(0)

    def collect():
        for i in range(njobs):
            submitted.acquire()
            gi, lam, k, seed = spec[i]
            results[i] = kd.kadabra_poll(ids[i], graphs[gi].n, k, wait=True)

    th = threading.Thread(target=collect)
    th.start()
    t0 = time.perf_counter()
    t_next = t0
    for i in range(njobs):
        t_next += gap[i]
        d = t_next - time.perf_counter()
        if d > 0:
            time.sleep(d)
        gi, lam, k, seed = spec[i]
        ids[i] = kd.kadabra_submit(handles[gi], lam, b["delta"], k, seed, check_interval=0)
        submitted.release()
    th.join()
    wall = max(r.t_done for r in results) - min(r.t_submit for r in results)
    lat = np.array([r.t_done - r.t_submit for r in results]) * 1e3
    paths = sum(int(r.alpha) * (2 if spec[i][2] else 1) + int(r.tau) for i, r in enumerate(results))
    # the same result alone as in the mix, for a few jobs
    check = [int(x) for x in np.linspace(0, njobs - 1, 6)]
    for i in check:
        gi, lam, k, seed = spec[i]
        alone = kd.kadabra_run(handles[gi], lam, b["delta"], k, seed, check_interval=0)
        r = results[i]
        assert alone.tau == r.tau and np.array_equal(alone.counts, r.counts), f"job {i} differs alone"
        if k:
            assert np.array_equal(alone.topk, r.topk), f"job {i} ranking differs alone"
    kd.kadabra_serve_shutdown()
    for h in handles:
        h.free()
    if rank == 0:
        line = {
            "metric": METRIC, "value": paths / wall, "unit": "paths/s", "n_gpus": world, "steps": njobs,
            "warmup": max(3, args.warmup), "ms_per_step": float(np.mean(lat)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
            "config": {
                "workload": (f"serving: {njobs} Poisson jobs at {b['rate']:g}/s on {len(graphs)} graphs "
                             f"(Erdos-Renyi / Chung-Lu / Barabasi-Albert, n log-uniform in [{b['n_lo']}, "
                             f"{b['n_hi']}]); all-nodes or top-k k in {{10, 50}}; lambda in {list(b['lams'])}, "
                             f"delta={b['delta']}; check interval max(1024, ceil(omega/32))"),
                "nodes_per_graph": [int(g.n) for g in graphs], "arcs_total": int(sum(g.m for g in graphs)),
                "latency_p50_ms": float(np.percentile(lat, 50)), "latency_p99_ms": float(np.percentile(lat, 99)),
                "latency_max_ms": float(lat.max()), "jobs_per_s": njobs / wall, "offered_jobs_per_s": b["rate"],
                "wall_s": wall, "results": "6 jobs re-run alone: identical tau, counts, ranking",
            },
        }
        print(json.dumps(line), flush=True)


def run_edge_exponent(args, kd, rank, world):
    """Edges scanned per sample as a power of m (Sec. 4 theorem; the Sec. 6
    figure plots alpha = log(m_avg) / log(m) per graph).  For a family of
    graphs of growing size, 2^16 main-loop samples each on the GPU; m_avg =
    arcs scanned by the bb-BFS per sample (work counter EDGES).  Prints the
    per-graph alpha and the least-squares slope of log m_avg against log m:
    the theorem gives 1/2 + o(1) for degrees with a finite second moment (ER)
    and (4 - beta)/2 + o(1) for power-law degrees with 2 < beta < 3 (Chung-Lu,
    beta = 2.5: 0.75); the directed R-MAT family, outside the theorem's
    models, is measured beside them.  Not a timing; rank 0 only."""
    import torch
    from paper_1604_08553_gb300 import graphgen
    if rank != 0:
        return
    samples = 1 << 16
    families = {
        "erdos_renyi_d8": lambda n: graphgen.erdos_renyi(n, 8.0, 1),
        # natural cutoff of the weights, n^(1/(beta-1)): 10^4 at n = 10^6 as in the Chung-Lu workload
        "chung_lu_b2.5_d16": lambda n: graphgen.chung_lu(n, 2.5, 16.0, float(n) ** (1 / 1.5), 1),
        # directed, every id kept: many (s, t) pairs are disconnected and end early
        "rmat_ef16_directed": lambda n: graphgen.rmat(int(n).bit_length() - 1, 16, 0.57, 0.19, 0.19, 1),
    }
    out = {}
    for fam, make in families.items():
        rows = []
        for lg in range(14, 22):
            g = make(1 << lg)
            G = kd.kadabra_load_csr(g)
            c = torch.zeros(g.n, dtype=torch.int32, device="cuda")
            t = torch.zeros(kd.NSTAT, dtype=torch.int64, device="cuda")
            kd.kadabra_sample_batch(G, 1, 0, 0, samples, c, t)
            kd.kadabra_sync_status(G)
            G.free()
            m_avg = int(t[0].item()) / samples
            rows.append({"n": int(g.n), "m": int(g.m), "m_avg": round(m_avg, 2),
                         "alpha": round(float(np.log(m_avg) / np.log(g.m)), 4)})
        x = np.log([r["m"] for r in rows])
        y = np.log([r["m_avg"] for r in rows])
        slope = float(np.polyfit(x, y, 1)[0])
        out[fam] = {"slope": round(slope, 4), "graphs": rows}
    print(json.dumps({"metric": "edges scanned per sample as m^alpha (bb-BFS, Sec. 4)", "unit": "exponent",
                      "samples_per_graph": samples, "data": "synthetic", "families": out}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sampler-only", type=int, default=0, metavar="LAUNCHES",
                    help="only time LAUNCHES sampler batches of K samples (for profilers)")
    ap.add_argument("--serve-jobs", type=int, default=0, help="serving workload: jobs (default 2000)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the batched-vs-plain and R-MAT 24 roofline measurements")
    ap.add_argument("--workload", default="chung_lu_1m",
                    choices=[*WORKLOADS, "batched", "serving", "edge_exponent"],
                    help="one-graph workload (default chung_lu_1m), or batched: 64 uneven Barabasi-Albert graphs, "
                         "batched run against one-graph-at-a-time runs, or serving, or edge_exponent: the "
                         "edges-per-sample exponent diagnostic (no timing)")
    args = ap.parse_args()
    global WORKLOAD
    if args.workload in WORKLOADS:
        WORKLOAD = WORKLOADS[args.workload]
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, rank, world)
        return

    import torch
    from paper_1604_08553_gb300 import kadabra as kd

    torch.cuda.set_device(local_rank)
    if args.workload == "batched":
        run_batched(args, kd, rank, world)
        return
    if args.workload == "serving":
        run_serving(args, kd, rank, world)
        return
    if args.workload == "edge_exponent":
        run_edge_exponent(args, kd, rank, world)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    g = make_graph()
    w = WORKLOAD
    G = kd.kadabra_load_csr(g)
    if args.sampler_only:
        sampler_only(kd, G, g, args.sampler_only)
        G.free()
        return
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    d_counts = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    d_btilde = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(seed):
        return kd.kadabra_run(G, w["lam"], w["delta"], w.get("k", 0), seed, check_interval=w["check_interval"],
                              stream=sp,
                              d_counts=d_counts, d_btilde=d_btilde, want_host=False)

    # the clock sampler starts before the warm-up steps, so that its own
    # start-up does not land in the timed region
    clocks = ClockSampler(local_rank)
    clocks.start()
    for i in range(args.warmup):
        step(1000 + i)

    # ---- timed region: device-resident graph, one full adaptive run per step
    barrier()
    torch.cuda.synchronize()
    times, paths, launches, results, edges = [], 0, 0, [], 0
    for i in range(args.steps):
        flush.fill_(float(i))
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        r = step(replica_seed(rank, i))
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1) / 1e3)
        paths += r.alpha + r.tau
        edges += int(r.totals[0])
        launches += run_launches(r, w)
        results.append(r)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total, paths = reduce_replicas(dist, sum(times), paths, "cuda")
    value = paths / total

    # ---- dominant kernel: the sampler, timed per launch on its stream
    K = w["check_interval"]
    d_tot = torch.zeros(kd.NSTAT, dtype=torch.int64, device="cuda")
    samp_times, samp_bytes, samp_sectors = [], [], []
    for i in range(4):
        flush.fill_(float(i))
        d_counts.zero_()
        d_tot.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        kd.kadabra_sample_batch(G, 1, 0, i * K, K, d_counts, d_tot, stream=sp)
        ev1.record(stream)
        ev1.synchronize()
        kd.kadabra_sync_status(G, sp)
        if i == 0:
            continue  # first launch of this shape: warm-up
        samp_times.append(ev0.elapsed_time(ev1) / 1e3)
        hits = int(d_counts.sum().item())
        samp_bytes.append(algorithmic_bytes(d_tot.cpu().numpy(), hits))
        samp_sectors.append(sector_bytes(d_tot.cpu().numpy(), hits))
    avg_t = sum(samp_times) / len(samp_times)
    avg_b = sum(samp_bytes) / len(samp_bytes)
    avg_s = sum(samp_sectors) / len(samp_sectors)
    peak, peak_src = peaks()
    achieved = avg_b / avg_t / 1e9
    tot_np = d_tot.cpu().numpy()

    # ---- end to end through the C ABI with host buffers: the CSR in pinned
    # host memory is uploaded by kadabra_load_csr inside the timed region, and
    # the counts and b~ come back into pinned host buffers
    e2e_steps = max(2, min(args.steps, 3))

    def pinned(a, dtype):
        t = torch.empty(len(a), dtype=dtype, pin_memory=True)
        t.numpy()[:] = a
        return t

    class PinnedCSR:
        pass

    gp = PinnedCSR()
    gp.n, gp.directed = g.n, g.directed
    keep = [pinned(g.row_ptr, torch.int32), pinned(g.col, torch.int32)]
    if g.directed:
        keep += [pinned(g.rrow_ptr, torch.int32), pinned(g.rcol, torch.int32)]
    gp.row_ptr, gp.col = keep[0].numpy(), keep[1].numpy()
    gp.rrow_ptr, gp.rcol = (keep[2].numpy(), keep[3].numpy()) if g.directed else (None, None)
    counts_t = torch.zeros(g.n, dtype=torch.int32, pin_memory=True)
    btilde_t = torch.zeros(g.n, dtype=torch.float64, pin_memory=True)
    counts_h = counts_t.numpy().view(np.uint32)
    btilde_h = btilde_t.numpy()
    h2d = (4 * (g.n + 1) + 4 * g.m) * (2 if g.directed else 1)  # forward (+ reverse) CSR
    d2h = 4 * g.n + 8 * g.n
    torch.cuda.synchronize()
    e2e_paths = 0
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        Gh = kd.kadabra_load_csr(gp)
        r = kd.kadabra_run(Gh, w["lam"], w["delta"], w.get("k", 0), 500 + i, check_interval=K, counts=counts_h,
                           btilde=btilde_h)
        Gh.free()
        e2e_paths += r.alpha + r.tau
    torch.cuda.synchronize()
    e2e_dt = time.perf_counter() - t0
    e2e_dt, e2e_paths = reduce_replicas(dist, e2e_dt, e2e_paths, "cuda")
    e2e_value = e2e_paths / e2e_dt

    # the metric's batched-vs-plain comparison and the HBM-bound roofline,
    # measured on the same box after the timed steps (default workload, N=1)
    extras = {}
    if world == 1 and args.workload == "chung_lu_1m" and not args.no_extras:
        extras["batched_vs_plain"] = batched_vs_plain(kd, make_batched_graphs(), 1, 3)
        extras["batched_vs_plain"]["workload"] = batched_workload_name()
        extras["roofline_rmat_24"] = rmat24_roofline(kd)

    cpu = cpu_multi = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(g)
        cpu_multi = cpu_baseline_multicore(g, cpu["value"])
    # L2 roofline, for graphs whose CSR fits in L2
    import torch
    csr_bytes = (4 * (g.n + 1) + 4 * g.m) * (2 if g.directed else 1)
    l2_size = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    roof_l2 = None
    if csr_bytes < l2_size:
        l2 = l2_read_peak_gbs()
        sec = avg_s / avg_t / 1e9
        roof_l2 = {"bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s", "frac": achieved / l2,
                   "peak_source": "measured here: kadabra_l2_read_probe, 32 MB L2-resident buffer read 50 times",
                   "csr_bytes": csr_bytes, "l2_bytes": l2_size,
                   "sector_bytes_per_launch": avg_s, "achieved_sector_granular": sec, "frac_sector_granular": sec / l2}

    if rank == 0:
        r0 = results[0]
        line = {
            "metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
            "config": workload_config(g, {
                "parallelism": "replicas" if world > 1 else "single",
                "time_to_lambda_delta_ms": [round(1e3 * t, 3) for t in times],
                "tau": [int(r.tau) for r in results], "alpha": int(r0.alpha), "omega": r0.omega,
                **({"k": w["k"], "topk_first_step": [int(x) for x in r0.topk]} if w.get("k") else {}),
                "checks": [int(r.checks) for r in results],
                **step_spread(times, results),
                "edges_per_s": edges / total if world == 1 else None,
                "edges_per_sample": float(tot_np[0]) / K,
            }),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": w["sampler_dram_bytes"], "kernel": "k_sample (sampler batch)",
                         "bytes_per_launch": avg_b, "launch_ms": 1e3 * avg_t, "samples_per_launch": K,
                         "peak_source": peak_src, "bytes_basis": BYTES_BASIS},
            "e2e": {"value": e2e_value, "unit": "paths/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
        }
        if clk:
            line["clocks"] = clk
        if cpu:
            line["cpu_baseline"] = cpu
        if cpu_multi:
            line["cpu_baseline_multicore"] = cpu_multi
        if roof_l2:
            line["roofline_l2"] = roof_l2
        line.update(extras)
        print(json.dumps(line), flush=True)
    G.free()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
