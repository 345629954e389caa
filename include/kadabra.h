/*
 * kadabra.h -- C ABI of the GB300 (sm_103a) implementation of KADABRA's
 * adaptive sampling loop (Borassi & Natale, "KADABRA is an ADaptive
 * Algorithm for Betweenness via Random Approximation").
 *
 * The library estimates the normalised betweenness centrality
 *     bc(v) = 1/(n(n-1)) * sum_{s != v != t} sigma_st(v) / sigma_st    (Sec. 2)
 * of every node of an unweighted graph by sampling shortest paths with a
 * balanced bidirectional BFS (Sec. 4) and stopping adaptively once every
 * node's confidence interval is within lambda (Alg. 1, Thm. 1 and 2).
 *
 * Conventions
 *   - Every call returns a kadabra_status; nothing throws across the ABI.
 *   - Graph arrays are int32 CSR: row_ptr has n+1 entries starting at 0,
 *     col has m = row_ptr[n] entries, every row strictly increasing, no
 *     self-loops, all ids in [0, n).  n >= 2, m < 2^31, n <= 2^24.
 *   - Undirected graphs store both arcs of every edge; directed graphs also
 *     pass the reverse CSR (in-arcs) that the backward search reads.
 *   - Pointers named d_* are CUDA device pointers; all others are host
 *     pointers.  The caller owns every buffer it passes; the library owns
 *     the kadabra_graph object and the device memory it allocates.
 *   - `stream` arguments are cudaStream_t values passed as void* (NULL =
 *     the legacy default stream).  Calls are synchronous with respect to the
 *     host unless stated otherwise.
 *   - Randomness: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter
 *     = (sample index lo, hi, draw, domain); domain 0 = main loop,
 *     1 = warm-up, 2 = top-k preliminary estimate, 3 = the sampler
 *     autotuner's probe batches (nothing recorded).  Results depend only on
 *     (graph, parameters, seed).
 */
#ifndef KADABRA_H
#define KADABRA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KADABRA_OK = 0,
  KADABRA_ERR_ARG = 1,            /* invalid argument (NULL, range, lambda/delta)   */
  KADABRA_ERR_CSR = 2,            /* malformed CSR (offsets, ids, order, loops)     */
  KADABRA_ERR_OOM = 3,            /* device allocation failed                       */
  KADABRA_ERR_SIGMA_OVERFLOW = 4, /* a shortest-path count exceeded 2^64-1          */
  KADABRA_ERR_CAPACITY = 5,       /* an internal bound was exceeded (see message)   */
  KADABRA_ERR_TIMEOUT = 6,        /* reserved: no kernel of this library waits on a
                                     flag or another CTA, so no call returns it     */
  KADABRA_ERR_CUDA = 7,           /* a CUDA runtime call failed                     */
  KADABRA_ERR_UNSUPPORTED = 8,    /* reserved (every mode of the ABI is implemented) */
  KADABRA_ERR_INTERNAL = 9        /* an invariant of the method failed (a bug)      */
} kadabra_status;

/* Per-sample work counters, summed in kadabra_result.totals and returned
 * per sample by kadabra_sample_paths.  Only levels that did not touch the
 * other search contribute NEW and SIGMA_ADDS (a touching level ends the
 * BFS, Sec. 4). */
enum {
  KADABRA_STAT_EDGES = 0,      /* arcs scanned while expanding levels          */
  KADABRA_STAT_EXPANDED = 1,   /* frontier nodes expanded                       */
  KADABRA_STAT_NEW = 2,        /* nodes added by non-touching levels            */
  KADABRA_STAT_SIGMA_ADDS = 3, /* repeat discoveries in those levels            */
  KADABRA_STAT_PI = 4,         /* candidate (touch) edges                       */
  KADABRA_STAT_LEVELS = 5,     /* levels expanded                               */
  KADABRA_STAT_BT_SCANNED = 6, /* adjacency positions up to each backtrack pick */
  KADABRA_STAT_PATH_NODES = 7, /* nodes on the sampled path incl. s and t       */
  KADABRA_STAT_SIGMA_LO = 8,   /* sigma_st low 32 bits (per sample only)        */
  KADABRA_STAT_SIGMA_HI = 9,   /* sigma_st high 32 bits (per sample only)       */
  KADABRA_STAT_DIST = 10,      /* d(s,t) in arcs, -1 if disconnected            */
  KADABRA_NSTAT = 11
};

/* Opaque device-resident graph plus its cached sampler workspace. */
typedef struct kadabra_graph kadabra_graph;

/* Optional knobs (kadabra_config_default fills the defaults). */
typedef struct {
  int64_t vd;              /* vertex-diameter bound VD for omega; 0 = the library's
                              bound, computed at load: the heaviest path of the
                              condensation into strongly connected components,
                              each weighing its node count, except the component
                              of r (lowest-id node of maximum undirected degree):
                              e_in + e_out + 1, its largest distances to and from
                              r (2*ecc(r)+1 for a connected undirected graph)     */
  double eps;              /* computeDelta epsilon (App. D; default 0.001)        */
  uint64_t check_interval; /* K: samples between stop tests (default 1000; 0 = chosen
                              by the library from omega: max(1024, ceil(omega/32)))  */
  void* stream;            /* cudaStream_t for all work of the call (NULL = default) */
  int32_t ctas_per_sm;     /* shared-memory sampler tier, as resident CTAs per SM: 0 =
                              autotuned per graph (on the first one-graph run a probe
                              batch of min(K, 65536) samples times every allowed setup
                              of table and warp tier; the choice is cached per graph
                              fingerprint), or one of the two values the library
                              offers (4: 4096-slot tables, lists of 3072 nodes; 5:
                              the compact layout, lists of 2048 nodes; on GB300);
                              any other value is KADABRA_ERR_ARG.  Results do not
                              depend on it.  A batch run tunes it on its largest
                              graph; serving uses the default.                    */
  int32_t warp_tier;       /* one-warp-per-sample tier in front of tier S (samples whose
                              search outgrows its 512-slot table go on to tier S):
                              0 = autotuned together with ctas_per_sm, 1 = on,
                              -1 = off; any other value is KADABRA_ERR_ARG.
                              Results do not depend on it.                        */
  int32_t reserved[6];
} kadabra_config;

void kadabra_config_default(kadabra_config* cfg);

/* Result of kadabra_run.  The caller sets the output buffer pointers (any
 * may be NULL); the library fills the rest. */
typedef struct {
  /* outputs */
  uint64_t tau;        /* main-loop samples taken (Alg. 1 tau)                    */
  uint64_t omega_cap;  /* ceil(omega), the sample cap                             */
  uint64_t alpha;      /* warm-up samples, max(1, floor(omega/100)) (Alg. 2)      */
  uint64_t checks;     /* stop tests evaluated                                    */
  int64_t vd;          /* VD used                                                 */
  double omega;        /* 0.5/lambda^2 * (floor(log2(VD-2)) + 1 + ln(2/delta))    */
  double C;            /* computeDelta bisection constant                         */
  double max_f;        /* max_v f(v) at the final tau (Thm. 2)                    */
  double max_g;        /* max_v g(v) at the final tau                             */
  int64_t totals[KADABRA_NSTAT]; /* work counters, warm-up + main loop              */
  uint64_t check_interval; /* K used                                                */
  int32_t stopped_early; /* 1 if the stop test held before ceil(omega) samples    */
  int32_t status;        /* same as the call's return value                       */
  /* caller-owned buffers (inputs; NULL = not wanted) */
  uint32_t* counts;    /* host, n: main-loop hits per node (b~ * tau)             */
  double* btilde;      /* host, n: b~(v) = counts / tau                           */
  uint32_t* d_counts;  /* device, n                                               */
  double* d_btilde;    /* device, n                                               */
  int32_t* topk;       /* host, k: top-k mode's ranking (k > 0; may be NULL)      */
  /* serving (kadabra_submit / kadabra_poll): host monotonic clock, seconds   */
  double t_submit;     /* submitted                                                */
  double t_start;      /* admitted (device state allocated)                        */
  double t_done;       /* result ready                                             */
  int32_t ctas_per_sm; /* shared-memory sampler tier used (resident CTAs per SM)   */
  int32_t warp_tier;   /* 1 if the one-warp-per-sample tier ran first, else 0      */
} kadabra_result;

/* Copies a host CSR to the device and prepares the graph (Sec. 2 graph
 * G=(V,E); directed graphs need the reverse CSR, Sec. 4).  Validates the
 * CSR (KADABRA_ERR_CSR on any violation) and computes the default VD bound.
 * rrow_ptr/rcol must be NULL when directed == 0. */
kadabra_status kadabra_load_csr(int32_t n, int64_t m, const int32_t* row_ptr, const int32_t* col, int directed,
                                const int32_t* rrow_ptr, const int32_t* rcol, kadabra_graph** out);

/* Same, for a CSR already in device memory (e.g. torch tensors).  The
 * arrays are not copied and must outlive the graph object. */
kadabra_status kadabra_load_csr_device(int32_t n, int64_t m, const int32_t* d_row_ptr, const int32_t* d_col,
                                       int directed, const int32_t* d_rrow_ptr, const int32_t* d_rcol,
                                       kadabra_graph** out);

/* Releases the graph and the device memory the library allocated for it,
 * except its sampler workspace (tier tables, queues, scratch; up to about
 * 1.5 GB for large graphs).  The library keeps one such workspace per device
 * for the next graph object on that device whose node and arc counts fit in
 * it, which spares that object the allocation and initialisation.
 * kadabra_release_cached frees the kept workspaces.  The graph's own buffers
 * (its CSR copies, counters, load scratch) come from the device's default
 * stream-ordered memory pool, which this library sets to keep freed memory
 * (no release threshold): the next load reuses it without cudaMalloc.
 * Graph views of a batch (kadabra_batch_graph) are released with the batch;
 * passing one here does nothing. */
void kadabra_free_graph(kadabra_graph* g);

/* Frees the sampler workspaces kept by kadabra_free_graph (all devices) and
 * trims the current device's default memory pool to its memory in use.
 * Call it with no work of the library in flight. */
void kadabra_release_cached(void);

/* ---------------------------------------------------------------- batches
 * Several graphs sampled together (Alg. 1 for each graph, all graphs' sample
 * batches in one launch per round).  The CSRs of the G graphs are packed
 * into one device arena.  Each graph's result is identical to kadabra_run on
 * that graph with the same lambda, delta, seed and check interval. */
typedef struct kadabra_batch kadabra_batch;

#define KADABRA_MAX_BATCH_GRAPHS 65535

/* Copies G host CSRs (arrays of G pointers / sizes; rrow_ptr/rcol entries
 * NULL for undirected graphs, the arrays themselves may be NULL if no graph
 * is directed) into one device arena, validating each (KADABRA_ERR_CSR).
 * 1 <= G <= KADABRA_MAX_BATCH_GRAPHS, else KADABRA_ERR_ARG. */
kadabra_status kadabra_load_batch(int32_t G, const int32_t* n, const int64_t* m, const int32_t* const* row_ptr,
                                  const int32_t* const* col, const int* directed, const int32_t* const* rrow_ptr,
                                  const int32_t* const* rcol, kadabra_batch** out);

/* Releases the batch, its arena and its graph views. */
void kadabra_free_batch(kadabra_batch* b);

/* A graph object viewing graph i of the batch (for kadabra_run and the
 * other per-graph calls).  Owned by the batch.  Calls on the views of one
 * batch and on the batch itself share its workspace: do not overlap them. */
kadabra_status kadabra_batch_graph(kadabra_batch* b, int32_t i, kadabra_graph** view);

/* KADABRA on every graph of the batch (all-nodes mode), graph i with
 * lambda[i], delta[i], seed[i].  cfg (may be NULL) gives eps, the check
 * interval (0 = per graph from its omega, see kadabra_config), the sampler
 * setup (ctas_per_sm, warp_tier; autotuned on the batch's largest graph when
 * 0) and the stream; cfg->vd must be 0 (each graph uses its own VD bound).
 * out[i] receives graph i's result (set its buffer pointers as for
 * kadabra_run).  Rounds: one sampler launch over the next batch of every
 * unfinished graph, then one stop-test launch over all of them; after the
 * first round (sampled with the warm-up) the rounds run on the device as a
 * CUDA graph (a while loop), with one host wait for the rest of the run when
 * some graph allows more than four rounds.  Results do not depend on the
 * sampler setup or on where the rounds run.  Blocking. */
kadabra_status kadabra_run_batch(kadabra_batch* b, const double* lambda, const double* delta, const uint64_t* seed,
                                 const kadabra_config* cfg, kadabra_result* out);

/* Measurement helper (no counterpart in the paper): reads a zeroed device
 * buffer of `bytes` bytes `reps` times in one launch with loads cached in L2
 * only, after one warming pass, and returns the read rate in GB/s.  With a
 * buffer that fits in L2 this is the denominator of the sampler's L2
 * roofline.  Allocates and frees the buffer; synchronous on the current
 * device.  KADABRA_ERR_ARG for bytes < 16 or reps < 1. */
kadabra_status kadabra_l2_read_probe(uint64_t bytes, int32_t reps, double* gbs);

/* ---------------------------------------------------------------- serving
 * Continuous batching of KADABRA runs (either mode of kadabra_run) on the
 * graph's device.  A worker thread admits submitted jobs in arrival order
 * while their device state (hit counters, computeDelta tables, scratch:
 * about 12 bytes per node, 40 in top-k mode) fits the memory budget and a
 * slot is free; each round samples the next batch of every admitted job in
 * one sampler launch (a new job's warm-up, or its next K main-loop
 * samples), then runs computeDelta for jobs whose warm-up is done and the
 * stop tests of the others.  A job's result is identical to kadabra_run
 * with the same arguments, whatever runs beside it.  The graph must stay
 * loaded until its jobs are collected. */

/* Sets the memory budget (bytes of job state on the device; 0 = a quarter
 * of the free memory when the server starts) and the most jobs admitted at
 * once.  Only before the first submit (KADABRA_ERR_ARG after). */
kadabra_status kadabra_serve_configure(uint64_t budget_bytes, int32_t max_active);

/* Queues one run of KADABRA on g (arguments as kadabra_run; cfg->stream,
 * cfg->ctas_per_sm and cfg->warp_tier are ignored: the server has its own
 * stream and shares launches between jobs).  Returns at once with a job id
 * in *job.  Argument errors are returned here, including a batch's graph
 * view (not accepted).  g must stay loaded until the job is collected by
 * kadabra_poll or dropped by kadabra_serve_shutdown. */
kadabra_status kadabra_submit(kadabra_graph* g, double lambda, double delta, int32_t k, uint64_t seed,
                              const kadabra_config* cfg, uint64_t* job);

/* *done = 1 and the result in *out (same fields and caller-owned buffers as
 * kadabra_run; t_submit, t_start, t_done set) once the job has finished, or
 * *done = 0 at once if it has not and wait == 0; wait != 0 blocks until it
 * has.  A finished job is collected by this call: its id is then unknown
 * (KADABRA_ERR_ARG).  Returns the job's own status when done. */
kadabra_status kadabra_poll(uint64_t job, int32_t wait, int32_t* done, kadabra_result* out);

/* Finishes every admitted and queued job, stops the worker threads and
 * frees their device memory; results not yet collected are dropped. */
void kadabra_serve_shutdown(void);

kadabra_status kadabra_graph_info(const kadabra_graph* g, int32_t* n, int64_t* m, int* directed, int64_t* vd);

/* Graph flags.  A sample's visited set lives in a small shared-memory table
 * while it fits, then in a large shared-memory table, then in medium
 * per-CTA global tables, then in n-sized global tables (each sample goes as
 * far as it needs; results are identical in every tier).  The flags make
 * every sample start further down that list: KADABRA_FLAG_LARGE_SHARED_TABLES
 * at the large shared-memory table, KADABRA_FLAG_MEDIUM_TABLES at the medium
 * global tables, KADABRA_FLAG_GLOBAL_TABLES at the n-sized tables.  They
 * exist to test those paths and for graphs whose searches are known to be
 * deep or wide.  KADABRA_FLAG_WARP_TIER makes every sample start one step
 * earlier, at the one-warp-per-sample table (512 slots, 256 visited nodes,
 * 128 candidate edges), in every entry point that takes the graph object;
 * a batch or serving launch shared by several graphs runs that tier first if
 * any of them has the flag (and ignores their other flags).  It has no effect
 * together with one of the three flags above.  KADABRA_FLAG_ASYNC_SCAN makes
 * the level scans of the 4096-slot shared-memory table read every stretch of
 * at least 131 arcs inside one row with 16-byte loads (128 arcs per warp
 * load).  The library does this by itself for graphs whose CSR (forward plus
 * reverse) exceeds the device's L2, where each load waits on HBM; the flag
 * asks for it on any graph, and a shared launch takes it from any of its
 * graphs.
 * KADABRA_FLAG_FRONTIER_SEGMENTS makes the shared-memory tables scan every
 * frontier in segments of 64 nodes, as they do for frontiers beyond their
 * frontier array (1024 nodes, 512 in the compact tier-S layout), and
 * to take at most two searched long rows per segment; it exists to test
 * those paths and only slows sampling.  KADABRA_FLAG_COMPACT_TABLES runs tier
 * S in the compact layout (the autotuner's 5-CTA setup: lists of 2048 nodes,
 * 38 levels per side) whatever the tuned setup, except with the 16-byte
 * scans, which have no compact variant.  No flag changes a result.  Returns
 * KADABRA_ERR_ARG for unknown bits. */
enum {
  KADABRA_FLAG_GLOBAL_TABLES = 1,
  KADABRA_FLAG_MEDIUM_TABLES = 2,
  KADABRA_FLAG_LARGE_SHARED_TABLES = 4,
  KADABRA_FLAG_WARP_TIER = 8,
  KADABRA_FLAG_ASYNC_SCAN = 16,
  KADABRA_FLAG_FRONTIER_SEGMENTS = 32,
  KADABRA_FLAG_COMPACT_TABLES = 64
};
kadabra_status kadabra_graph_set_flags(kadabra_graph* g, uint32_t flags);

/* KADABRA (Alg. 1): warm-up, computeDelta (Alg. 2), then sample batches
 * of K with a stop test after each, until the test holds or ceil(omega)
 * samples.  lambda in (0,1), delta in (0,1); cfg may be NULL.  Blocking.
 *   k = 0: all-nodes mode, the rule f,g <= lambda for every node (Sec. 2).
 *     When ceil(omega) allows more than 4 rounds of K samples, the main loop
 *     runs on the device as a CUDA graph (a while node over {next batch,
 *     stop test}) and the host waits once for it; otherwise the host runs
 *     the rounds.  Results are the same either way.
 *   1 <= k <= 256: the k most central nodes (Sec. 5): a preliminary
 *     estimate of alpha samples (RNG domain 2) sets per-node targets
 *     lambda_L(v), lambda_U(v); Alg. 2 runs with those targets; the stop
 *     test is Alg. 3.  Nodes are ranked by b~ decreasing, ties by id;
 *     out->topk (caller-owned, k entries) receives the min(k, n) first
 *     nodes of the final ranking.  Other k: KADABRA_ERR_ARG. */
kadabra_status kadabra_run(kadabra_graph* g, double lambda, double delta, int32_t k, uint64_t seed,
                           const kadabra_config* cfg, kadabra_result* out);

/* One batch of the sampler (Sec. 4 plus Alg. 1 hit update): samples indices
 * [first_idx, first_idx+count) of `domain`, adding each path's interior
 * hits into d_counts (device, n) and the work counters into d_totals
 * (device, KADABRA_NSTAT int64, may be NULL).  Asynchronous on `stream`;
 * errors found on the device (sigma overflow, capacity) are reported by the
 * next kadabra_sync_status.  It takes the sampler setup that an autotuned
 * kadabra_run on the same graph object chose for batches of this size (the
 * default setup if none has); results do not depend on it. */
kadabra_status kadabra_sample_batch(kadabra_graph* g, uint64_t seed, uint32_t domain, uint64_t first_idx,
                                    uint64_t count, uint32_t* d_counts, int64_t* d_totals, void* stream);

/* The sampler batch without any device allocation.  It has no counterpart in
 * the paper.  It exists for callers that cannot allocate device memory: code
 * whose device memory belongs entirely to another allocator (a framework's
 * memory pool), and latency-critical code that must not call cudaMalloc or
 * cudaFree after start-up (both can synchronize the whole device).
 *
 * Same sampling as kadabra_sample_batch (identical hit counts and work
 * counters), from a CSR the caller already holds on the device (the arrays
 * of kadabra_load_csr_device, assumed valid: this call does not check them).
 * The library's scratch for this call is one file-scope device array of
 * 63.5 MiB (candidate-edge buffers for up to 304 CTAs, 2 per SM on a 152-SM
 * GPU, 512 edges per warp; 32 medium hash tables in global memory; two
 * queues of 65536 entries), which every GPU that loads the library holds
 * until the process exits.  Limits:
 *   - count <= 65536 samples per call (larger counts: KADABRA_ERR_CAPACITY);
 *   - the shared-memory tiers and one global-memory tier are used (no
 *     n-sized tables): if any sample outgrows them (more than 16384 nodes
 *     before the touching level, more than 1022 levels per side, or more
 *     than 512 candidate edges found by one warp), the call returns
 *     KADABRA_ERR_CAPACITY and its counts are incomplete.
 * The first call on a device sets that device up (kernel attributes and the
 * scratch array's device address); make that first call before any stream
 * capture.  Every call shares the one scratch array, which keeps the last
 * call's contents (the call clears what must start at zero), so calls that
 * overlap on the GPU, from any stream or thread, race: serialise them.
 * Blocking: waits for `stream` before returning. */
kadabra_status kadabra_sample_batch_noalloc(int32_t n, int64_t m, const int32_t* d_row_ptr, const int32_t* d_col,
                                            int directed, const int32_t* d_rrow_ptr, const int32_t* d_rcol,
                                            uint64_t seed, uint32_t domain, uint64_t first_idx, uint64_t count,
                                            uint32_t* d_counts, int64_t* d_totals, void* stream);

/* Waits for `stream` and returns (then clears) the device error word of g. */
kadabra_status kadabra_sync_status(kadabra_graph* g, void* stream);

/* Test hook: samples [first_idx, first_idx+count) of `domain` and returns,
 * per sample, (s,t) in st_out (host, 2*count), the path s..t in paths (host,
 * count*max_len, -1 padded; may be NULL), its node count in path_len (host,
 * count), the work counters in stats (host, count*KADABRA_NSTAT, may be
 * NULL) and a per-sample status (host, count). */
kadabra_status kadabra_sample_paths(kadabra_graph* g, uint64_t seed, uint32_t domain, uint64_t first_idx,
                                    uint32_t count, int32_t* st_out, int32_t* path_len, int32_t* paths,
                                    int32_t max_len, int64_t* stats, int32_t* status);

/* Test hook: the device Philox4x32-10 block for counters
 * (idx, idx_hi, j, domain), idx in [first_idx, first_idx+count), written
 * to out (host, 4*count uint32). */
kadabra_status kadabra_philox(uint64_t seed, uint32_t domain, uint32_t j, uint64_t first_idx, uint32_t count,
                              uint32_t* out);

/* Stop test of the all-nodes mode on the device (Thm. 2 f and g in FP64,
 * rule f <= lambda and g <= lambda for all v).  Host inputs counts (n),
 * ln_inv_dl/ln_inv_du (n, ln(1/delta_L(v)), ln(1/delta_U(v))); outputs the
 * maxima of f and g and the decision. */
kadabra_status kadabra_check(int64_t n, const uint32_t* counts, uint64_t tau, double omega,
                             const double* ln_inv_dl, const double* ln_inv_du, double lambda, double* max_f,
                             double* max_g, int* stop);

/* computeDelta (Alg. 2, App. D) with lambda_L = lambda_U = lambda: from the
 * warm-up hits count0 (host, n) of alpha samples, finds C by bisection and
 * writes ln(1/delta_L(v)) and ln(1/delta_U(v)) (host, n each). */
kadabra_status kadabra_compute_delta(int64_t n, const uint32_t* count0, uint64_t alpha, double omega,
                                     double lambda, double delta, double eps, double* ln_inv_dl,
                                     double* ln_inv_du, double* C);

/* omega of Alg. 1 for the given VD (c = 0.5, natural log). */
double kadabra_omega(double lambda, double delta, int64_t vd);

/* Human-readable text of the last error raised in this thread. */
const char* kadabra_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KADABRA_H */
