// KADABRA oracle: plain, single-threaded CPU restatement of the method.
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg load this library.  It shares no code, header
// or constant generator with the CUDA path; the two are written separately
// from the same reading of the paper (Borassi & Natale, "KADABRA is an
// ADaptive Algorithm for Betweenness via Random Approximation").
//
// What each function follows:
//   philox4x32_10      Salmon et al., SC'11 "Parallel Random Numbers: As Easy
//                      as 1, 2, 3" (the paper is silent on its RNG).
//   sample_one         Sec. 4 (balanced bidirectional BFS), the candidate-edge
//                      choice proportional to sigma_sv*sigma_wt and the
//                      backtracking to a uniform shortest path; Sec. 2 for the
//                      hit variables X_i(v) (1 iff v on the path, v != s,t).
//   omega_of           Alg. 1 first line and Sec. 2: omega = c/lambda^2 *
//                      (floor(log2(VD-2)) + 1 + ln(2/delta)), c = 0.5.
//   vd_bound           the upper bound on VD that omega needs (Alg. 1,
//                      Sec. 2); the paper does not say how it is obtained.
//   compute_delta      Alg. 2 and App. D (warm-up of omega/100 samples,
//                      c_L, c_U, bisection for C, delta_L, delta_U).
//   check_stop         Thm. 2 (functions f and g) and the all-nodes stopping
//                      rule f <= lambda and g <= lambda for every node (Sec. 2).
//   topk_lambdas       Sec. 5: lambda_L(v), lambda_U(v) from a preliminary
//                      estimate, for the top-k stopping condition.
//   check_stop_topk    Alg. 3 (haveToStop for the k most central nodes).
//   run                Alg. 1 with the stop test evaluated every K samples;
//                      all-nodes mode, or top-k mode (Sec. 5, Alg. 3).
//   brandes            exact normalised betweenness (Sec. 2 definition), by
//                      Brandes' dependency accumulation; used only by tests.
//   enumerate_paths    brute-force list of all shortest s-t paths; tests only.
//
// Readings where the paper is silent (each also listed in the design notes):
//   * RNG: Philox4x32-10, key = (seed_lo, seed_hi), counter = (idx_lo, idx_hi,
//     draw j, domain); domain 0 = main loop, 1 = warm-up.  Each decision takes
//     one whole 128-bit block: j=0 (s,t), j=1 candidate edge, j=2.. one per
//     backtracking step, s side first, then t side.
//   * (s,t): s = floor(u*n/2^64), t' = floor(u'*(n-1)/2^64), t = t' + (t'>=s),
//     with u = w0|w1<<32, u' = w2|w3<<32: a uniform ordered pair with s != t.
//   * bb-BFS: the side whose frontier degree sum is <= the other's expands
//     (ties go to s); a level is always processed completely; touch edges are
//     recorded as (v on the s side, w on the t side).
//   * The frontier being expanded is processed in increasing node id, each
//     row in sorted order; candidate edges are ordered as found, i.e. by
//     (x, y) with x the node on the expanding side.  A weighted choice with
//     total S takes r = floor(U128 * S / 2^128) and picks the first entry
//     whose inclusive prefix sum exceeds r.  Backtracking uses the same rule
//     over the predecessors of x in sorted adjacency order, weighted by sigma.
//   * Only a level that does not touch the other search is kept: a touching
//     level ends the BFS after all its arcs are scanned (Sec. 4), and the
//     nodes it discovered on its own side play no further part.
//   * sigma is an exact uint64; any overflow, or sigma_st > 2^64-1, fails the
//     sample with status SIGMA_OVERFLOW.
//   * VD when not given: a bound from the condensation into strongly
//     connected components (vd_bound), r the lowest-id node of maximum
//     degree in the underlying undirected graph; 2*ecc(r)+1 for a connected
//     undirected graph.
//   * alpha = max(1, floor(omega/100)); eps = configurable (paper: 0.001 in
//     App. D text, 0.0001 in Alg. 2).
//   * The bisection for C keeps the upper end so sum(delta) <= delta/2 and
//     stops at the FP64 fixed point; terms with c(v) = 0 are 0.
//   * Top-k mode: the preliminary estimate of Sec. 5 takes alpha samples in
//     RNG domain 2.  Nodes are ranked by b~ decreasing, ties by id
//     increasing.  Undefined neighbours of the ranking: lambda_U(v_1) = 1
//     (no node lies above v_1, and betweenness is at most 1) and
//     lambda_L(v_n) = 1; in Alg. 3, b~(v_0) - f = +inf and
//     b~(v_{n+1}) + g = -inf.  k > n is taken as k = n.  The Sec. 5 rules
//     apply in the order the text gives them (top-k nodes, the others, then
//     small gaps); a gap b~(v_i) - b~(v_{i+1}) < 2 lambda (i <= k) is
//     "small"; finally every lambda_L, lambda_U below lambda is raised to
//     lambda (the rule for the other nodes can give values <= 0).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <vector>

typedef unsigned __int128 u128;

namespace {

// ---------------------------------------------------------------- status
enum {
  ORC_OK = 0,
  ORC_ERR_ARG = 1,
  ORC_ERR_SIGMA_OVERFLOW = 4,
  ORC_ERR_CAPACITY = 5,
  ORC_ERR_INTERNAL = 99,  // an invariant of the method failed (a bug)
};

// ---------------------------------------------------------------- graph
struct Graph {
  int64_t n;
  const int32_t* rp;   // out-arc offsets
  const int32_t* ci;   // out-arc targets
  const int32_t* rrp;  // in-arc offsets (== rp for undirected)
  const int32_t* rci;  // in-arc sources (== ci for undirected)
};

Graph make_graph(int64_t n, const int32_t* rp, const int32_t* ci, int directed, const int32_t* rrp,
                 const int32_t* rci) {
  Graph g;
  g.n = n;
  g.rp = rp;
  g.ci = ci;
  if (directed) {
    g.rrp = rrp;
    g.rci = rci;
  } else {
    g.rrp = rp;
    g.rci = ci;
  }
  return g;
}

int64_t out_deg(const Graph& g, int32_t v) { return g.rp[v + 1] - g.rp[v]; }
int64_t in_deg(const Graph& g, int32_t v) { return g.rrp[v + 1] - g.rrp[v]; }

// ---------------------------------------------------------------- Philox
// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).  One round:
// two 32x32->64 multiplications of counter words 0 and 2, the high halves
// xor-ed with the other counter words and the round key; the key is bumped
// by the two Weyl constants between rounds.
void philox4x32_10(uint32_t key0, uint32_t key1, const uint32_t ctr[4], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key0, k1 = key1;
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * x0;
    uint64_t p1 = (uint64_t)M1 * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

struct Block {
  uint32_t w[4];
};

Block draw_block(uint64_t seed, uint32_t domain, uint64_t idx, uint32_t j) {
  uint32_t ctr[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), j, domain};
  Block b;
  philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), ctr, b.w);
  return b;
}

// floor(u * n / 2^64)
uint64_t scale64(uint64_t u, uint64_t n) { return (uint64_t)(((u128)u * n) >> 64); }

// floor(U * S / 2^128), U = the block as a 128-bit integer (w0 least significant)
uint64_t scale128(const Block& b, uint64_t S) {
  uint64_t lo = (uint64_t)b.w[0] | ((uint64_t)b.w[1] << 32);
  uint64_t hi = (uint64_t)b.w[2] | ((uint64_t)b.w[3] << 32);
  u128 low_part = ((u128)lo * S) >> 64;   // floor(lo*S / 2^64)
  u128 high_part = (u128)hi * S;          // hi*S, weight 2^64
  return (uint64_t)((high_part + low_part) >> 64);
}

// ---------------------------------------------------------------- sampler
// Per-sample work counters (the paper reports edges visited per sample).
enum {
  ST_EDGES = 0,      // arcs scanned while expanding levels
  ST_EXPANDED,       // frontier nodes expanded
  ST_NEW,            // nodes added by levels that did not touch
  ST_SIGMA_ADDS,     // repeat discoveries (sigma additions) in those levels
  ST_PI,             // candidate (touch) edges
  ST_LEVELS,         // levels expanded
  ST_BT_SCANNED,     // adjacency entries read while backtracking
  ST_PATH_NODES,     // nodes on the path including s and t (0 if none)
  ST_SIGMA_LO,       // sigma_st, low 32 bits (0 if disconnected)
  ST_SIGMA_HI,       // sigma_st, high 32 bits
  ST_DIST,           // d(s,t) in arcs, or -1
  ST_COUNT
};

struct Work {
  std::vector<int32_t> dist_s, dist_t;
  std::vector<uint64_t> sig_s, sig_t;
  std::vector<int32_t> touched;
  explicit Work(int64_t n) : dist_s(n, -1), dist_t(n, -1), sig_s(n, 0), sig_t(n, 0) {}
  void reset() {
    for (int32_t v : touched) {
      dist_s[v] = -1;
      dist_t[v] = -1;
      sig_s[v] = 0;
      sig_t[v] = 0;
    }
    touched.clear();
  }
};

struct Sample {
  int32_t s = -1, t = -1;
  int status = ORC_OK;
  std::vector<int32_t> path;  // s ... t, empty when s and t are not connected
  int64_t st[ST_COUNT] = {0};
};

struct PiEdge {
  int32_t v, w;
};

// One sample for a given ordered pair (s,t); block 0 has already been used
// to draw (s,t) (or (s,t) was fixed by the caller), so this starts at j=1.
void sample_pair(const Graph& g, uint64_t seed, uint32_t domain, uint64_t idx, int32_t s, int32_t t,
                 Work& wk, Sample& out) {
  out.s = s;
  out.t = t;
  out.status = ORC_OK;
  out.path.clear();
  std::memset(out.st, 0, sizeof(out.st));
  out.st[ST_DIST] = -1;

  std::vector<int32_t>& dist_s = wk.dist_s;
  std::vector<int32_t>& dist_t = wk.dist_t;
  std::vector<uint64_t>& sig_s = wk.sig_s;
  std::vector<uint64_t>& sig_t = wk.sig_t;

  dist_s[s] = 0;
  sig_s[s] = 1;
  dist_t[t] = 0;
  sig_t[t] = 1;
  wk.touched.push_back(s);
  wk.touched.push_back(t);

  std::vector<int32_t> front_s(1, s), front_t(1, t), next;
  int64_t cost_s = out_deg(g, s);  // sum of degrees of the current s frontier
  int64_t cost_t = in_deg(g, t);
  std::vector<PiEdge> pi;  // in discovery order, which is the canonical order
  bool overflow = false;

  for (;;) {
    next.clear();
    int64_t level_new = 0, level_adds = 0;
    bool level_overflow = false;
    out.st[ST_LEVELS]++;
    const bool expand_s = cost_s <= cost_t;
    std::vector<int32_t>& front = expand_s ? front_s : front_t;
    // frontier nodes are processed in increasing id order, each row in its
    // sorted order: candidate edges are then found in (x, y) order, x on the
    // expanding side
    std::sort(front.begin(), front.end());
    for (int32_t x : front) {
      out.st[ST_EXPANDED]++;
      if (expand_s) {
        // s side: out-arcs x -> y
        for (int32_t e = g.rp[x]; e < g.rp[x + 1]; ++e) {
          int32_t y = g.ci[e];
          out.st[ST_EDGES]++;
          if (dist_t[y] >= 0) {
            pi.push_back({x, y});
          } else if (dist_s[y] < 0) {
            dist_s[y] = dist_s[x] + 1;
            sig_s[y] = sig_s[x];
            next.push_back(y);
            wk.touched.push_back(y);
            level_new++;
          } else if (dist_s[y] == dist_s[x] + 1) {
            uint64_t before = sig_s[y];
            sig_s[y] = before + sig_s[x];
            if (sig_s[y] < before) level_overflow = true;
            level_adds++;
          }
        }
      } else {
        // t side: in-arcs y -> x; a touch edge is stored as (y on the s side, x)
        for (int32_t e = g.rrp[x]; e < g.rrp[x + 1]; ++e) {
          int32_t y = g.rci[e];
          out.st[ST_EDGES]++;
          if (dist_s[y] >= 0) {
            pi.push_back({y, x});
          } else if (dist_t[y] < 0) {
            dist_t[y] = dist_t[x] + 1;
            sig_t[y] = sig_t[x];
            next.push_back(y);
            wk.touched.push_back(y);
            level_new++;
          } else if (dist_t[y] == dist_t[x] + 1) {
            uint64_t before = sig_t[y];
            sig_t[y] = before + sig_t[x];
            if (sig_t[y] < before) level_overflow = true;
            level_adds++;
          }
        }
      }
    }
    // a level that touches the other search ends the BFS; the nodes it
    // discovered on its own side are never used and are not counted
    if (!pi.empty() || next.empty()) break;
    if (level_overflow) {  // sigma of a node that the search goes on with
      overflow = true;
      break;
    }
    out.st[ST_NEW] += level_new;
    out.st[ST_SIGMA_ADDS] += level_adds;
    int64_t cost = 0;
    if (expand_s) {
      front_s.swap(next);
      for (int32_t v : front_s) cost += out_deg(g, v);
      cost_s = cost;
    } else {
      front_t.swap(next);
      for (int32_t v : front_t) cost += in_deg(g, v);
      cost_t = cost;
    }
  }

  if (overflow) {
    out.status = ORC_ERR_SIGMA_OVERFLOW;
    wk.reset();
    return;
  }
  out.st[ST_PI] = (int64_t)pi.size();
  if (pi.empty()) {  // s and t are not connected: the sample hits nothing
    wk.reset();
    return;
  }

  // every candidate edge joins the two frontiers: d(s,v) + 1 + d(w,t) is the
  // same for all of them (the touch happens between adjacent levels)
  for (const PiEdge& p : pi)
    if (dist_s[p.v] + dist_t[p.w] != dist_s[pi[0].v] + dist_t[pi[0].w]) {
      out.status = ORC_ERR_INTERNAL;
      wk.reset();
      return;
    }

  // choose (v,w) with probability sigma_sv * sigma_wt / sigma_st
  u128 total = 0;
  for (const PiEdge& p : pi) total += (u128)sig_s[p.v] * sig_t[p.w];
  if (total > (u128)UINT64_MAX) {
    out.status = ORC_ERR_SIGMA_OVERFLOW;
    wk.reset();
    return;
  }
  const uint64_t sigma_st = (uint64_t)total;
  out.st[ST_SIGMA_LO] = (int64_t)(sigma_st & 0xffffffffu);
  out.st[ST_SIGMA_HI] = (int64_t)(sigma_st >> 32);
  uint32_t j = 1;
  uint64_t r = scale128(draw_block(seed, domain, idx, j++), sigma_st);
  uint64_t acc = 0;
  PiEdge chosen = pi.back();
  for (const PiEdge& p : pi) {
    acc += sig_s[p.v] * sig_t[p.w];
    if (acc > r) {
      chosen = p;
      break;
    }
  }
  out.st[ST_DIST] = dist_s[chosen.v] + 1 + dist_t[chosen.w];

  // backtrack v -> s over predecessors y (arc y->v) one level closer to s
  std::vector<int32_t> left;
  int32_t x = chosen.v;
  left.push_back(x);
  while (dist_s[x] > 0) {
    uint64_t rr = scale128(draw_block(seed, domain, idx, j++), sig_s[x]);
    uint64_t a = 0;
    int32_t pick = -1;
    for (int32_t e = g.rrp[x]; e < g.rrp[x + 1]; ++e) {
      int32_t y = g.rci[e];
      out.st[ST_BT_SCANNED]++;
      if (dist_s[y] == dist_s[x] - 1) {
        a += sig_s[y];
        if (a > rr) {
          pick = y;
          break;
        }
      }
    }
    if (pick < 0) {
      out.status = ORC_ERR_INTERNAL;
      wk.reset();
      return;
    }
    x = pick;
    left.push_back(x);
  }
  // backtrack w -> t over successors z (arc w->z) one level closer to t
  std::vector<int32_t> right;
  x = chosen.w;
  right.push_back(x);
  while (dist_t[x] > 0) {
    uint64_t rr = scale128(draw_block(seed, domain, idx, j++), sig_t[x]);
    uint64_t a = 0;
    int32_t pick = -1;
    for (int32_t e = g.rp[x]; e < g.rp[x + 1]; ++e) {
      int32_t z = g.ci[e];
      out.st[ST_BT_SCANNED]++;
      if (dist_t[z] == dist_t[x] - 1) {
        a += sig_t[z];
        if (a > rr) {
          pick = z;
          break;
        }
      }
    }
    if (pick < 0) {
      out.status = ORC_ERR_INTERNAL;
      wk.reset();
      return;
    }
    x = pick;
    right.push_back(x);
  }
  for (auto it = left.rbegin(); it != left.rend(); ++it) out.path.push_back(*it);
  for (int32_t y : right) out.path.push_back(y);
  out.st[ST_PATH_NODES] = (int64_t)out.path.size();
  wk.reset();
}

void sample_one(const Graph& g, uint64_t seed, uint32_t domain, uint64_t idx, Work& wk, Sample& out) {
  Block b0 = draw_block(seed, domain, idx, 0);
  uint64_t u = (uint64_t)b0.w[0] | ((uint64_t)b0.w[1] << 32);
  uint64_t u2 = (uint64_t)b0.w[2] | ((uint64_t)b0.w[3] << 32);
  int32_t s = (int32_t)scale64(u, (uint64_t)g.n);
  int32_t tp = (int32_t)scale64(u2, (uint64_t)(g.n - 1));
  int32_t t = tp + (tp >= s ? 1 : 0);
  sample_pair(g, seed, domain, idx, s, t, wk, out);
}

// ---------------------------------------------------------------- omega, VD
int64_t floor_log2_i64(int64_t x) {  // x >= 1
  int64_t k = 0;
  while (x >= 2) {
    x >>= 1;
    ++k;
  }
  return k;
}

double omega_of(double lambda, double delta, int64_t vd) {
  int64_t fl = (vd - 2 >= 1) ? floor_log2_i64(vd - 2) : 0;
  return (0.5 / (lambda * lambda)) * ((double)(fl + 1) + std::log(2.0 / delta));
}

// The root of the VD bound: the lowest-id node of maximum degree in the
// underlying undirected graph, |out(v) U in(v)| (rows are sorted).
int32_t vd_root(const Graph& g) {
  auto und_deg = [&](int32_t v) {
    int64_t a = g.rp[v], ae = g.rp[v + 1], b = g.rrp[v], be = g.rrp[v + 1];
    if (g.rp == g.rrp) return ae - a;
    int64_t d = 0;
    while (a < ae || b < be) {
      if (b >= be || (a < ae && g.ci[a] < g.rci[b])) {
        ++a;
      } else if (a >= ae || g.rci[b] < g.ci[a]) {
        ++b;
      } else {
        ++a;
        ++b;
      }
      ++d;
    }
    return d;
  };
  int32_t r = 0;
  int64_t best = -1;
  for (int32_t v = 0; v < g.n; ++v) {
    int64_t d = und_deg(v);
    if (d > best) {
      best = d;
      r = v;
    }
  }
  return r;
}

// Distances from r along the arcs of one CSR (out-arcs: from r; in-arcs: to r).
std::vector<int32_t> bfs_dist(int64_t n, const int32_t* rp, const int32_t* ci, int32_t r) {
  std::vector<int32_t> dist(n, -1), q;
  dist[r] = 0;
  q.push_back(r);
  for (size_t h = 0; h < q.size(); ++h) {
    int32_t v = q[h];
    for (int32_t e = rp[v]; e < rp[v + 1]; ++e)
      if (dist[ci[e]] < 0) {
        dist[ci[e]] = dist[v] + 1;
        q.push_back(ci[e]);
      }
  }
  return dist;
}

// Strongly connected components over the out-arcs (Tarjan, with an explicit
// stack).  comp[v] is the component's index; components come out in reverse
// topological order: an arc from component a to component b != a has b < a.
// For an undirected graph they are its connected components.
int64_t tarjan_scc(const Graph& g, std::vector<int64_t>& comp) {
  const int64_t n = g.n;
  std::vector<int64_t> index(n, -1), low(n, 0);
  std::vector<char> on_stack(n, 0);
  std::vector<int32_t> stack;
  std::vector<std::pair<int32_t, int32_t>> call;  // (node, next arc)
  comp.assign(n, -1);
  int64_t next_index = 0, ncomp = 0;
  for (int32_t root = 0; root < n; ++root) {
    if (index[root] >= 0) continue;
    call.push_back({root, g.rp[root]});
    index[root] = low[root] = next_index++;
    stack.push_back(root);
    on_stack[root] = 1;
    while (!call.empty()) {
      int32_t v = call.back().first;
      int32_t& e = call.back().second;
      if (e < g.rp[v + 1]) {
        int32_t w = g.ci[e++];
        if (index[w] < 0) {
          index[w] = low[w] = next_index++;
          stack.push_back(w);
          on_stack[w] = 1;
          call.push_back({w, g.rp[w]});
        } else if (on_stack[w]) {
          low[v] = std::min(low[v], index[w]);
        }
        continue;
      }
      call.pop_back();
      if (!call.empty()) {
        int32_t u = call.back().first;
        low[u] = std::min(low[u], low[v]);
      }
      if (low[v] == index[v]) {
        int32_t w;
        do {
          w = stack.back();
          stack.pop_back();
          on_stack[w] = 0;
          comp[w] = ncomp;
        } while (w != v);
        ++ncomp;
      }
    }
  }
  return ncomp;
}

// Upper bound on the vertex diameter VD (the most nodes on any shortest
// path), which omega needs (Alg. 1; Sec. 2).  The paper does not say how
// KADABRA bounds VD.  A shortest path visits the strongly connected
// components in the order of a path of the condensation, each one in a
// contiguous stretch that is a shortest path inside it.  A stretch inside a
// component C has at most |C| nodes; inside the component C_r of the root r
// it has at most d(u,r) + d(r,v) + 1 <= e_in + e_out + 1 nodes, with e_out
// and e_in the largest distances from and to r within C_r.  The bound is the
// largest sum of these weights along a path of the condensation.  For a
// connected undirected graph it is 2 ecc(r) + 1.
int64_t vd_bound(const Graph& g) {
  const int32_t r = vd_root(g);
  std::vector<int64_t> comp;
  const int64_t ncomp = tarjan_scc(g, comp);
  std::vector<int32_t> dout = bfs_dist(g.n, g.rp, g.ci, r);
  std::vector<int32_t> din = bfs_dist(g.n, g.rrp, g.rci, r);
  int64_t e_out = 0, e_in = 0;
  std::vector<int64_t> w(ncomp, 0);
  for (int32_t v = 0; v < g.n; ++v) {
    w[comp[v]] += 1;
    if (comp[v] == comp[r]) {
      e_out = std::max<int64_t>(e_out, dout[v]);
      e_in = std::max<int64_t>(e_in, din[v]);
    }
  }
  w[comp[r]] = e_out + e_in + 1;
  // longest weighted path of the condensation, starting at each component:
  // every component an arc leads to has a smaller index, so is done already
  std::vector<int64_t> from(ncomp, 0);
  std::vector<std::vector<int32_t>> members(ncomp);
  for (int32_t v = 0; v < g.n; ++v) members[comp[v]].push_back(v);
  int64_t best = 0;
  for (int64_t c = 0; c < ncomp; ++c) {
    int64_t tail = 0;
    for (int32_t v : members[c])
      for (int32_t e = g.rp[v]; e < g.rp[v + 1]; ++e)
        if (comp[g.ci[e]] != c) tail = std::max(tail, from[comp[g.ci[e]]]);
    from[c] = w[c] + tail;
    best = std::max(best, from[c]);
  }
  return best;
}

// ---------------------------------------------------------------- computeDelta
// Alg. 2 with per-node targets lambda_L(v), lambda_U(v).  Writes
// ln(1/delta_L(v)) and ln(1/delta_U(v)); returns C.
double compute_delta_lv(int64_t n, const uint32_t* count0, uint64_t alpha, double omega, const double* lamL,
                        const double* lamU, double delta, double eps, double* ln_inv_dl, double* ln_inv_du) {
  std::vector<double> cL(n), cU(n);
  bool any = false;
  for (int64_t v = 0; v < n; ++v) {
    double b0 = (double)count0[v] / (double)alpha;
    cL[v] = ((2.0 * b0) * omega) / (lamL[v] * lamL[v]);
    cU[v] = ((2.0 * b0) * omega) / (lamU[v] * lamU[v]);
    if (cL[v] > 0.0 || cU[v] > 0.0) any = true;
  }
  const double target = (delta / 2.0) - (eps * delta);
  auto sum_at = [&](double C) {
    double sum = 0.0;
    for (int64_t v = 0; v < n; ++v) {
      double eL = cL[v] > 0.0 ? std::exp(-C / cL[v]) : 0.0;
      double eU = cU[v] > 0.0 ? std::exp(-C / cU[v]) : 0.0;
      sum += eL + eU;
    }
    return sum;
  };
  double C = 0.0;
  if (any) {
    double lo = 0.0, hi = 1.0;
    while (!(sum_at(hi) <= target)) {
      lo = hi;
      hi = 2.0 * hi;
    }
    for (;;) {
      double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sum_at(mid) <= target)
        hi = mid;
      else
        lo = mid;
    }
    C = hi;
  }
  const double floor_term = (eps * delta) / (2.0 * (double)n);
  for (int64_t v = 0; v < n; ++v) {
    double dL = (cL[v] > 0.0 ? std::exp(-C / cL[v]) : 0.0) + floor_term;
    double dU = (cU[v] > 0.0 ? std::exp(-C / cU[v]) : 0.0) + floor_term;
    ln_inv_dl[v] = -std::log(dL);
    ln_inv_du[v] = -std::log(dU);
  }
  return C;
}

// Alg. 2 in all-nodes mode: lambda_L = lambda_U = lambda for every node.
double compute_delta(int64_t n, const uint32_t* count0, uint64_t alpha, double omega, double lambda,
                     double delta, double eps, double* ln_inv_dl, double* ln_inv_du) {
  std::vector<double> lam(n, lambda);
  return compute_delta_lv(n, count0, alpha, omega, lam.data(), lam.data(), delta, eps, ln_inv_dl, ln_inv_du);
}

// ---------------------------------------------------------------- top-k (Sec. 5)
// Nodes in decreasing order of b~ = count / denom, ties by increasing id.
std::vector<int64_t> rank_nodes(int64_t n, const uint32_t* count, double denom) {
  std::vector<int64_t> order(n);
  for (int64_t v = 0; v < n; ++v) order[v] = v;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    double ba = (double)count[a] / denom, bb = (double)count[b] / denom;
    if (ba != bb) return ba > bb;
    return a < b;
  });
  return order;
}

// Sec. 5: the error targets that separate the k most central nodes of a
// preliminary estimate (count_pre / alpha_pre) from one another and from the
// rest.  Writes lambda_L(v), lambda_U(v) for every node.
void topk_lambdas(int64_t n, const uint32_t* count_pre, uint64_t alpha_pre, int64_t k, double lambda, double* lamL,
                  double* lamU) {
  const double a = (double)alpha_pre;
  std::vector<int64_t> vv = rank_nodes(n, count_pre, a);  // v_1 .. v_n at vv[0 .. n-1]
  auto bt = [&](int64_t i) { return (double)count_pre[vv[i - 1]] / a; };  // b~(v_i), 1-based
  if (k > n) k = n;
  // the k first nodes: half the gaps to their neighbours in the ranking
  for (int64_t i = 1; i <= k; ++i) {
    const int64_t v = vv[i - 1];
    lamU[v] = i == 1 ? 1.0 : (bt(i - 1) - bt(i)) / 2.0;
    lamL[v] = i == n ? 1.0 : (bt(i) - bt(i + 1)) / 2.0;
  }
  // the other nodes: show that they lie below the k-th node's lower end
  for (int64_t i = k + 1; i <= n; ++i) {
    const int64_t v = vv[i - 1];
    lamL[v] = 1.0;
    lamU[v] = bt(k) - lamL[vv[k - 1]] - bt(i);
  }
  // small gaps: the order of the two nodes is not known, plain lambda for both
  for (int64_t i = 1; i <= k && i + 1 <= n; ++i) {
    if (bt(i) - bt(i + 1) < 2.0 * lambda) {
      lamL[vv[i - 1]] = lamU[vv[i - 1]] = lambda;
      lamL[vv[i]] = lamU[vv[i]] = lambda;
    }
  }
  for (int64_t v = 0; v < n; ++v) {
    if (!(lamL[v] >= lambda)) lamL[v] = lambda;
    if (!(lamU[v] >= lambda)) lamU[v] = lambda;
  }
}

// ---------------------------------------------------------------- stop test
// f and g of Thm. 2 for one node, evaluated with this exact expression tree.
void f_and_g(uint32_t count, uint64_t tau, double omega, double lnL, double lnU, double* f, double* g) {
  double t = (double)tau;
  double b = (double)count / t;
  double aL = (1.0 / 3.0) - omega / t;
  double aU = (1.0 / 3.0) + omega / t;
  *f = (lnL / t) * (aL + std::sqrt(aL * aL + ((2.0 * b) * omega) / lnL));
  *g = (lnU / t) * (aU + std::sqrt(aU * aU + ((2.0 * b) * omega) / lnU));
}

// all-nodes haveToStop: every node has f <= lambda and g <= lambda
int check_stop(int64_t n, const uint32_t* count, uint64_t tau, double omega, const double* lnL,
               const double* lnU, double lambda, double* max_f, double* max_g) {
  int stop = 1;
  double mf = 0.0, mg = 0.0;
  for (int64_t v = 0; v < n; ++v) {
    double f, g;
    f_and_g(count[v], tau, omega, lnL[v], lnU[v], &f, &g);
    if (!(f <= lambda) || !(g <= lambda)) stop = 0;
    if (f > mf) mf = f;
    if (g > mg) mg = g;
  }
  *max_f = mf;
  *max_g = mg;
  return stop;
}

// Alg. 3: haveToStop for the k most central nodes.  Ranks the nodes by the
// current b~ = count / tau; a node whose f or g exceeds lambda must have a
// confidence interval separated from its neighbours' in the ranking (the k
// first nodes) or from the k-th node's (the others).  Writes the k first
// nodes of the ranking to topk (if not NULL) and max f, max g over all nodes.
int check_stop_topk(int64_t n, const uint32_t* count, uint64_t tau, double omega, const double* lnL,
                    const double* lnU, double lambda, int64_t k, int32_t* topk, double* max_f, double* max_g) {
  if (k > n) k = n;
  std::vector<double> f(n), g(n), b(n);
  double mf = 0.0, mg = 0.0;
  const double t = (double)tau;
  for (int64_t v = 0; v < n; ++v) {
    f_and_g(count[v], tau, omega, lnL[v], lnU[v], &f[v], &g[v]);
    b[v] = (double)count[v] / t;
    if (f[v] > mf) mf = f[v];
    if (g[v] > mg) mg = g[v];
  }
  *max_f = mf;
  *max_g = mg;
  std::vector<int64_t> vv = rank_nodes(n, count, t);
  if (topk)
    for (int64_t i = 0; i < k; ++i) topk[i] = (int32_t)vv[i];
  auto loose = [&](int64_t v) { return f[v] > lambda || g[v] > lambda; };
  for (int64_t i = 1; i <= k; ++i) {
    const int64_t v = vv[i - 1];
    if (!loose(v)) continue;
    if (i > 1) {
      const int64_t u = vv[i - 2];
      if (b[u] - f[u] < b[v] + g[v]) return 0;
    }
    if (i < n) {
      const int64_t w = vv[i];
      if (b[v] - f[v] < b[w] + g[w]) return 0;
    }
  }
  const int64_t vk = vv[k - 1];
  for (int64_t i = k + 1; i <= n; ++i) {
    const int64_t v = vv[i - 1];
    if (!loose(v)) continue;
    if (b[vk] - f[vk] < b[v] + g[v]) return 0;
  }
  return 1;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

// Result of one oracle run (mirrors the library's result fields).
typedef struct {
  uint64_t tau;        // samples taken in the main loop
  uint64_t omega_cap;  // ceil(omega)
  uint64_t alpha;      // warm-up samples
  uint64_t checks;     // stop tests evaluated
  int64_t vd;          // vertex-diameter bound used
  double omega;
  double C;            // bisection constant of computeDelta
  double max_f, max_g; // at the final tau
  int64_t edges_warm;  // arcs scanned during the warm-up
  int64_t edges_main;  // arcs scanned during the main loop
  int32_t stopped_early;  // 1 if the stop test fired before ceil(omega)
  int32_t status;
} orc_result;

void orc_philox(uint64_t seed, uint32_t domain, uint64_t idx, uint32_t j, uint32_t out[4]) {
  Block b = draw_block(seed, domain, idx, j);
  std::memcpy(out, b.w, sizeof(b.w));
}

// Blocks for counters (idx, j, domain), idx in [first, first+count): out is 4*count.
void orc_philox_many(uint64_t seed, uint32_t domain, uint32_t j, uint64_t first, int64_t count, uint32_t* out) {
  for (int64_t i = 0; i < count; ++i) {
    Block b = draw_block(seed, domain, first + (uint64_t)i, j);
    std::memcpy(out + 4 * i, b.w, sizeof(b.w));
  }
}

// Raw Philox4x32-10 block for an arbitrary key and counter.
void orc_philox_raw(uint32_t k0, uint32_t k1, const uint32_t ctr[4], uint32_t out[4]) {
  philox4x32_10(k0, k1, ctr, out);
}

uint64_t orc_scale128(const uint32_t w[4], uint64_t S) {
  Block b;
  std::memcpy(b.w, w, sizeof(b.w));
  return scale128(b, S);
}

int orc_stat_count(void) { return ST_COUNT; }

// Samples indices [first_idx, first_idx+count) of one RNG domain.
// st_out: 2*count (s,t); path_len: count; paths: count*max_len (row-major,
// -1 padded); stats: count*ST_COUNT (may be NULL); status: count.
int orc_sample_paths(int64_t n, const int32_t* rp, const int32_t* ci, int directed, const int32_t* rrp,
                     const int32_t* rci, uint64_t seed, uint32_t domain, uint64_t first_idx, int64_t count,
                     int32_t* st_out, int32_t* path_len, int32_t* paths, int32_t max_len, int64_t* stats,
                     int32_t* status) {
  if (n < 2 || count < 0 || max_len < 0) return ORC_ERR_ARG;
  Graph g = make_graph(n, rp, ci, directed, rrp, rci);
  Work wk(n);
  Sample smp;
  int worst = ORC_OK;
  for (int64_t i = 0; i < count; ++i) {
    sample_one(g, seed, domain, first_idx + (uint64_t)i, wk, smp);
    st_out[2 * i] = smp.s;
    st_out[2 * i + 1] = smp.t;
    path_len[i] = (int32_t)smp.path.size();
    if (paths) {
      for (int32_t k = 0; k < max_len; ++k)
        paths[i * max_len + k] = k < (int32_t)smp.path.size() ? smp.path[k] : -1;
      if ((int32_t)smp.path.size() > max_len && worst == ORC_OK) worst = ORC_ERR_CAPACITY;
    }
    if (stats)
      for (int k = 0; k < ST_COUNT; ++k) stats[i * ST_COUNT + k] = smp.st[k];
    status[i] = smp.status;
    if (smp.status != ORC_OK) worst = smp.status;
  }
  return worst;
}

// Samples `count` paths for a fixed ordered pair (s,t), indices
// [first_idx, first_idx+count), domain `domain`; block 0 is unused.
int orc_sample_fixed_pair(int64_t n, const int32_t* rp, const int32_t* ci, int directed, const int32_t* rrp,
                          const int32_t* rci, int32_t s, int32_t t, uint64_t seed, uint32_t domain,
                          uint64_t first_idx, int64_t count, int32_t* path_len, int32_t* paths, int32_t max_len,
                          int64_t* stats) {
  if (n < 2 || s < 0 || t < 0 || s >= n || t >= n || s == t) return ORC_ERR_ARG;
  Graph g = make_graph(n, rp, ci, directed, rrp, rci);
  Work wk(n);
  Sample smp;
  int worst = ORC_OK;
  for (int64_t i = 0; i < count; ++i) {
    sample_pair(g, seed, domain, first_idx + (uint64_t)i, s, t, wk, smp);
    path_len[i] = (int32_t)smp.path.size();
    for (int32_t k = 0; k < max_len; ++k)
      paths[i * max_len + k] = k < (int32_t)smp.path.size() ? smp.path[k] : -1;
    if (stats)
      for (int k = 0; k < ST_COUNT; ++k) stats[i * ST_COUNT + k] = smp.st[k];
    if (smp.status != ORC_OK) worst = smp.status;
  }
  return worst;
}

// Adds the interior hits of samples [first_idx, first_idx+count) into
// counts[n]; totals[ST_COUNT] receives the summed work counters.
int orc_accumulate(int64_t n, const int32_t* rp, const int32_t* ci, int directed, const int32_t* rrp,
                   const int32_t* rci, uint64_t seed, uint32_t domain, uint64_t first_idx, int64_t count,
                   uint32_t* counts, int64_t* totals) {
  if (n < 2 || count < 0) return ORC_ERR_ARG;
  Graph g = make_graph(n, rp, ci, directed, rrp, rci);
  Work wk(n);
  Sample smp;
  for (int64_t i = 0; i < count; ++i) {
    sample_one(g, seed, domain, first_idx + (uint64_t)i, wk, smp);
    if (smp.status != ORC_OK) return smp.status;
    for (size_t k = 1; k + 1 < smp.path.size(); ++k) counts[smp.path[k]] += 1;
    if (totals)
      for (int k = 0; k < ST_COUNT; ++k) totals[k] += smp.st[k];
  }
  return ORC_OK;
}

double orc_omega(double lambda, double delta, int64_t vd) { return omega_of(lambda, delta, vd); }

int64_t orc_vd_bound(int64_t n, const int32_t* rp, const int32_t* ci, int directed, const int32_t* rrp,
                     const int32_t* rci) {
  Graph g = make_graph(n, rp, ci, directed, rrp, rci);
  return vd_bound(g);
}

double orc_compute_delta(int64_t n, const uint32_t* count0, uint64_t alpha, double omega, double lambda,
                         double delta, double eps, double* ln_inv_dl, double* ln_inv_du) {
  return compute_delta(n, count0, alpha, omega, lambda, delta, eps, ln_inv_dl, ln_inv_du);
}

void orc_f_and_g(uint32_t count, uint64_t tau, double omega, double lnL, double lnU, double* f, double* g) {
  f_and_g(count, tau, omega, lnL, lnU, f, g);
}

int orc_check_stop(int64_t n, const uint32_t* count, uint64_t tau, double omega, const double* lnL,
                   const double* lnU, double lambda, double* max_f, double* max_g) {
  return check_stop(n, count, tau, omega, lnL, lnU, lambda, max_f, max_g);
}

// Alg. 1 with the stop test every K samples: all-nodes mode (k = 0), or the
// k most central nodes (k > 0: Sec. 5 targets from a preliminary estimate,
// Alg. 2 with those targets, Alg. 3 as the stop test).
// counts: n (main-loop hits); count0: n or NULL (warm-up hits);
// ln_inv_dl/du: n or NULL (the computeDelta tables); topk: k or NULL;
// count_pre, lam_l, lam_u: n or NULL (top-k preliminary hits and targets).
static int run_impl(int64_t n, const int32_t* rp, const int32_t* ci, int directed, const int32_t* rrp,
                    const int32_t* rci, double lambda, double delta, uint64_t seed, uint64_t K, int64_t vd,
                    double eps, int64_t k, uint32_t* counts, uint32_t* count0_out, double* ln_inv_dl_out,
                    double* ln_inv_du_out, int32_t* topk_out, uint32_t* count_pre_out, double* lam_l_out,
                    double* lam_u_out, orc_result* res) {
  std::memset(res, 0, sizeof(*res));
  if (n < 2 || !(lambda > 0.0) || !(delta > 0.0) || !(delta < 1.0) || K == 0 || !(eps >= 0.0) ||
      !(eps < 0.5) || k < 0) {
    res->status = ORC_ERR_ARG;
    return ORC_ERR_ARG;
  }
  Graph g = make_graph(n, rp, ci, directed, rrp, rci);
  res->vd = vd > 0 ? vd : vd_bound(g);
  res->omega = omega_of(lambda, delta, res->vd);
  res->omega_cap = (uint64_t)std::ceil(res->omega);
  uint64_t alpha = (uint64_t)std::floor(res->omega / 100.0);
  if (alpha < 1) alpha = 1;
  res->alpha = alpha;

  Work wk(n);
  Sample smp;
  // alpha samples of one RNG domain, hits of interior nodes into cnt
  auto sample_into = [&](uint32_t domain, std::vector<uint32_t>& cnt) {
    for (uint64_t i = 0; i < alpha; ++i) {
      sample_one(g, seed, domain, i, wk, smp);
      if (smp.status != ORC_OK) return smp.status;
      for (size_t q = 1; q + 1 < smp.path.size(); ++q) cnt[smp.path[q]] += 1;
      res->edges_warm += smp.st[ST_EDGES];
    }
    return (int)ORC_OK;
  };

  // top-k: preliminary estimate (domain 2) and the Sec. 5 targets
  std::vector<double> lamL(n, lambda), lamU(n, lambda);
  std::vector<uint32_t> count_pre;
  if (k > 0) {
    count_pre.assign(n, 0);
    int st = sample_into(2, count_pre);
    if (st != ORC_OK) {
      res->status = st;
      return st;
    }
    topk_lambdas(n, count_pre.data(), alpha, k, lambda, lamL.data(), lamU.data());
  }
  // warm-up (domain 1) and computeDelta
  std::vector<uint32_t> count0(n, 0);
  {
    int st = sample_into(1, count0);
    if (st != ORC_OK) {
      res->status = st;
      return st;
    }
  }
  std::vector<double> lnL(n), lnU(n);
  if (k > 0)
    res->C = compute_delta_lv(n, count0.data(), alpha, res->omega, lamL.data(), lamU.data(), delta, eps,
                              lnL.data(), lnU.data());
  else
    res->C = compute_delta(n, count0.data(), alpha, res->omega, lambda, delta, eps, lnL.data(), lnU.data());

  // main loop (domain 0)
  for (int64_t v = 0; v < n; ++v) counts[v] = 0;
  uint64_t tau = 0;
  const uint64_t cap = res->omega_cap;
  auto stop_test = [&](double* mf, double* mg, int32_t* topk) {
    if (k > 0) return check_stop_topk(n, counts, tau, res->omega, lnL.data(), lnU.data(), lambda, k, topk, mf, mg);
    return check_stop(n, counts, tau, res->omega, lnL.data(), lnU.data(), lambda, mf, mg);
  };
  for (;;) {
    uint64_t B = std::min<uint64_t>(K, cap - tau);
    for (uint64_t i = 0; i < B; ++i) {
      sample_one(g, seed, 0, tau + i, wk, smp);
      if (smp.status != ORC_OK) {
        res->status = smp.status;
        return smp.status;
      }
      for (size_t q = 1; q + 1 < smp.path.size(); ++q) counts[smp.path[q]] += 1;
      res->edges_main += smp.st[ST_EDGES];
    }
    tau += B;
    if (tau >= cap) break;
    res->checks++;
    double mf, mg;
    if (stop_test(&mf, &mg, nullptr)) {
      res->stopped_early = 1;
      break;
    }
  }
  res->tau = tau;
  stop_test(&res->max_f, &res->max_g, topk_out);
  if (count0_out) std::memcpy(count0_out, count0.data(), sizeof(uint32_t) * n);
  if (ln_inv_dl_out) std::memcpy(ln_inv_dl_out, lnL.data(), sizeof(double) * n);
  if (ln_inv_du_out) std::memcpy(ln_inv_du_out, lnU.data(), sizeof(double) * n);
  if (k > 0 && count_pre_out) std::memcpy(count_pre_out, count_pre.data(), sizeof(uint32_t) * n);
  if (lam_l_out) std::memcpy(lam_l_out, lamL.data(), sizeof(double) * n);
  if (lam_u_out) std::memcpy(lam_u_out, lamU.data(), sizeof(double) * n);
  res->status = ORC_OK;
  return ORC_OK;
}

// Alg. 1 in all-nodes mode with the stop test every K samples.
int orc_run(int64_t n, const int32_t* rp, const int32_t* ci, int directed, const int32_t* rrp, const int32_t* rci,
            double lambda, double delta, uint64_t seed, uint64_t K, int64_t vd, double eps, uint32_t* counts,
            uint32_t* count0_out, double* ln_inv_dl_out, double* ln_inv_du_out, orc_result* res) {
  return run_impl(n, rp, ci, directed, rrp, rci, lambda, delta, seed, K, vd, eps, 0, counts, count0_out,
                  ln_inv_dl_out, ln_inv_du_out, nullptr, nullptr, nullptr, nullptr, res);
}

// Alg. 1 in top-k mode (k >= 1): Sec. 5 targets, Alg. 2, Alg. 3 every K samples.
int orc_run_topk(int64_t n, const int32_t* rp, const int32_t* ci, int directed, const int32_t* rrp,
                 const int32_t* rci, double lambda, double delta, uint64_t seed, uint64_t K, int64_t vd, double eps,
                 int64_t k, uint32_t* counts, uint32_t* count0_out, double* ln_inv_dl_out, double* ln_inv_du_out,
                 int32_t* topk_out, uint32_t* count_pre_out, double* lam_l_out, double* lam_u_out, orc_result* res) {
  if (k < 1) {
    std::memset(res, 0, sizeof(*res));
    res->status = ORC_ERR_ARG;
    return ORC_ERR_ARG;
  }
  return run_impl(n, rp, ci, directed, rrp, rci, lambda, delta, seed, K, vd, eps, k, counts, count0_out,
                  ln_inv_dl_out, ln_inv_du_out, topk_out, count_pre_out, lam_l_out, lam_u_out, res);
}

double orc_compute_delta_lv(int64_t n, const uint32_t* count0, uint64_t alpha, double omega, const double* lamL,
                            const double* lamU, double delta, double eps, double* ln_inv_dl, double* ln_inv_du) {
  return compute_delta_lv(n, count0, alpha, omega, lamL, lamU, delta, eps, ln_inv_dl, ln_inv_du);
}

void orc_topk_lambdas(int64_t n, const uint32_t* count_pre, uint64_t alpha_pre, int64_t k, double lambda,
                      double* lamL, double* lamU) {
  topk_lambdas(n, count_pre, alpha_pre, k, lambda, lamL, lamU);
}

int orc_check_stop_topk(int64_t n, const uint32_t* count, uint64_t tau, double omega, const double* lnL,
                        const double* lnU, double lambda, int64_t k, int32_t* topk, double* max_f, double* max_g) {
  return check_stop_topk(n, count, tau, omega, lnL, lnU, lambda, k, topk, max_f, max_g);
}

// Exact normalised betweenness bc(v) = 1/(n(n-1)) sum_{s!=v!=t} sigma_st(v)/sigma_st
// over ordered pairs (Sec. 2), by Brandes' dependency accumulation.
int orc_brandes(int64_t n, const int32_t* rp, const int32_t* ci, int directed, const int32_t* rrp,
                const int32_t* rci, double* bc) {
  if (n < 2) return ORC_ERR_ARG;
  Graph g = make_graph(n, rp, ci, directed, rrp, rci);
  for (int64_t v = 0; v < n; ++v) bc[v] = 0.0;
  std::vector<int32_t> dist(n), order;
  std::vector<double> sigma(n), dep(n);
  for (int32_t s = 0; s < n; ++s) {
    std::fill(dist.begin(), dist.end(), -1);
    std::fill(sigma.begin(), sigma.end(), 0.0);
    std::fill(dep.begin(), dep.end(), 0.0);
    order.clear();
    dist[s] = 0;
    sigma[s] = 1.0;
    order.push_back(s);
    for (size_t h = 0; h < order.size(); ++h) {
      int32_t v = order[h];
      for (int32_t e = g.rp[v]; e < g.rp[v + 1]; ++e) {
        int32_t w = g.ci[e];
        if (dist[w] < 0) {
          dist[w] = dist[v] + 1;
          order.push_back(w);
        }
        if (dist[w] == dist[v] + 1) sigma[w] += sigma[v];
      }
    }
    for (size_t h = order.size(); h-- > 0;) {
      int32_t w = order[h];
      for (int32_t e = g.rrp[w]; e < g.rrp[w + 1]; ++e) {
        int32_t v = g.rci[e];
        if (dist[v] >= 0 && dist[v] == dist[w] - 1) dep[v] += sigma[v] / sigma[w] * (1.0 + dep[w]);
      }
      if (w != s) bc[w] += dep[w];
    }
  }
  const double norm = 1.0 / ((double)n * (double)(n - 1));
  for (int64_t v = 0; v < n; ++v) bc[v] *= norm;
  return ORC_OK;
}

// All shortest s->t paths by brute force (DFS over the BFS layering from
// s, pruned by the distance to t).  Returns the number of paths (or -1 if
// more than max_paths); paths is max_paths*max_len, -1 padded.
int64_t orc_enumerate_paths(int64_t n, const int32_t* rp, const int32_t* ci, int directed, const int32_t* rrp,
                            const int32_t* rci, int32_t s, int32_t t, int64_t max_paths, int32_t max_len,
                            int32_t* paths) {
  Graph g = make_graph(n, rp, ci, directed, rrp, rci);
  std::vector<int32_t> ds(n, -1), dt(n, -1), q;
  ds[s] = 0;
  q.push_back(s);
  for (size_t h = 0; h < q.size(); ++h)
    for (int32_t e = g.rp[q[h]]; e < g.rp[q[h] + 1]; ++e)
      if (ds[g.ci[e]] < 0) {
        ds[g.ci[e]] = ds[q[h]] + 1;
        q.push_back(g.ci[e]);
      }
  q.clear();
  dt[t] = 0;
  q.push_back(t);
  for (size_t h = 0; h < q.size(); ++h)
    for (int32_t e = g.rrp[q[h]]; e < g.rrp[q[h] + 1]; ++e)
      if (dt[g.rci[e]] < 0) {
        dt[g.rci[e]] = dt[q[h]] + 1;
        q.push_back(g.rci[e]);
      }
  if (ds[t] < 0) return 0;
  const int32_t d = ds[t];
  if (d + 1 > max_len) return -1;
  int64_t found = 0;
  std::vector<int32_t> stack_path(1, s);
  // iterative DFS with explicit edge cursors
  std::vector<int32_t> cursor(1, g.rp[s]);
  while (!stack_path.empty()) {
    int32_t v = stack_path.back();
    if (v == t) {
      if (found >= max_paths) return -1;
      for (int32_t k = 0; k < max_len; ++k)
        paths[found * max_len + k] = k < (int32_t)stack_path.size() ? stack_path[k] : -1;
      ++found;
      stack_path.pop_back();
      cursor.pop_back();
      continue;
    }
    int32_t& e = cursor.back();
    bool pushed = false;
    while (e < g.rp[v + 1]) {
      int32_t w = g.ci[e++];
      if (ds[w] == ds[v] + 1 && dt[w] >= 0 && ds[w] + dt[w] == d) {
        stack_path.push_back(w);
        cursor.push_back(g.rp[w]);
        pushed = true;
        break;
      }
    }
    if (!pushed) {
      stack_path.pop_back();
      cursor.pop_back();
    }
  }
  return found;
}

}  // extern "C"
