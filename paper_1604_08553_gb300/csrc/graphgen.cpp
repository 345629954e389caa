// Seeded synthetic graph generators (input side only).
//
// These produce the unweighted graphs G=(V,E) that the sampler and the
// oracle both consume (paper Sec. 2: unweighted static graphs, directed or
// undirected; directed graphs need forward and backward adjacency, Sec. 4).
// Nothing here computes any part of the betweenness method: the output is an
// int32 CSR with sorted, de-duplicated rows, no self-loops, plus the reverse
// CSR for directed graphs.
//
// Families (paper Sec. 6 measures real SNAP/KONECT/LASAGNE networks that are
// not available here; these stand in for them):
//   * Erdos-Renyi G(n,p)
//   * Chung-Lu with a power-law expected-degree sequence (App. E, Rank-1
//     inhomogeneous random graphs: edge {u,v} with prob. min(1, w_u w_v / M))
//   * Barabasi-Albert preferential attachment
//   * R-MAT (recursive matrix), directed
//
// Randomness: splitmix64 streams (Steele, Lea, Flood, OOPSLA 2014), one
// stream per independent unit of work, so threaded generation is
// deterministic regardless of the thread count.  ER and R-MAT decisions use
// integer thresholds only; Chung-Lu and the large-n ER path call libm log/pow,
// so their output is reproducible on one machine but may differ across libm
// builds in rare edge decisions.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

struct gg_graph {
  int64_t n = 0;
  int directed = 0;
  std::vector<int32_t> row_ptr, col;    // forward CSR (out-arcs)
  std::vector<int32_t> rrow_ptr, rcol;  // reverse CSR (in-arcs), directed only
};

namespace {

using Graph = gg_graph;

inline uint64_t sm64_next(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

inline uint64_t stream_seed(uint64_t seed, uint64_t unit, uint64_t salt) {
  uint64_t x = seed ^ (0xD1B54A32D192ED03ULL * (salt + 1));
  uint64_t a = sm64_next(x);
  uint64_t y = unit ^ a;
  return sm64_next(y);
}

// uniform in (0,1), never 0 or 1
inline double u01_open(uint64_t& st) {
  return ((double)(sm64_next(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

unsigned num_workers() {
  unsigned h = std::thread::hardware_concurrency();
  if (h == 0) h = 1;
  if (h > 64) h = 64;
  return h;
}

template <class F>
void parallel_chunks(int64_t nchunks, F&& f) {
  unsigned w = num_workers();
  if (w <= 1 || nchunks <= 1) {
    for (int64_t c = 0; c < nchunks; ++c) f(c);
    return;
  }
  std::vector<std::thread> th;
  std::atomic_int64_t next{0};
  for (unsigned i = 0; i < w; ++i)
    th.emplace_back([&] {
      for (;;) {
        int64_t c = next.fetch_add(1);
        if (c >= nchunks) break;
        f(c);
      }
    });
  for (auto& t : th) t.join();
}

// Builds a CSR (sorted rows, no duplicates, no self-loops) from an arc list.
void build_csr(int64_t n, const std::vector<int32_t>& src, const std::vector<int32_t>& dst,
               std::vector<int32_t>& row_ptr, std::vector<int32_t>& col) {
  const int64_t m = (int64_t)src.size();
  std::vector<int64_t> deg(n + 1, 0);
  for (int64_t e = 0; e < m; ++e)
    if (src[e] != dst[e]) deg[src[e] + 1]++;
  for (int64_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
  std::vector<int32_t> tmp(deg[n]);
  {
    std::vector<int64_t> pos(deg.begin(), deg.end() - 1);
    for (int64_t e = 0; e < m; ++e)
      if (src[e] != dst[e]) tmp[pos[src[e]]++] = dst[e];
  }
  // sort + unique each row (chunked by node ranges, deterministic)
  std::vector<int64_t> newdeg(n, 0);
  const int64_t CH = 1 << 14;
  const int64_t nch = (n + CH - 1) / CH;
  parallel_chunks(nch, [&](int64_t c) {
    int64_t lo = c * CH, hi = std::min<int64_t>(n, lo + CH);
    for (int64_t v = lo; v < hi; ++v) {
      int32_t* b = tmp.data() + deg[v];
      int32_t* e = tmp.data() + deg[v + 1];
      std::sort(b, e);
      newdeg[v] = std::unique(b, e) - b;
    }
  });
  row_ptr.assign(n + 1, 0);
  for (int64_t v = 0; v < n; ++v) row_ptr[v + 1] = (int32_t)(row_ptr[v] + newdeg[v]);
  col.resize(row_ptr[n]);
  parallel_chunks(nch, [&](int64_t c) {
    int64_t lo = c * CH, hi = std::min<int64_t>(n, lo + CH);
    for (int64_t v = lo; v < hi; ++v)
      std::memcpy(col.data() + row_ptr[v], tmp.data() + deg[v], sizeof(int32_t) * newdeg[v]);
  });
}

int32_t uf_find(std::vector<int32_t>& p, int32_t x) {
  while (p[x] != x) {
    p[x] = p[p[x]];
    x = p[x];
  }
  return x;
}

// Keeps only the largest weakly connected component (ties: the component
// holding the smallest node id); nodes are renumbered in increasing order.
void keep_lcc(int64_t& n, std::vector<int32_t>& src, std::vector<int32_t>& dst) {
  std::vector<int32_t> p(n);
  std::iota(p.begin(), p.end(), 0);
  for (size_t e = 0; e < src.size(); ++e) {
    int32_t a = uf_find(p, src[e]), b = uf_find(p, dst[e]);
    if (a != b) {
      if (a < b) std::swap(a, b);
      p[a] = b;
    }
  }
  std::vector<int64_t> sz(n, 0);
  for (int64_t v = 0; v < n; ++v) sz[uf_find(p, (int32_t)v)]++;
  int32_t best = 0;
  for (int64_t v = 0; v < n; ++v)
    if (sz[v] > sz[best]) best = (int32_t)v;
  std::vector<int32_t> id(n, -1);
  int32_t k = 0;
  for (int64_t v = 0; v < n; ++v)
    if (uf_find(p, (int32_t)v) == best) id[v] = k++;
  size_t w = 0;
  for (size_t e = 0; e < src.size(); ++e) {
    if (id[src[e]] >= 0) {
      src[w] = id[src[e]];
      dst[w] = id[dst[e]];
      ++w;
    }
  }
  src.resize(w);
  dst.resize(w);
  n = k;
}

Graph* finish_undirected(int64_t n, std::vector<int32_t>& a, std::vector<int32_t>& b, int lcc) {
  if (lcc) keep_lcc(n, a, b);
  const size_t m = a.size();
  std::vector<int32_t> src(2 * m), dst(2 * m);
  for (size_t e = 0; e < m; ++e) {
    src[2 * e] = a[e];
    dst[2 * e] = b[e];
    src[2 * e + 1] = b[e];
    dst[2 * e + 1] = a[e];
  }
  std::vector<int32_t>().swap(a);
  std::vector<int32_t>().swap(b);
  Graph* g = new Graph;
  g->n = n;
  g->directed = 0;
  build_csr(n, src, dst, g->row_ptr, g->col);
  return g;
}

Graph* finish_directed(int64_t n, std::vector<int32_t>& src, std::vector<int32_t>& dst, int lcc) {
  if (lcc) keep_lcc(n, src, dst);
  Graph* g = new Graph;
  g->n = n;
  g->directed = 1;
  build_csr(n, src, dst, g->row_ptr, g->col);
  // reverse CSR from the de-duplicated forward arcs
  std::vector<int32_t> rs(g->col.size()), rd(g->col.size());
  for (int64_t v = 0; v < n; ++v)
    for (int32_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
      rs[e] = g->col[e];
      rd[e] = (int32_t)v;
    }
  std::vector<int32_t>().swap(src);
  std::vector<int32_t>().swap(dst);
  build_csr(n, rs, rd, g->rrow_ptr, g->rcol);
  return g;
}

}  // namespace

extern "C" {

// Erdos-Renyi G(n, p) with p = avg_deg / (n-1).  For n <= 65536 every pair
// {u<v} is one Bernoulli trial decided by a 64-bit integer threshold; larger
// n uses geometric skipping over the pair index (Batagelj & Brandes 2005).
gg_graph* gg_erdos_renyi(int64_t n, double avg_deg, uint64_t seed, int lcc) {
  if (n < 2 || n > (int64_t)INT32_MAX) return nullptr;
  const double p = avg_deg / (double)(n - 1);
  if (!(p > 0.0) || p >= 1.0) return nullptr;
  std::vector<int32_t> a, b;
  if (n <= 65536) {
    const uint64_t thr = (uint64_t)std::ldexp(p, 64);
    for (int64_t u = 0; u < n; ++u) {
      uint64_t st = stream_seed(seed, (uint64_t)u, 1);
      for (int64_t v = u + 1; v < n; ++v)
        if (sm64_next(st) < thr) {
          a.push_back((int32_t)u);
          b.push_back((int32_t)v);
        }
    }
  } else {
    uint64_t st = stream_seed(seed, 0, 2);
    const double lq = std::log1p(-p);
    int64_t v = 1, w = -1;
    while (v < n) {
      double r = u01_open(st);
      w += 1 + (int64_t)std::floor(std::log(r) / lq);
      while (w >= v && v < n) {
        w -= v;
        ++v;
      }
      if (v < n) {
        a.push_back((int32_t)w);
        b.push_back((int32_t)v);
      }
    }
  }
  return finish_undirected(n, a, b, lcc);
}

// Chung-Lu: expected degrees w_i proportional to (i+1)^(-1/(beta-1)),
// scaled to mean `mean_deg` with the maximum capped at `max_deg` (the
// uncapped weights are rescaled until the mean holds).  Edge {u,v}, u<v, is
// present with probability min(1, w_u w_v / sum(w)).  Generated with the
// skip method of Miller & Hagberg (WAW 2011), one stream per node u.
gg_graph* gg_chung_lu(int64_t n, double beta, double mean_deg, double max_deg, uint64_t seed, int lcc) {
  if (n < 2 || n > (int64_t)INT32_MAX || !(beta > 2.0)) return nullptr;
  std::vector<double> w(n);
  const double ex = -1.0 / (beta - 1.0);
  for (int64_t i = 0; i < n; ++i) w[i] = std::pow((double)(i + 1), ex);
  std::vector<char> capped(n, 0);
  for (int it = 0; it < 64; ++it) {
    double sum_c = 0.0, sum_u = 0.0;
    for (int64_t i = 0; i < n; ++i) (capped[i] ? sum_c : sum_u) += w[i];
    const double target = mean_deg * (double)n - sum_c;
    const double sc = target / sum_u;
    bool changed = false;
    for (int64_t i = 0; i < n; ++i)
      if (!capped[i]) {
        w[i] *= sc;
        if (w[i] > max_deg) {
          w[i] = max_deg;
          capped[i] = 1;
          changed = true;
        }
      }
    if (!changed) break;
  }
  double S = 0.0;
  for (int64_t i = 0; i < n; ++i) S += w[i];
  const int64_t CH = 4096;
  const int64_t nch = (n + CH - 1) / CH;
  std::vector<std::vector<int32_t>> ca(nch), cb(nch);
  parallel_chunks(nch, [&](int64_t c) {
    int64_t lo = c * CH, hi = std::min<int64_t>(n - 1, lo + CH);
    for (int64_t u = lo; u < hi; ++u) {
      uint64_t st = stream_seed(seed, (uint64_t)u, 3);
      int64_t v = u + 1;
      double p = std::min(w[u] * w[v] / S, 1.0);
      while (v < n && p > 0.0) {
        if (p != 1.0) {
          double r = u01_open(st);
          v += (int64_t)std::floor(std::log(r) / std::log1p(-p));
        }
        if (v < n) {
          double q = std::min(w[u] * w[v] / S, 1.0);
          double r = u01_open(st);
          if (r < q / p) {
            ca[c].push_back((int32_t)u);
            cb[c].push_back((int32_t)v);
          }
          p = q;
          ++v;
        }
      }
    }
  });
  std::vector<int32_t> a, b;
  for (int64_t c = 0; c < nch; ++c) {
    a.insert(a.end(), ca[c].begin(), ca[c].end());
    b.insert(b.end(), cb[c].begin(), cb[c].end());
    std::vector<int32_t>().swap(ca[c]);
    std::vector<int32_t>().swap(cb[c]);
  }
  return finish_undirected(n, a, b, lcc);
}

// Barabasi-Albert preferential attachment with m edges per new node, in the
// linear-time form of Batagelj & Brandes (2005): each new edge copies a
// uniformly chosen endpoint of an earlier edge.  Duplicate edges and
// self-loops are dropped afterwards, so the graph is simple.
gg_graph* gg_barabasi_albert(int64_t n, int32_t m, uint64_t seed) {
  if (n < 2 || m < 1 || n > (int64_t)INT32_MAX) return nullptr;
  std::vector<int32_t> M((size_t)2 * n * m);
  uint64_t st = stream_seed(seed, 0, 4);
  for (int64_t v = 0; v < n; ++v)
    for (int32_t i = 0; i < m; ++i) {
      const uint64_t k = 2 * ((uint64_t)v * m + i);
      M[k] = (int32_t)v;
      // uniform in [0, k]
      const uint64_t r = (uint64_t)(((unsigned __int128)sm64_next(st) * (k + 1)) >> 64);
      M[k + 1] = M[r];
    }
  std::vector<int32_t> a((size_t)n * m), b((size_t)n * m);
  for (size_t e = 0; e < (size_t)n * m; ++e) {
    a[e] = M[2 * e];
    b[e] = M[2 * e + 1];
  }
  std::vector<int32_t>().swap(M);
  return finish_undirected(n, a, b, 0);
}

// R-MAT (Chakrabarti, Zhan, Faloutsos 2004), directed, 2^scale nodes and
// edge_factor * 2^scale generated arcs; quadrant probabilities (a,b,c,d) are
// applied at every level with 32-bit integer thresholds.  Self-loops and
// duplicate arcs are removed; all node ids are kept (no LCC).
gg_graph* gg_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed) {
  if (scale < 1 || scale > 30 || edge_factor < 1) return nullptr;
  const int64_t n = (int64_t)1 << scale;
  const int64_t m = n * edge_factor;
  const uint64_t ta = (uint64_t)std::ldexp(a, 32);
  const uint64_t tb = (uint64_t)std::ldexp(a + b, 32);
  const uint64_t tc = (uint64_t)std::ldexp(a + b + c, 32);
  std::vector<int32_t> src(m), dst(m);
  const int64_t CH = 1 << 16;
  const int64_t nch = (m + CH - 1) / CH;
  parallel_chunks(nch, [&](int64_t ch) {
    int64_t lo = ch * CH, hi = std::min<int64_t>(m, lo + CH);
    for (int64_t e = lo; e < hi; ++e) {
      uint64_t st = stream_seed(seed, (uint64_t)e, 5);
      uint32_t u = 0, v = 0;
      uint64_t bits = 0;
      for (int32_t l = 0; l < scale; ++l) {
        if ((l & 1) == 0) bits = sm64_next(st);
        const uint64_t r = (l & 1) ? (bits >> 32) : (bits & 0xffffffffULL);
        u <<= 1;
        v <<= 1;
        if (r < ta) {
        } else if (r < tb) {
          v |= 1;
        } else if (r < tc) {
          u |= 1;
        } else {
          u |= 1;
          v |= 1;
        }
      }
      src[e] = (int32_t)u;
      dst[e] = (int32_t)v;
    }
  });
  return finish_directed(n, src, dst, 0);
}

int64_t gg_num_nodes(const gg_graph* g) { return g ? g->n : -1; }
int64_t gg_num_arcs(const gg_graph* g) { return g ? (int64_t)g->col.size() : -1; }
int gg_is_directed(const gg_graph* g) { return g ? g->directed : -1; }

// Copies the CSR out; rrow_ptr/rcol may be NULL and are ignored for
// undirected graphs.
int gg_copy(const gg_graph* g, int32_t* row_ptr, int32_t* col, int32_t* rrow_ptr, int32_t* rcol) {
  if (!g) return -1;
  std::memcpy(row_ptr, g->row_ptr.data(), sizeof(int32_t) * (g->n + 1));
  std::memcpy(col, g->col.data(), sizeof(int32_t) * g->col.size());
  if (g->directed && rrow_ptr && rcol) {
    std::memcpy(rrow_ptr, g->rrow_ptr.data(), sizeof(int32_t) * (g->n + 1));
    std::memcpy(rcol, g->rcol.data(), sizeof(int32_t) * g->rcol.size());
  }
  return 0;
}

void gg_free(gg_graph* g) { delete g; }

}  // extern "C"
