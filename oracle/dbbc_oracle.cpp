// CPU oracle for balanced / unbalanced butterfly counting in signed bipartite
// graphs. TEST INFRASTRUCTURE ONLY: tests, the smoke check and the CPU-baseline
// leg of the benchmark use it; the product path never does.
//
// Everything here is plain, serial-by-default C++17 written from the paper's
// definitions, with no blocking or reordering beyond what they state:
//
//   * Def. 1 / Def. 2 (Section III): a butterfly is {u,u'} x {v,v'} with all four
//     edges present; it is balanced iff the number of negative edges is even.
//   * Def. 3 (Section III): vertex priority over U u V, higher degree first, ties
//     broken by the larger id. Ids here are one unified space: id(u) = u for
//     u in U and id(v) = |U| + v for v in V.
//   * Algorithm 1, Phase 5 (Section IV-A): for every pivot u, for every
//     neighbour v with p(v) < p(u), for every neighbour w of v with p(w) < p(u),
//     bump B1[w] if s(u,v) = s(v,w) and B2[w] otherwise; then every touched
//     endpoint adds C(B1,2) + C(B2,2) balanced butterflies and the buckets are
//     reset.
//   * Lemma 1 (Section III), case 3: a symmetric and an asymmetric wedge with the
//     same endpoints close an unbalanced butterfly, so each touched endpoint
//     adds B1 * B2 unbalanced ones (the paper counts only the balanced ones).
//   * Duplicate edges keep the latest occurrence (Section V, dataset
//     preprocessing).
//
// Signs are int8 +1 / -1. Counts are accumulated in 128-bit integers and the
// call fails with code 5 if a total does not fit in 64 bits.
//
// Also here: a brute-force enumerator of Def. 1-2 over a dense sign matrix,
// sharing nothing with the Algorithm 1 code above it.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

using u128 = unsigned __int128;

enum { OK = 0, BAD_INPUT = 1, OVERFLOW_64 = 5 };

struct SignedGraph {
  int64_t n = 0;  // |U| + |V|
  std::vector<std::vector<std::pair<int32_t, int8_t>>> adj;  // unified ids
  std::vector<int64_t> deg;
};

// Validate, keep the latest sign of every (u, v) pair, and build adjacency
// lists over the unified id space.
int build_graph(const int32_t* u, const int32_t* v, const int8_t* s, int64_t m, int32_t n_u, int32_t n_v,
                SignedGraph& g) {
  if (m < 0 || n_u < 0 || n_v < 0) return BAD_INPUT;
  for (int64_t i = 0; i < m; i++) {
    if (u[i] < 0 || u[i] >= n_u || v[i] < 0 || v[i] >= n_v) return BAD_INPUT;
    if (s[i] != 1 && s[i] != -1) return BAD_INPUT;
  }
  std::unordered_map<uint64_t, int8_t> latest;
  latest.reserve(static_cast<size_t>(m) * 2 + 1);
  for (int64_t i = 0; i < m; i++) {
    uint64_t key = (static_cast<uint64_t>(u[i]) << 32) | static_cast<uint32_t>(v[i]);
    latest[key] = s[i];  // a later occurrence overwrites an earlier one
  }
  g.n = static_cast<int64_t>(n_u) + n_v;
  g.adj.assign(static_cast<size_t>(g.n), {});
  for (const auto& kv : latest) {
    int32_t a = static_cast<int32_t>(kv.first >> 32);
    int32_t b = n_u + static_cast<int32_t>(kv.first & 0xFFFFFFFFu);
    g.adj[a].push_back({b, kv.second});
    g.adj[b].push_back({a, kv.second});
  }
  g.deg.resize(static_cast<size_t>(g.n));
  for (int64_t x = 0; x < g.n; x++) g.deg[x] = static_cast<int64_t>(g.adj[x].size());
  return OK;
}

// Def. 3: p(a) < p(b).
inline bool lower_priority(const SignedGraph& g, int64_t a, int64_t b) {
  if (g.deg[a] != g.deg[b]) return g.deg[a] < g.deg[b];
  return a < b;
}

inline u128 choose2(u128 x) { return x < 2 ? 0 : x * (x - 1) / 2; }

struct Totals {
  u128 balanced = 0, unbalanced = 0, wedges = 0;
};

// Pivots visited by one run: first, first + step, first + 2*step, ... below n.
struct PivotSample {
  int64_t first = 0, step = 1;
  int64_t count(int64_t n) const { return first >= n ? 0 : (n - first + step - 1) / step; }
};

// Algorithm 1, Phase 5, for the sample's pivots taken from `next` (an index
// into the sample) until exhausted. Optional per-pivot outputs are indexed by
// unified id.
void count_pivots(const SignedGraph& g, PivotSample ps, std::atomic<int64_t>* next, int64_t chunk, Totals* out,
                  uint64_t* bal_pp, uint64_t* unb_pp, uint64_t* wed_pp) {
  std::vector<uint32_t> B1(static_cast<size_t>(g.n), 0), B2(static_cast<size_t>(g.n), 0);
  std::vector<int32_t> touched;
  std::vector<uint8_t> seen(static_cast<size_t>(g.n), 0);
  Totals t;
  const int64_t total = ps.count(g.n);
  for (;;) {
    int64_t begin = next->fetch_add(chunk);
    if (begin >= total) break;
    int64_t end = std::min(begin + chunk, total);
    for (int64_t k = begin; k < end; k++) {
      const int64_t u = ps.first + k * ps.step;
      for (const auto& uv : g.adj[u]) {
        int32_t v = uv.first;
        if (!lower_priority(g, v, u)) continue;
        for (const auto& vw : g.adj[v]) {
          int32_t w = vw.first;
          if (!lower_priority(g, w, u)) continue;
          if (uv.second == vw.second) B1[w]++; else B2[w]++;
          if (!seen[w]) { seen[w] = 1; touched.push_back(w); }
        }
      }
      u128 bal = 0, unb = 0, wed = 0;
      for (int32_t w : touched) {
        bal += choose2(B1[w]) + choose2(B2[w]);
        unb += static_cast<u128>(B1[w]) * B2[w];
        wed += static_cast<u128>(B1[w]) + B2[w];
        B1[w] = 0;
        B2[w] = 0;
        seen[w] = 0;
      }
      touched.clear();
      t.balanced += bal;
      t.unbalanced += unb;
      t.wedges += wed;
      if (bal_pp) bal_pp[u] = static_cast<uint64_t>(bal);
      if (unb_pp) unb_pp[u] = static_cast<uint64_t>(unb);
      if (wed_pp) wed_pp[u] = static_cast<uint64_t>(wed);
    }
  }
  *out = t;
}

int count_graph(const SignedGraph& g, PivotSample ps, int threads, uint64_t* balanced, uint64_t* unbalanced,
                uint64_t* wedges, uint64_t* bal_pp, uint64_t* unb_pp, uint64_t* wed_pp) {
  if (threads < 1) threads = 1;
  std::atomic<int64_t> next{0};
  std::vector<Totals> part(static_cast<size_t>(threads));
  if (threads == 1) {
    count_pivots(g, ps, &next, std::max<int64_t>(ps.count(g.n), 1), &part[0], bal_pp, unb_pp, wed_pp);
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; t++)
      pool.emplace_back(count_pivots, std::cref(g), ps, &next, int64_t{64}, &part[t], bal_pp, unb_pp, wed_pp);
    for (auto& th : pool) th.join();
  }
  Totals tot;
  for (const auto& p : part) {
    tot.balanced += p.balanced;
    tot.unbalanced += p.unbalanced;
    tot.wedges += p.wedges;
  }
  const u128 lim = static_cast<u128>(UINT64_MAX);
  if (tot.balanced > lim || tot.unbalanced > lim || tot.wedges > lim) return OVERFLOW_64;
  if (balanced) *balanced = static_cast<uint64_t>(tot.balanced);
  if (unbalanced) *unbalanced = static_cast<uint64_t>(tot.unbalanced);
  if (wedges) *wedges = static_cast<uint64_t>(tot.wedges);
  return OK;
}

int run_algorithm1(const int32_t* u, const int32_t* v, const int8_t* s, int64_t m, int32_t n_u, int32_t n_v,
                   int threads, uint64_t* balanced, uint64_t* unbalanced, uint64_t* wedges, uint64_t* bal_pp,
                   uint64_t* unb_pp, uint64_t* wed_pp) {
  SignedGraph g;
  int rc = build_graph(u, v, s, m, n_u, n_v, g);
  if (rc != OK) return rc;
  return count_graph(g, PivotSample{}, threads, balanced, unbalanced, wedges, bal_pp, unb_pp, wed_pp);
}

}  // namespace

extern "C" {

// Totals of Algorithm 1 (balanced, Lemma-1 unbalanced, accepted wedges).
// threads > 1 splits the pivots over std::threads with private buckets, the
// scheme the paper uses inside one node (Section IV-A, Phase 5).
int oracle_count(const int32_t* u, const int32_t* v, const int8_t* s, int64_t m, int32_t n_u, int32_t n_v,
                 int threads, uint64_t* balanced, uint64_t* unbalanced, uint64_t* wedges) {
  return run_algorithm1(u, v, s, m, n_u, n_v, threads, balanced, unbalanced, wedges, nullptr, nullptr, nullptr);
}

// Per-pivot contributions of Algorithm 1, indexed by unified id (arrays of
// length n_u + n_v). Each butterfly is attributed to its highest-priority
// vertex (Theorem 1).
int oracle_count_per_pivot(const int32_t* u, const int32_t* v, const int8_t* s, int64_t m, int32_t n_u,
                           int32_t n_v, int threads, uint64_t* bal_pp, uint64_t* unb_pp, uint64_t* wed_pp) {
  uint64_t b, ub, w;
  return run_algorithm1(u, v, s, m, n_u, n_v, threads, &b, &ub, &w, bal_pp, unb_pp, wed_pp);
}

// A graph built once (validation, keep-latest dedup, adjacency) and counted
// many times, so that Algorithm 1 can be timed alone on pivot samples.
void* oracle_graph_new(const int32_t* u, const int32_t* v, const int8_t* s, int64_t m, int32_t n_u, int32_t n_v,
                       int* status) {
  SignedGraph* g = new SignedGraph();
  int rc = build_graph(u, v, s, m, n_u, n_v, *g);
  if (status) *status = rc;
  if (rc != OK) {
    delete g;
    return nullptr;
  }
  return g;
}

// Algorithm 1 over the pivots first, first + step, ... of a built graph.
int oracle_graph_count_sample(const void* h, int64_t first, int64_t step, int threads, uint64_t* balanced,
                              uint64_t* unbalanced, uint64_t* wedges) {
  if (!h || first < 0 || step < 1) return BAD_INPUT;
  PivotSample ps;
  ps.first = first;
  ps.step = step;
  return count_graph(*static_cast<const SignedGraph*>(h), ps, threads, balanced, unbalanced, wedges, nullptr, nullptr,
                     nullptr);
}

void oracle_graph_free(void* h) { delete static_cast<SignedGraph*>(h); }

// Butterflies containing each vertex (unified ids), following Algorithm 1:
// after a pivot's buckets are complete, every touched endpoint w and the
// pivot itself are in C(B1[w],2) + C(B2[w],2) balanced and B1[w]*B2[w]
// unbalanced butterflies of that pivot; a middle vertex v of a symmetric
// wedge u-v-w pairs with the B1[w] - 1 other symmetric wedges (balanced) and
// the B2[w] asymmetric ones (unbalanced), and an asymmetric middle the other
// way round (Lemma 1). The middles are found by walking the pivot's wedges a
// second time.
int oracle_count_per_vertex(const int32_t* u, const int32_t* v, const int8_t* s, int64_t m, int32_t n_u,
                            int32_t n_v, uint64_t* bal_v, uint64_t* unb_v) {
  SignedGraph g;
  int rc = build_graph(u, v, s, m, n_u, n_v, g);
  if (rc != OK) return rc;
  std::vector<uint32_t> B1(static_cast<size_t>(g.n), 0), B2(static_cast<size_t>(g.n), 0);
  std::vector<uint8_t> seen(static_cast<size_t>(g.n), 0);
  std::vector<int32_t> touched;
  std::vector<u128> bal(static_cast<size_t>(g.n), 0), unb(static_cast<size_t>(g.n), 0);
  for (int64_t p = 0; p < g.n; p++) {
    for (const auto& pv : g.adj[p]) {
      if (!lower_priority(g, pv.first, p)) continue;
      for (const auto& vw : g.adj[pv.first]) {
        if (!lower_priority(g, vw.first, p)) continue;
        if (pv.second == vw.second) B1[vw.first]++; else B2[vw.first]++;
        if (!seen[vw.first]) { seen[vw.first] = 1; touched.push_back(vw.first); }
      }
    }
    for (int32_t w : touched) {
      const u128 c = choose2(B1[w]) + choose2(B2[w]), d = static_cast<u128>(B1[w]) * B2[w];
      bal[p] += c;
      unb[p] += d;
      bal[w] += c;
      unb[w] += d;
    }
    for (const auto& pv : g.adj[p]) {  // second walk: the middle vertices
      if (!lower_priority(g, pv.first, p)) continue;
      for (const auto& vw : g.adj[pv.first]) {
        if (!lower_priority(g, vw.first, p)) continue;
        const uint32_t same = pv.second == vw.second ? B1[vw.first] : B2[vw.first];
        const uint32_t other = pv.second == vw.second ? B2[vw.first] : B1[vw.first];
        bal[pv.first] += same - 1;
        unb[pv.first] += other;
      }
    }
    for (int32_t w : touched) {
      B1[w] = 0;
      B2[w] = 0;
      seen[w] = 0;
    }
    touched.clear();
  }
  const u128 lim = static_cast<u128>(UINT64_MAX);
  for (int64_t x = 0; x < g.n; x++) {
    if (bal[x] > lim || unb[x] > lim) return OVERFLOW_64;
    bal_v[x] = static_cast<uint64_t>(bal[x]);
    unb_v[x] = static_cast<uint64_t>(unb[x]);
  }
  return OK;
}

// Butterflies containing each edge (the pairs (qu[i], qv[i]), local ids; a
// pair that is not an edge is in none), following Algorithm 1: once a pivot's
// buckets are complete, the wedge u-v-w pairs with the other wedges that end
// at w, B1[w] - 1 + B2[w] of them, closing a butterfly through both of its
// edges (u, v) and (v, w); the pairs with the wedges of the same sign class are
// balanced and the others unbalanced (Lemma 1). Every butterfly is found at its
// highest-priority vertex with its four edges on its two wedges, so each edge
// is credited once per butterfly. The wedges are walked a second time.
int oracle_count_per_edge(const int32_t* u, const int32_t* v, const int8_t* s, int64_t m, int32_t n_u,
                          int32_t n_v, const int32_t* qu, const int32_t* qv, int64_t k, uint64_t* bal_e,
                          uint64_t* unb_e) {
  SignedGraph g;
  int rc = build_graph(u, v, s, m, n_u, n_v, g);
  if (rc != OK) return rc;
  if (k < 0) return BAD_INPUT;
  for (int64_t i = 0; i < k; i++)
    if (qu[i] < 0 || qu[i] >= n_u || qv[i] < 0 || qv[i] >= n_v) return BAD_INPUT;
  // an edge is keyed by its U end and its V end (local V id)
  auto key = [n_u](int64_t a, int64_t b) -> uint64_t {
    if (a >= n_u) std::swap(a, b);
    return (static_cast<uint64_t>(a) << 32) | static_cast<uint64_t>(b - n_u);
  };
  std::unordered_map<uint64_t, std::pair<u128, u128>> per_edge;
  std::vector<uint32_t> B1(static_cast<size_t>(g.n), 0), B2(static_cast<size_t>(g.n), 0);
  std::vector<uint8_t> seen(static_cast<size_t>(g.n), 0);
  std::vector<int32_t> touched;
  for (int64_t p = 0; p < g.n; p++) {
    for (const auto& pv : g.adj[p]) {
      if (!lower_priority(g, pv.first, p)) continue;
      for (const auto& vw : g.adj[pv.first]) {
        if (!lower_priority(g, vw.first, p)) continue;
        if (pv.second == vw.second) B1[vw.first]++; else B2[vw.first]++;
        if (!seen[vw.first]) { seen[vw.first] = 1; touched.push_back(vw.first); }
      }
    }
    for (const auto& pv : g.adj[p]) {  // second walk over the same wedges
      if (!lower_priority(g, pv.first, p)) continue;
      for (const auto& vw : g.adj[pv.first]) {
        if (!lower_priority(g, vw.first, p)) continue;
        const bool sym = pv.second == vw.second;
        const u128 same = (sym ? B1[vw.first] : B2[vw.first]) - 1;
        const u128 other = sym ? B2[vw.first] : B1[vw.first];
        for (uint64_t e : {key(p, pv.first), key(pv.first, vw.first)}) {
          auto& c = per_edge[e];
          c.first += same;
          c.second += other;
        }
      }
    }
    for (int32_t w : touched) {
      B1[w] = 0;
      B2[w] = 0;
      seen[w] = 0;
    }
    touched.clear();
  }
  const u128 lim = static_cast<u128>(UINT64_MAX);
  for (int64_t i = 0; i < k; i++) {
    const auto it = per_edge.find(key(qu[i], static_cast<int64_t>(n_u) + qv[i]));
    u128 b = 0, ub = 0;
    if (it != per_edge.end()) {
      b = it->second.first;
      ub = it->second.second;
    }
    if (b > lim || ub > lim) return OVERFLOW_64;
    bal_e[i] = static_cast<uint64_t>(b);
    unb_e[i] = static_cast<uint64_t>(ub);
  }
  return OK;
}

// Butterflies containing each queried pair by direct enumeration of Def. 1-2
// on a dense sign matrix (tiny graphs only; shares nothing with the code
// above): every butterfly adds one to each of its four edges.
int oracle_brute_force_per_edge(const int32_t* u, const int32_t* v, const int8_t* s, int64_t m, int32_t n_u,
                                int32_t n_v, const int32_t* qu, const int32_t* qv, int64_t k, uint64_t* bal_e,
                                uint64_t* unb_e) {
  if (m < 0 || n_u < 0 || n_v < 0 || k < 0) return BAD_INPUT;
  if (static_cast<int64_t>(n_u) * n_v > (int64_t{1} << 24)) return BAD_INPUT;
  const size_t cells = static_cast<size_t>(n_u) * n_v;
  std::vector<int8_t> S(cells, 0);
  for (int64_t i = 0; i < m; i++) {
    if (u[i] < 0 || u[i] >= n_u || v[i] < 0 || v[i] >= n_v) return BAD_INPUT;
    if (s[i] != 1 && s[i] != -1) return BAD_INPUT;
    S[static_cast<size_t>(u[i]) * n_v + v[i]] = s[i];
  }
  std::vector<uint64_t> B(cells, 0), UB(cells, 0);
  for (int32_t a = 0; a < n_u; a++)
    for (int32_t b = a + 1; b < n_u; b++)
      for (int32_t c = 0; c < n_v; c++)
        for (int32_t d = c + 1; d < n_v; d++) {
          const size_t cell[4] = {(size_t)a * n_v + c, (size_t)a * n_v + d, (size_t)b * n_v + c,
                                  (size_t)b * n_v + d};
          if (!S[cell[0]] || !S[cell[1]] || !S[cell[2]] || !S[cell[3]]) continue;
          const int negatives = (S[cell[0]] < 0) + (S[cell[1]] < 0) + (S[cell[2]] < 0) + (S[cell[3]] < 0);
          std::vector<uint64_t>& out = negatives % 2 == 0 ? B : UB;
          for (size_t x : cell) out[x]++;
        }
  for (int64_t i = 0; i < k; i++) {
    if (qu[i] < 0 || qu[i] >= n_u || qv[i] < 0 || qv[i] >= n_v) return BAD_INPUT;
    const size_t x = static_cast<size_t>(qu[i]) * n_v + qv[i];
    bal_e[i] = B[x];
    unb_e[i] = UB[x];
  }
  return OK;
}

// Butterflies containing each vertex by direct enumeration of Def. 1-2 on a
// dense sign matrix (tiny graphs only; shares nothing with the code above).
int oracle_brute_force_per_vertex(const int32_t* u, const int32_t* v, const int8_t* s, int64_t m, int32_t n_u,
                                  int32_t n_v, uint64_t* bal_v, uint64_t* unb_v) {
  if (m < 0 || n_u < 0 || n_v < 0) return BAD_INPUT;
  if (static_cast<int64_t>(n_u) * n_v > (int64_t{1} << 24)) return BAD_INPUT;
  std::vector<int8_t> S(static_cast<size_t>(n_u) * n_v, 0);
  for (int64_t i = 0; i < m; i++) {
    if (u[i] < 0 || u[i] >= n_u || v[i] < 0 || v[i] >= n_v) return BAD_INPUT;
    if (s[i] != 1 && s[i] != -1) return BAD_INPUT;
    S[static_cast<size_t>(u[i]) * n_v + v[i]] = s[i];
  }
  const int64_t n = static_cast<int64_t>(n_u) + n_v;
  for (int64_t x = 0; x < n; x++) bal_v[x] = unb_v[x] = 0;
  for (int32_t a = 0; a < n_u; a++)
    for (int32_t b = a + 1; b < n_u; b++)
      for (int32_t c = 0; c < n_v; c++)
        for (int32_t d = c + 1; d < n_v; d++) {
          const int8_t e[4] = {S[(size_t)a * n_v + c], S[(size_t)a * n_v + d], S[(size_t)b * n_v + c],
                               S[(size_t)b * n_v + d]};
          if (!e[0] || !e[1] || !e[2] || !e[3]) continue;
          const int negatives = (e[0] < 0) + (e[1] < 0) + (e[2] < 0) + (e[3] < 0);
          uint64_t* out = negatives % 2 == 0 ? bal_v : unb_v;
          out[a]++;
          out[b]++;
          out[n_u + c]++;
          out[n_u + d]++;
        }
  return OK;
}

// Def. 1-2 enumerated directly: a dense |U| x |V| sign matrix (later edges
// overwrite earlier ones), every pair u1 < u2 and every pair v1 < v2, parity of
// the negative edges among the four. Only for tiny graphs.
int oracle_brute_force(const int32_t* u, const int32_t* v, const int8_t* s, int64_t m, int32_t n_u, int32_t n_v,
                       uint64_t* balanced, uint64_t* unbalanced) {
  if (m < 0 || n_u < 0 || n_v < 0) return BAD_INPUT;
  if (static_cast<int64_t>(n_u) * n_v > (int64_t{1} << 26)) return BAD_INPUT;
  std::vector<int8_t> S(static_cast<size_t>(n_u) * n_v, 0);
  for (int64_t i = 0; i < m; i++) {
    if (u[i] < 0 || u[i] >= n_u || v[i] < 0 || v[i] >= n_v) return BAD_INPUT;
    if (s[i] != 1 && s[i] != -1) return BAD_INPUT;
    S[static_cast<size_t>(u[i]) * n_v + v[i]] = s[i];
  }
  uint64_t bal = 0, unb = 0;
  for (int32_t a = 0; a < n_u; a++)
    for (int32_t b = a + 1; b < n_u; b++)
      for (int32_t c = 0; c < n_v; c++) {
        int8_t ac = S[static_cast<size_t>(a) * n_v + c], bc = S[static_cast<size_t>(b) * n_v + c];
        if (!ac || !bc) continue;
        for (int32_t d = c + 1; d < n_v; d++) {
          int8_t ad = S[static_cast<size_t>(a) * n_v + d], bd = S[static_cast<size_t>(b) * n_v + d];
          if (!ad || !bd) continue;
          int negatives = (ac < 0) + (bc < 0) + (ad < 0) + (bd < 0);
          if (negatives % 2 == 0) bal++; else unb++;
        }
      }
  *balanced = bal;
  *unbalanced = unb;
  return OK;
}

// Eq. (1), Section IV-A Phase 3: W(x) = sum of d(y) over the neighbours y of x,
// for every vertex x (unified ids, after keep-latest deduplication).
int oracle_workload_eq1(const int32_t* u, const int32_t* v, const int8_t* s, int64_t m, int32_t n_u, int32_t n_v,
                        uint64_t* W) {
  SignedGraph g;
  int rc = build_graph(u, v, s, m, n_u, n_v, g);
  if (rc != OK) return rc;
  for (int64_t x = 0; x < g.n; x++) {
    uint64_t acc = 0;
    for (const auto& y : g.adj[x]) acc += static_cast<uint64_t>(g.deg[y.first]);
    W[x] = acc;
  }
  return OK;
}

// Phase 3 greedy bin packing (Section IV-A, Example 2): take the items in
// descending workload order and give each to the bin with the smallest load so
// far (lowest bin index on ties). Writes the bin of every item and the loads.
int oracle_lpt(const uint64_t* work, int64_t n_items, int32_t n_bins, int32_t* bin_of, uint64_t* loads) {
  if (n_items < 0 || n_bins <= 0) return BAD_INPUT;
  std::vector<int64_t> order(static_cast<size_t>(n_items));
  for (int64_t i = 0; i < n_items; i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return work[a] > work[b]; });
  for (int32_t b = 0; b < n_bins; b++) loads[b] = 0;
  for (int64_t i : order) {
    int32_t best = 0;
    for (int32_t b = 1; b < n_bins; b++)
      if (loads[b] < loads[best]) best = b;
    bin_of[i] = best;
    loads[best] += work[i];
  }
  return OK;
}

}  // extern "C"
