// Device building blocks shared by the single-graph kernels (count.cu) and
// the batched kernels (batch.cu): packed wedge counters, the incremental
// Lemma 1 contribution, shared-memory hashing, the warp walk over a pivot's
// lower neighbours, and one window of the hub sweep.
#pragma once

#include "internal.h"
#include "common.cuh"

namespace dbbc {

// One packed increment: symmetric wedge -> +1, asymmetric -> +2^32.
__device__ __forceinline__ unsigned long long wedge_inc(uint32_t x, uint32_t s1) {
  return ((x ^ s1) & 1u) ? (1ull << 32) : 1ull;
}

// Lemma 1 contribution of one wedge, from its endpoint counter just before the
// increment (sym = p, asym = q): adding a symmetric wedge to (p, q) closes p
// new balanced pairs (C(p+1,2) - C(p,2) = p) and q unbalanced ones ((p+1)q - pq);
// an asymmetric wedge closes q balanced and p unbalanced ones. Summed over all
// wedges this equals C(p,2) + C(q,2) and p*q per endpoint.
__device__ __forceinline__ void wedge_contrib(unsigned long long old, unsigned long long inc, uint64_t& bal,
                                              uint64_t& unb) {
  const uint64_t p = old & 0xFFFFFFFFull, q = old >> 32;
  const bool sym = inc == 1ull;
  bal += sym ? p : q;
  unb += sym ? q : p;
}

__device__ __forceinline__ uint32_t hash_slot(uint32_t w, int log_h) {
  return (w * 2654435769u) >> (32 - log_h);
}

// Find or insert endpoint w in a shared table of 2^log_h slots and add inc;
// returns the counter's previous value through *old. Returns false if the
// probe sequence ran past the table (cannot happen when the table has more
// slots than the pivot's accepted wedges).
__device__ __forceinline__ bool smem_hash_add(uint32_t* keys, unsigned long long* vals, int log_h, uint32_t w,
                                              unsigned long long inc, unsigned long long* old) {
  const uint32_t mask = (1u << log_h) - 1u;
  uint32_t h = hash_slot(w, log_h);
  for (uint32_t probe = 0; probe <= mask; probe++) {
    uint32_t cur = *reinterpret_cast<volatile uint32_t*>(&keys[h]);
    if (cur == kEmptyKey) cur = atomicCAS(&keys[h], kEmptyKey, w);
    if (cur == kEmptyKey || cur == w) {
      *old = atomicAdd(&vals[h], inc);
      return true;
    }
    h = (h + 1u) & mask;
  }
  return false;
}

// Smallest 2^k >= (work << mult_log) slots (at least 32, at most 2^max_log).
// The tiers keep work <= 2^(max_log - 1), so a table always has more slots
// than the pivot has accepted wedges (and hence distinct endpoints).
__device__ __forceinline__ int table_log(uint64_t work, int max_log, int mult_log) {
  int k = 5;
  while (k < max_log && (1ull << k) < (work << mult_log)) k++;
  return k;
}

struct PivotGeom {
  int64_t rb;    // row start of the pivot
  uint32_t L;    // lower neighbours
  uint32_t lim;  // entries x < lim are accepted endpoints: (side_rank(p) << 1)
  int64_t base;  // first row of the other side
};

__device__ __forceinline__ PivotGeom pivot_geom(const CsrView& g, int32_t p) {
  PivotGeom q;
  const bool ok = DBBC_CHECK(p >= 0 && p < g.n);  // checked builds: a bad pivot walks no neighbour
  if (!ok) p = 0;
  q.rb = g.row_ptr[p];
  q.L = ok ? g.lower[p] : 0u;
#if DBBC_CHECKED
  if (q.L && !DBBC_CHECK(q.rb >= 0 && q.rb + q.L <= g.row_ptr[p + 1] && g.row_ptr[p + 1] <= g.nnz)) q.L = 0;
#endif
  const bool is_u = p < g.n_u;
  q.lim = (is_u ? (uint32_t)p : (uint32_t)(p - g.n_u)) << 1;
  q.base = is_u ? (int64_t)g.n_u : 0;
  return q;
}

// Row [b, en) of the vertex of the other side named by the CSR entry e of a
// pivot with geometry q, and the sign bit of their edge. Checked builds test
// the row index and bounds; a failed test gives an empty row.
__device__ __forceinline__ uint32_t neighbour_row(const CsrView& g, const PivotGeom& q, uint32_t e, int64_t& b,
                                                  int64_t& en) {
  const int64_t vrow = q.base + (e >> 1);
  if (DBBC_CHECK(vrow >= 0 && vrow < g.n)) {
    b = g.row_ptr[vrow];
    en = g.row_ptr[vrow + 1];
    if (!DBBC_CHECK(b >= 0 && b <= en && en <= g.nnz)) en = b;
  } else {
    b = en = 0;
  }
  return e & 1u;
}

// The warp walks lower-neighbour positions [a, b) of the pivot in groups of
// 32 (`step` = distance between this warp's groups) and, for each lower
// neighbour v, the accepted prefix of v's row in chunks of 32 * U entries.
// visit(x[U], s1) is called by all lanes together; lane l holds entries
// chunk + u*32 + l, with x = 0xFFFFFFFF where nothing is accepted.
template <int U, typename Visit>
__device__ __forceinline__ void warp_walk(const CsrView& g, const PivotGeom& q, uint32_t a, uint32_t b,
                                          uint32_t step, Visit&& visit) {
  const unsigned lane = lane_id();
  for (uint32_t i0 = a; i0 < b; i0 += step) {
    uint32_t e = 0;
    int64_t vb = 0, ve = 0;
    if (i0 + lane < b) {
      e = g.col[q.rb + i0 + lane];
      neighbour_row(g, q, e, vb, ve);
    }
    const uint32_t cnt = min(32u, b - i0);
    for (uint32_t k = 0; k < cnt; k++) {
      const uint32_t s1 = __shfl_sync(kFullMask, e, k) & 1u;
      const int64_t jb0 = __shfl_sync(kFullMask, vb, k);
      const int64_t je = __shfl_sync(kFullMask, ve, k);
      for (int64_t jb = jb0; jb < je; jb += 32 * U) {
        uint32_t x[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int64_t j = jb + u * 32 + lane;
          x[u] = j < je ? g.col[j] : 0xFFFFFFFFu;
        }
        bool stop = false;
#pragma unroll
        for (int u = 0; u < U; u++) {
          if (x[u] >= q.lim) {
            x[u] = 0xFFFFFFFFu;
            stop = true;
          }
        }
        visit(x, s1);
        if (__any_sync(kFullMask, stop)) break;  // rows ascend: nothing accepted beyond
      }
    }
  }
}

template <int G>
__device__ __forceinline__ unsigned group_mask() {
  const unsigned lane = lane_id();
  return G == 32 ? kFullMask : (((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));
}

// Hash tiers: groups of G lanes (group gid of `groups`) take lower neighbours
// gid, gid + groups, ... of the pivot; a group walks its neighbour's accepted
// prefix G entries at a time and adds every wedge to the shared hash table,
// accumulating the Lemma 1 contributions. The next neighbour's row bounds are
// loaded while the current one is walked. Returns false if the table ran out
// of slots. G is chosen from the pivot's mean accepted segment (work / L) so
// that short segments do not leave most lanes of a warp idle.
template <int G>
__device__ __forceinline__ bool hash_walk(uint32_t gid, uint32_t groups, const CsrView& g, const PivotGeom& q,
                                          uint32_t* keys, unsigned long long* vals, int log_h, uint64_t& bal,
                                          uint64_t& unb) {
  const int gl = threadIdx.x & (G - 1);
  const unsigned gmask = group_mask<G>();
  bool fits = true;
  int64_t b_nx = 0, en_nx = 0;
  uint32_t s1_nx = 0;
  if (gid < q.L) s1_nx = neighbour_row(g, q, g.col[q.rb + gid], b_nx, en_nx);
  for (uint32_t i = gid; i < q.L; i += groups) {
    const int64_t b = b_nx, en = en_nx;
    const uint32_t s1 = s1_nx;
    if (i + groups < q.L) s1_nx = neighbour_row(g, q, g.col[q.rb + i + groups], b_nx, en_nx);
    for (int64_t c = b; c < en; c += G) {
      const int64_t j = c + gl;
      const uint32_t x = j < en ? g.col[j] : 0xFFFFFFFFu;
      const bool ok = x < q.lim;
      if (ok) {
        const unsigned long long inc = wedge_inc(x, s1);
        unsigned long long old;
        if (smem_hash_add(keys, vals, log_h, x >> 1, inc, &old)) wedge_contrib(old, inc, bal, unb);
        else fits = false;
      }
      if (__ballot_sync(gmask, !ok)) break;  // rows ascend: nothing accepted beyond
    }
  }
  return fits;
}

// log2 of the lanes per neighbour for a pivot whose lower neighbours carry
// `work` accepted wedges in all (at least 4 lanes, at most `max_log`).
__device__ __forceinline__ int hash_group_log(uint64_t work, uint32_t L, int max_log) {
  const uint64_t mean = work / (L ? L : 1);
  const int lg = mean >= 24 ? 5 : mean >= 12 ? 4 : mean >= 6 ? 3 : 2;
  return lg < max_log ? lg : max_log;
}

template <typename... A>
__device__ __forceinline__ bool hash_walk_dispatch(int group_log, uint32_t tid, uint32_t threads, A&&... a) {
  switch (group_log) {
    case 2: return hash_walk<4>(tid >> 2, threads >> 2, a...);
    case 3: return hash_walk<8>(tid >> 3, threads >> 3, a...);
    case 4: return hash_walk<16>(tid >> 4, threads >> 4, a...);
    default: return hash_walk<32>(tid >> 5, threads >> 5, a...);
  }
}

// log2 of the hash slots a tier's tables need at most: table_log of the
// tier's largest accepted-wedge count (5..cap). Kernels of a tier get this
// many slots per table, so small tiers leave room for more CTAs per SM.
inline int tier_slots_log(uint64_t max_work, int mult_log, int cap) {
  int k = 5;
  while (k < cap && (1ull << k) < (max_work << mult_log)) k++;
  return k;
}

constexpr int kLightWarps = 8;

constexpr int kMediumThreads = 256;
constexpr int kMediumWarps = kMediumThreads / 32;

// ------------------------------------------------------------------ hub tier
// Window sweep. A hub pivot's accepted endpoints [0, side_rank(p)) are cut
// into windows of kSweepWindow16 (or kSweepWindow32) consecutive side ranks. A
// work item is one hub and a span of its windows, owned by one CTA, so the
// counts of every endpoint in a window are complete inside that CTA: they live
// in shared memory, and the Lemma 1 contributions come from the value each
// atomic returns. Each lower neighbour v keeps a cursor into its row (uint32
// positions: a CSR has fewer than 2^32 entries); rows ascend, so sweeping the
// windows in order moves every cursor forward only. Counters pack
// (asym << 16) | sym when the hub has fewer than 2^16 lower neighbours (no
// count can exceed that), else (asym << 32) | sym.
constexpr int kSweepThreads = DBBC_SWEEP_THREADS;
constexpr int kSweepUnroll = DBBC_SWEEP_UNROLL;
static_assert(kSweepWindow16 % 4 == 0, "window buffers are cleared 16 bytes at a time");

// Clear the first `words` 32-bit words of a window (16 bytes per store; the
// window buffer holds a multiple of 4 words).
template <int THREADS = kSweepThreads>
__device__ __forceinline__ void zero_words(uint32_t* w, uint32_t words) {
  uint4* q = reinterpret_cast<uint4*>(w);
  const uint32_t quads = (words + 3) >> 2;
  for (uint32_t j = threadIdx.x; j < quads; j += THREADS) q[j] = make_uint4(0u, 0u, 0u, 0u);
}

// x[u] = entry at position c + u*G + gl of a row ending at en, or ~0 past it.
template <int G>
__device__ __forceinline__ void load_chunk(const uint32_t* col, uint32_t c, uint32_t en, int gl,
                                           uint32_t (&x)[kSweepUnroll]) {
#pragma unroll
  for (int u = 0; u < kSweepUnroll; u++) {
    const uint32_t off = (uint32_t)(u * G + gl);
    x[u] = en - c > off ? __ldg(col + c + off) : 0xFFFFFFFFu;
  }
}

// Counter widths of a window. CW = 16: one 32-bit word per endpoint packing
// (asym << 16) | sym, kSweepWindow16 ranks per window. CW = 8: two endpoints
// per 32-bit word, each (asym << 8) | sym, twice the ranks per window; used
// where every endpoint has degree < 256 or the hub has fewer than 256 lower
// neighbours (a count never exceeds either). CW = 4: four endpoints per word,
// each (asym << 4) | sym, four times the ranks, where counts stay below 16.
// CW = 32: one 64-bit word per endpoint, half the ranks.
template <int CW>
__host__ __device__ constexpr uint32_t window_ranks() {
  return CW == 4 ? 4 * kSweepWindow16 : CW == 8 ? 2 * kSweepWindow16 : CW == 16 ? kSweepWindow16 : kSweepWindow32;
}

template <int CW>
__device__ __forceinline__ uint32_t window_words(uint32_t ranks) {  // 32-bit words holding `ranks` counters
  return CW == 8 ? (ranks + 1) >> 1 : CW == 16 ? ranks : 2 * ranks;
}

// The windows of a work item: quarter ones over [lo, qe), tiny ones over
// [qe, te), narrow ones over [te, ne), wide ones over [ne, hi), numbered in
// rank order. `quarter` false folds the quarter part into the tiny one (for
// sweeps that have no 4-bit counters).
struct ItemWindows {
  uint32_t lo, qe, te, ne, hi;
  uint32_t rq, rt, rn, rw;
  ItemWindows() = default;
  __device__ __forceinline__ explicit ItemWindows(const SweepItem& it, bool quarter = true) {
    lo = it.lo;
    hi = it.hi;
    qe = quarter ? min(max(it.q_end, lo), hi) : lo;
    te = min(max(it.t_end, qe), hi);
    ne = min(max(it.n_end, te), hi);
    rq = (qe - lo + window_ranks<4>() - 1) / window_ranks<4>();
    rt = (te - qe + window_ranks<8>() - 1) / window_ranks<8>();
    rn = (ne - te + window_ranks<16>() - 1) / window_ranks<16>();
    rw = (hi - ne + window_ranks<32>() - 1) / window_ranks<32>();
  }
  __device__ __forceinline__ uint32_t count() const { return rq + rt + rn + rw; }
  // window r: its ranks [wlo, whi) and counter width
  __device__ __forceinline__ void window(uint32_t r, uint32_t& wlo, uint32_t& whi, int& cw) const {
    if (r < rq) {
      wlo = lo + r * window_ranks<4>();
      whi = min(wlo + window_ranks<4>(), qe);
      cw = 4;
    } else if (r < rq + rt) {
      wlo = qe + (r - rq) * window_ranks<8>();
      whi = min(wlo + window_ranks<8>(), te);
      cw = 8;
    } else if (r < rq + rt + rn) {
      wlo = te + (r - rq - rt) * window_ranks<16>();
      whi = min(wlo + window_ranks<16>(), ne);
      cw = 16;
    } else {
      wlo = ne + (r - rq - rt - rn) * window_ranks<32>();
      whi = min(wlo + window_ranks<32>(), hi);
      cw = 32;
    }
  }
  // the window holding rank x (lo <= x < hi)
  __device__ __forceinline__ uint32_t index_of(uint32_t x) const {
    if (x < qe) return (x - lo) / window_ranks<4>();
    if (x < te) return rq + (x - qe) / window_ranks<8>();
    if (x < ne) return rq + rt + (x - te) / window_ranks<16>();
    return rq + rt + rn + (x - ne) / window_ranks<32>();
  }
};

// Add one wedge (endpoint counter k, asym = the two edge signs differ) when
// `ok`, and accumulate its Lemma 1 contribution from the counter's old value:
// the old count of the wedge's own class (B1 for a symmetric wedge, B2 for an
// asymmetric one) closes balanced butterflies and the other class unbalanced
// ones. Packed counters are rotated for an asymmetric wedge so that its own
// class sits in the low half. Narrow widths sum into 32-bit accumulators (a
// segment adds fewer than 2^32 to each); the 64-bit width adds directly.
template <int CW>
__device__ __forceinline__ void add_wedge(bool ok, uint32_t k, uint32_t asym, uint32_t* c16, unsigned long long* c32,
                                          uint32_t& acc_same, uint32_t& acc_other, uint64_t& bal, uint64_t& unb) {
  if (ok && !DBBC_CHECK(k < window_ranks<CW>())) ok = false;
  if (CW == 8) {
    const uint32_t wsh = (k & 1u) << 4;  // which half of the word
    uint32_t old = 0;
    if (ok) old = atomicAdd(&c16[k >> 1], (asym ? 0x100u : 1u) << wsh);
    const uint32_t v = (old >> wsh) & 0xFFFFu;            // (asym << 8) | sym
    const uint32_t r = ((v << 16) | v) >> (asym << 3);  // own class in the low byte
    acc_same += r & 0xFFu;
    acc_other += (r >> 8) & 0xFFu;
  } else if (CW == 16) {
    const uint32_t sh = asym << 4;
    uint32_t old = 0;
    if (ok) old = atomicAdd(&c16[k], 1u << sh);
    const uint32_t v = __funnelshift_l(old, old, sh);  // (other class << 16) | own class
    acc_same += v & 0xFFFFu;
    acc_other += v >> 16;
  } else {
    const unsigned long long inc = asym ? (1ull << 32) : 1ull;
    unsigned long long old = 0;
    if (ok) old = atomicAdd(&c32[k], inc);
    wedge_contrib(old, inc, bal, unb);  // adds nothing when old == 0
  }
}

// A group of G lanes walks one neighbour's entries inside the window [lo,
// hl >> 1) from cursor c (the first chunk already in x) and returns the cursor
// past the window. Entries of the window are a prefix of what is left of the
// row, so the group stops at the first chunk that is not full. All groups of a
// warp run the loop in lockstep until the last of them is done (warp-wide
// votes, the atomic the only predicated step), which keeps the warp converged;
// a group that is not `active` (no neighbour) only votes. Contributions of
// the narrow widths are summed per segment in 32 bits (add_wedge).
template <int G, int CW>
__device__ __forceinline__ uint32_t walk_segment(const uint32_t* col, uint32_t c, uint32_t en, uint32_t s1,
                                                 uint32_t (&x)[kSweepUnroll], uint32_t lo2, uint32_t hl, int gl,
                                                 bool active, uint32_t* c16, unsigned long long* c32,
                                                 uint64_t& bal, uint64_t& unb) {
  const unsigned gshift = lane_id() & ~(unsigned)(G - 1);
  const unsigned gbits = G == 32 ? kFullMask : (1u << G) - 1u;
  uint32_t acc_same = 0, acc_other = 0;
  for (;;) {
    int n_ok = 0;
#pragma unroll
    for (int u = 0; u < kSweepUnroll; u++) {
      const bool ok = active && x[u] < hl;
      const uint32_t asym = (x[u] ^ s1) & 1u;
      const uint32_t k = (x[u] - lo2) >> 1;
      add_wedge<CW>(ok, k, asym, c16, c32, acc_same, acc_other, bal, unb);
      n_ok += __popc((__ballot_sync(kFullMask, ok) >> gshift) & gbits);
    }
    c += (uint32_t)n_ok;
    active = active && n_ok == G * kSweepUnroll;
    if (!__any_sync(kFullMask, active)) break;
    if (active) load_chunk<G>(col, c, en, gl, x);
  }
  bal += acc_same;
  unb += acc_other;
  return c;
}

// Cursors of an item: the first entry of each lower neighbour's row at or
// after rank `lo_rank`, and the row end.
__device__ __forceinline__ void init_cursor(const CsrView& g, const PivotGeom& q, uint32_t i, uint32_t lo_rank,
                                            uint32_t* cur, uint32_t& b_out, uint32_t& en_out) {
  int64_t b, en;
  neighbour_row(g, q, g.col[q.rb + i], b, en);
  const uint32_t first = lo_rank << 1;
  if (first) {  // lower_bound of `first` in the row
    int64_t lo = b, hi = en;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (g.col[mid] < first) lo = mid + 1; else hi = mid;
    }
    b = lo;
  }
  b_out = (uint32_t)b;
  en_out = (uint32_t)en;
  cur[2 * i] = b_out;
  cur[2 * i + 1] = en_out;
}

inline int blocks_per_sm(const void* fn, int threads, size_t smem) {
  int b = 0;
  DBBC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem));
  return b > 0 ? b : 1;
}

inline int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    DBBC_CUDA(cudaGetDevice(&dev));
    DBBC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (sms <= 0) sms = kNumSMs;
  }
  return sms;
}

}  // namespace dbbc
