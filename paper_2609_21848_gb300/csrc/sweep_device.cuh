// The hub tier's window sweep (Algorithm 1, Phase 5, for pivots with many
// accepted wedges): the inner loop shared by the single-graph and batched
// sweep kernels.
//
// A work item is one hub pivot and a span of its endpoint ranks, owned by one
// CTA; the span is cut into windows whose counters fill the CTA's shared
// memory (see ItemWindows in count_device.cuh for the 8/16/32-bit counter
// widths). Every lower neighbour v of the hub keeps a cursor into its row;
// rows ascend by rank, so the entries of v inside a window are the next run of
// its row and the cursor only moves forward across windows.
//
// Per entry the walk does one compare, the counter's shared address, the
// packed increment and one predicated shared-memory atomic; the segment end is
// detected once per chunk (the group's last entry), and the next chunk is
// loaded before the current one is counted. Lemma 1 is applied in one of two
// ways, chosen per item by its wedges per window:
//
//   * per wedge (RET): the atomic returns the endpoint's counter before the
//     increment, and a symmetric wedge that raises (p, q) to (p + 1, q) closes
//     p balanced and q unbalanced butterflies (an asymmetric one q and p);
//   * per window (FIN): the atomics return nothing, and when the window is
//     cleared every endpoint adds C(p,2) + C(q,2) balanced and p * q unbalanced
//     butterflies from its final counter. This is the paper's finalisation over
//     the touched endpoints, done for the whole window at once.
#pragma once

#include "count_device.cuh"

namespace dbbc {

// entries per lane per chunk (3 measured best on GB300: 2, 4 and 8 were 1-9%
// slower), and neighbours a lane group starts together
#ifndef DBBC_LEAN_UNROLL
#define DBBC_LEAN_UNROLL 3
#endif
#ifndef DBBC_LEAN_BATCH
#define DBBC_LEAN_BATCH 1
#endif
constexpr int kLU = DBBC_LEAN_UNROLL;
constexpr int kLB = DBBC_LEAN_BATCH;

// Shared counters of the sweep: one window, plus one word so that a window of
// 4-bit (8-bit) counters may start at the multiple of 4 (even rank) below its
// first rank.
constexpr uint32_t kSweepWords = kSweepWindow16 + 4;
constexpr size_t kSweepSmem = (size_t)kSweepWords * 4;

// A window of side ranks [wlo, whi): entries below h lie in it (cursors start
// at its first rank), and the counter word of rank r is at shared byte address
// wb + (r >> 2) * 4 (4-bit counters, four ranks per word, aligned to a
// multiple of 4), wb + (r >> 1) * 4 (8-bit counters, two ranks per word,
// aligned to an even rank), wb + r * 4 (16-bit) or wb + r * 8 (32-bit).
struct Win {
  uint32_t h;
  uint32_t wb;
  uint32_t words;  // 32-bit words in use
#if DBBC_CHECKED
  uint32_t l;             // wlo << 1: no entry below it may be counted
  uint32_t s_lo, s_hi;    // the counter buffer's shared byte addresses [s_lo, s_hi)
#endif
};

// WORDS: the counter buffer's size in 32-bit words.
template <uint32_t WORDS = kSweepWords>
__device__ __forceinline__ Win make_win(int cw, uint32_t wlo, uint32_t whi, uint32_t sbase) {
  Win w;
  w.h = whi << 1;
#if DBBC_CHECKED
  w.l = wlo << 1;
  w.s_lo = sbase;
  w.s_hi = sbase + WORDS * 4u;
#endif
  if (cw == 4) {
    const uint32_t l4 = wlo & ~3u;
    w.wb = sbase - l4;
    w.words = (whi - l4 + 3u) >> 2;
  } else if (cw == 8) {
    const uint32_t l2 = wlo & ~1u;
    w.wb = sbase - l2 * 2u;
    w.words = (whi - l2 + 1u) >> 1;
  } else if (cw == 16) {
    w.wb = sbase - wlo * 4u;
    w.words = whi - wlo;
  } else {
    w.wb = sbase - wlo * 8u;
    w.words = 2u * (whi - wlo);
  }
  if (!DBBC_CHECK(wlo <= whi && w.words <= WORDS)) {  // checked builds: count nothing in it
    w.h = 0u;
    w.words = 0u;
  }
  return w;
}

// Shared-memory atomics on 32-bit shared addresses, taken only when x < h.
__device__ __forceinline__ void red_if_u32(uint32_t x, uint32_t h, uint32_t addr, uint32_t v) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %0, %1;\n\t@p red.shared.add.u32 [%2], %3;\n\t}"
               :: "r"(x), "r"(h), "r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_if_u32(uint32_t x, uint32_t h, uint32_t addr, uint32_t v) {
  uint32_t old;
  asm volatile("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\tmov.u32 %0, 0;\n\t@p atom.shared.add.u32 %0, [%3], %4;\n\t}"
               : "=r"(old) : "r"(x), "r"(h), "r"(addr), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_if_u64(uint32_t x, uint32_t h, uint32_t addr, uint64_t v) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %0, %1;\n\t@p red.shared.add.u64 [%2], %3;\n\t}"
               :: "r"(x), "r"(h), "r"(addr), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t atom_if_u64(uint32_t x, uint32_t h, uint32_t addr, uint64_t v) {
  uint64_t old;
  asm volatile("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\tmov.u64 %0, 0;\n\t@p atom.shared.add.u64 %0, [%3], %4;\n\t}"
               : "=l"(old) : "r"(x), "r"(h), "r"(addr), "l"(v) : "memory");
  return old;
}

// Count one entry x (a CSR entry (side_rank << 1) | negative) of a neighbour
// whose edge to the hub has sign bit s1, if x < h. The wedge is symmetric when
// the two sign bits agree (bucket B1 of Algorithm 1, the low half of the
// packed counter) and asymmetric otherwise (B2, the high half). With RET the
// counter's old value gives the Lemma 1 contribution: rotated so that the
// wedge's own class is in the low half, it is summed into a_lo (own + other
// << 16, mod 2^32) and a_hi (other); the 64-bit width adds to bal / unb.
// Checked builds skip an entry below the window or whose counter address
// leaves the buffer.
template <int CW, bool RET>
__device__ __forceinline__ void lean_add(uint32_t x, uint32_t h, uint32_t s1, const Win& w, uint32_t& a_lo,
                                         uint32_t& a_hi, uint64_t& bal, uint64_t& unb) {
  const uint32_t wb = w.wb;
#if DBBC_CHECKED
  if (x < h) {
    const uint32_t addr = CW == 4 ? wb + ((x >> 1) & ~3u) : CW == 8 ? wb + (x & ~3u)
                        : CW == 16 ? wb + ((x >> 1) << 2) : wb + ((x >> 1) << 3);
    if (!DBBC_CHECK(x >= w.l && addr >= w.s_lo && addr + (CW == 32 ? 8u : 4u) <= w.s_hi)) h = 0u;
  }
#endif
  if constexpr (CW == 4) {
    // nibble (2 * (rank & 3) + asym) of the word: byte k = (asym_k << 4) | sym_k
    const uint32_t sel = (x ^ s1) & 7u;
    const uint32_t addr = wb + ((x >> 1) & ~3u);
    const uint32_t inc = 1u << (sel << 2);
    if constexpr (!RET) {
      red_if_u32(x, h, addr, inc);
    } else {
      const uint32_t old = atom_if_u32(x, h, addr, inc);
      const uint32_t own = (old >> (sel << 2)) & 0xFu, other = (old >> ((sel ^ 1u) << 2)) & 0xFu;
      a_lo += own | (other << 16);
      a_hi += other;
    }
  } else if constexpr (CW == 8) {
    // byte (2 * (rank & 1) + asym) of the word: (asym1, sym1, asym0, sym0)
    const uint32_t sel = (x ^ s1) & 3u;
    const uint32_t addr = wb + (x & ~3u);
    const uint32_t inc = 1u << (sel << 3);
    if constexpr (!RET) {
      red_if_u32(x, h, addr, inc);
    } else {
      const uint32_t old = atom_if_u32(x, h, addr, inc);
      // own class byte to byte 0, the other class to byte 2
      const uint32_t v = __byte_perm(old, 0u, (sel * 0x101u) ^ 0x4140u);
      a_lo += v;
      a_hi += v >> 16;
    }
  } else if constexpr (CW == 16) {
    const uint32_t asym = (x ^ s1) & 1u;
    const uint32_t addr = wb + ((x >> 1) << 2);
    const uint32_t inc = 1u + asym * 0xFFFFu;
    if constexpr (!RET) {
      red_if_u32(x, h, addr, inc);
    } else {
      const uint32_t old = atom_if_u32(x, h, addr, inc);
      const uint32_t v = __funnelshift_l(old, old, asym << 4);
      a_lo += v;
      a_hi += v >> 16;
    }
  } else {
    const uint32_t asym = (x ^ s1) & 1u;
    const uint32_t addr = wb + ((x >> 1) << 3);
    const uint64_t inc = asym ? (1ull << 32) : 1ull;
    if constexpr (!RET) {
      red_if_u64(x, h, addr, inc);
    } else {
      const uint64_t old = atom_if_u64(x, h, addr, inc);
      const uint64_t p = old & 0xFFFFFFFFull, q = old >> 32;
      bal += asym ? q : p;
      unb += asym ? p : q;
    }
  }
}

// x[u] = the entry at position c + u*G + gl of a row ending at en, or ~0 past
// the end (en >= c).
template <int G>
__device__ __forceinline__ void lean_load(const uint32_t* __restrict__ col, uint32_t c, uint32_t en, int gl,
                                          uint32_t (&x)[kLU]) {
  const uint32_t rem = en - c;
  const uint32_t* p = col + c + (uint32_t)gl;
#pragma unroll
  for (int u = 0; u < kLU; u++) x[u] = (uint32_t)(u * G + gl) < rem ? __ldg(p + u * G) : 0xFFFFFFFFu;
}

// A group of G lanes walks one neighbour's entries inside window w from
// cursor c (row end en, first chunk already in x) and returns the cursor past
// the window; x_next gets the neighbour's first entry past the window (~0 at
// the end of its row). All groups of the warp run the loop in lockstep until
// the last of them is done: the loop's only exit follows a warp-wide vote, so
// every shuffle and vote in it is reached by the whole warp. A group that is
// not `active` (no neighbour) only votes.
template <int G, int CW, bool RET>
__device__ __forceinline__ uint32_t lean_walk(const uint32_t* __restrict__ col, uint32_t c, uint32_t en, uint32_t s1,
                                              uint32_t (&x)[kLU], const Win& w, int gl, bool active, uint64_t& bal,
                                              uint64_t& unb, uint32_t& x_next) {
  const unsigned lane = lane_id();
  const unsigned gbase = lane & ~(unsigned)(G - 1);
  uint32_t h = active ? w.h : 0u;
  uint32_t a_lo = 0, a_hi = 0;
  for (;;) {
    // the chunk lies wholly inside the window iff its last entry does
    uint32_t xl = x[kLU - 1];
    if constexpr (G > 1) xl = __shfl_sync(kFullMask, xl, gbase + (G - 1));
    const bool cont = xl < h;
    uint32_t y[kLU];
    const uint32_t cn = c + (uint32_t)(G * kLU);
    lean_load<G>(col, cn, cont ? en : cn, gl, y);  // the next chunk, while this one is counted
#pragma unroll
    for (int u = 0; u < kLU; u++) lean_add<CW, RET>(x[u], h, s1, w, a_lo, a_hi, bal, unb);
    if (!__any_sync(kFullMask, cont)) break;
    if (cont) {
      c = cn;
#pragma unroll
      for (int u = 0; u < kLU; u++) x[u] = y[u];
    } else {
      h = 0u;  // done: keep its last chunk in x, count nothing more
    }
  }
  // the accepted entries of the group's last chunk are a prefix of it
  uint32_t n_ok = 0;
#pragma unroll
  for (int u = 0; u < kLU; u++) {
    const unsigned b = __ballot_sync(kFullMask, x[u] < w.h);
    n_ok += G == 32 ? __popc(b) : __popc((b >> gbase) & ((1u << G) - 1u));
  }
  const uint32_t ui = n_ok / G;
  uint32_t t = x[0];
#pragma unroll
  for (int u = 1; u < kLU; u++) t = ui == (uint32_t)u ? x[u] : t;
  x_next = G == 1 ? t : __shfl_sync(kFullMask, t, gbase + (n_ok & (G - 1)));
  if constexpr (RET && CW != 32) {
    // a_lo = own + (other << 16) mod 2^32; the own-class sum of one segment
    // stays below 2^32 (at most 57,344 entries of counts < 2^16, 114,688 of
    // counts < 2^8 or 229,376 of counts < 2^4)
    bal += a_lo - (a_hi << 16);
    unb += a_hi;
  }
  return c + n_ok;
}

// Neighbour slots: one uint2 per lower neighbour,
// {position, (entries left in its row) | (sign bit of the hub's edge to it) << 31}.
// Cursor mode keeps one per lower neighbour of the item; list mode keeps the
// same slots in per-window lists.
__device__ __forceinline__ void lean_cursor_start(const CsrView& g, const PivotGeom& q, uint32_t i, uint32_t lo_rank,
                                                  uint32_t& b_out, uint32_t& en_out, uint32_t& s1_out) {
  int64_t b, en;
  s1_out = neighbour_row(g, q, g.col[q.rb + i], b, en);
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
}

__device__ __forceinline__ uint2 lean_slot(uint32_t c, uint32_t en, uint32_t s1) {
  return make_uint2(c, (en - c) | (s1 << 31));
}

// Block-uniform state of the list-mode item being swept, kept in shared
// memory (it would otherwise occupy registers the walk needs). In list mode a
// neighbour is visited only in the windows that hold its entries: window r
// of the current span has a list (global memory, L slots) of the neighbours
// whose next entry falls in it; after walking its entries in window r, a
// neighbour is appended to the list of the window of its next entry (always
// a later window), to the overflow list if that entry lies in a later span of
// the item, or to no list at the end of its row or of the item. A neighbour is
// in at most one list at a time and in each list at most once, so L slots
// per list never overflow.
struct ListState {
  uint2* lists;                // [Rsub][L] window lists of the span
  uint2* over;                 // [L] neighbours waiting for the next span
  int cnt[kListMaxWindows];    // list lengths
  int ocnt;                    // overflow list length
  uint32_t L;
  uint32_t nwin;               // windows (lists) of the span
  ItemWindows iw;              // the item's windows
  uint32_t s0;                 // first window of the span
  uint32_t hl;                 // (last rank of the span + 1) << 1
  uint32_t item_hl;            // (last rank of the item + 1) << 1
};

// Queue a neighbour whose cursor c (row end en, edge sign s1) stopped at entry
// x (see ListState).
__device__ __forceinline__ void list_queue(ListState& ls, uint32_t x, uint32_t c, uint32_t en, uint32_t s1) {
  const uint2 slot = lean_slot(c, en, s1);
  if (x < ls.hl) {
    const uint32_t r = ls.iw.index_of(x >> 1) - ls.s0;
    if (!DBBC_CHECK(r < ls.nwin)) return;
    const int pos = atomicAdd(&ls.cnt[r], 1);
    if (DBBC_CHECK((uint32_t)pos < ls.L)) ls.lists[(size_t)r * ls.L + (uint32_t)pos] = slot;
  } else if (x < ls.item_hl) {
    const int pos = atomicAdd(&ls.ocnt, 1);
    if (DBBC_CHECK((uint32_t)pos < ls.L)) ls.over[pos] = slot;
  }
}

// The neighbours a warp starts together: its groups of G lanes take slots
// base + group, base + group + 32/G, ... (kLB each) of a slot array, with the
// slots and the first chunk of each segment loaded. `base` is handed out
// through a shared counter, so warps that finish early take more.
struct LaneBatch {
  uint32_t base;
  uint32_t c[kLB], en[kLB], s1[kLB];
  uint32_t x[kLB][kLU];
};

template <int G>
__device__ __forceinline__ void batch_fetch(const uint32_t* __restrict__ col, const uint2* slots, uint32_t n,
                                            uint32_t* next, LaneBatch& b) {
  const int gl = threadIdx.x & (G - 1);
  const uint32_t gw = lane_id() / G;
  constexpr uint32_t gpw = 32 / G;
  uint32_t base = 0;
  if (lane_id() == 0) base = atomicAdd(next, gpw * (uint32_t)kLB);
  b.base = __shfl_sync(kFullMask, base, 0);
#pragma unroll
  for (int k = 0; k < kLB; k++) {
    const uint32_t i = b.base + gw + k * gpw;
    b.c[k] = b.en[k] = b.s1[k] = 0;
    if (i < n) {
      const uint2 e = slots[i];
      b.c[k] = e.x;
      b.en[k] = e.x + (e.y & 0x7FFFFFFFu);
      b.s1[k] = e.y >> 31;
    }
  }
#pragma unroll
  for (int k = 0; k < kLB; k++) lean_load<G>(col, b.c[k], b.en[k], gl, b.x[k]);
}

// Walk a fetched batch in window w. Cursor mode (LIST false) writes each
// neighbour's new position back to its slot in `slots`; list mode queues the
// neighbour by its next entry.
template <int G, int CW, bool RET, bool LIST>
__device__ __forceinline__ void batch_walk(const uint32_t* __restrict__ col, LaneBatch& b, uint32_t n, uint2* slots,
                                           ListState* ls, const Win& w, uint64_t& bal, uint64_t& unb) {
  const int gl = threadIdx.x & (G - 1);
  const uint32_t gw = lane_id() / G;
  constexpr uint32_t gpw = 32 / G;
#pragma unroll
  for (int k = 0; k < kLB; k++) {
    const uint32_t i = b.base + gw + k * gpw;
    const bool active = i < n;
    uint32_t xn;
    const uint32_t cn = lean_walk<G, CW, RET>(col, b.c[k], b.en[k], b.s1[k], b.x[k], w, gl, active, bal, unb, xn);
    if (active && gl == 0) {
      if constexpr (LIST) {
        if (cn < b.en[k]) list_queue(*ls, xn, cn, b.en[k], b.s1[k]);
      } else if (cn != b.c[k]) {
        slots[i] = lean_slot(cn, b.en[k], b.s1[k]);
      }
    }
  }
}

// All n slots of one window: the warp's first batch `b` was fetched already
// (possibly while the previous window was being cleared); the warp then
// fetches and walks batches until the slots run out.
template <int G, int CW, bool RET, bool LIST>
__device__ __forceinline__ void window_walk(const uint32_t* __restrict__ col, LaneBatch& b, const uint2* src,
                                            uint32_t n, uint32_t* next, uint2* slots, ListState* ls, const Win& w,
                                            uint64_t& bal, uint64_t& unb) {
  while (b.base < n) {  // warp-uniform
    batch_walk<G, CW, RET, LIST>(col, b, n, slots, ls, w, bal, unb);
    batch_fetch<G>(col, src, n, next, b);
  }
}
// Clear the window's `words` counter words for the next window. With FIN,
// first add every endpoint's Lemma 1 total from its final counter:
// C(p,2) + C(q,2) balanced and p * q unbalanced butterflies.
template <int CW, bool FIN, int THREADS = kSweepThreads>
__device__ __forceinline__ void lean_clear(uint32_t* cnt, uint32_t words, uint64_t& bal, uint64_t& unb) {
  uint4* q4 = reinterpret_cast<uint4*>(cnt);
  const uint32_t quads = (words + 3u) >> 2;
  if constexpr (!FIN) {
    for (uint32_t j = threadIdx.x; j < quads; j += THREADS) q4[j] = make_uint4(0u, 0u, 0u, 0u);
  } else if constexpr (CW == 4) {
    // nibbles (q3, p3, ..., q0, p0): the p's and q's as bytes, then byte dot
    // products as for 8-bit counters (per-thread sums stay far below 2^32)
    uint32_t sq = 0, s = 0, pq = 0;
    for (uint32_t j = threadIdx.x; j < quads; j += THREADS) {
      const uint4 v = q4[j];
      if ((v.x | v.y | v.z | v.w) == 0u) continue;
      const uint32_t a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const uint32_t p = a[k] & 0x0F0F0F0Fu, q = (a[k] >> 4) & 0x0F0F0F0Fu;
        sq = __dp4a(p, p, __dp4a(q, q, sq));
        s = __dp4a(p + q, 0x01010101u, s);
        pq = __dp4a(p, q, pq);
      }
      q4[j] = make_uint4(0u, 0u, 0u, 0u);
    }
    bal += (uint64_t)((sq - s) >> 1);
    unb += (uint64_t)pq;
  } else if constexpr (CW == 8) {
    // bytes (q1, p1, q0, p0): sum of squares, sum, and twice the sum of
    // p * q, by 4-way byte dot products (each per-thread sum < 2^32: at most
    // 60 words of bytes < 256 per window)
    uint32_t sq = 0, s = 0, pq2 = 0;
    for (uint32_t j = threadIdx.x; j < quads; j += THREADS) {
      const uint4 v = q4[j];
      if ((v.x | v.y | v.z | v.w) == 0u) continue;
      const uint32_t a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; k++) {
        sq = __dp4a(a[k], a[k], sq);
        s = __dp4a(a[k], 0x01010101u, s);
        pq2 = __dp4a(a[k], __byte_perm(a[k], 0u, 0x2301u), pq2);
      }
      q4[j] = make_uint4(0u, 0u, 0u, 0u);
    }
    bal += (uint64_t)((sq - s) >> 1);
    unb += (uint64_t)(pq2 >> 1);
  } else if constexpr (CW == 16) {
    // C(p,2) + C(q,2) = C(p+q,2) - p*q
    uint64_t ss = 0, pq = 0;
    for (uint32_t j = threadIdx.x; j < quads; j += THREADS) {
      const uint4 v = q4[j];
      if ((v.x | v.y | v.z | v.w) == 0u) continue;
      const uint32_t a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const uint32_t p = a[k] & 0xFFFFu, q = a[k] >> 16, t = p + q;
        ss += (uint64_t)t * (t - 1u);  // 0 when t = 0
        pq += (uint64_t)p * q;
      }
      q4[j] = make_uint4(0u, 0u, 0u, 0u);
    }
    bal += (ss >> 1) - pq;
    unb += pq;
  } else {
    for (uint32_t j = threadIdx.x; j < quads; j += THREADS) {
      const uint4 v = q4[j];
      if ((v.x | v.y | v.z | v.w) == 0u) continue;
      const uint64_t p0 = v.x, q0 = v.y, p1 = v.z, q1 = v.w;
      bal += (p0 * (p0 - 1) >> 1) + (q0 * (q0 - 1) >> 1) + (p1 * (p1 - 1) >> 1) + (q1 * (q1 - 1) >> 1);
      unb += p0 * q0 + p1 * q1;
      q4[j] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}


template <int THREADS = kSweepThreads>
__device__ __forceinline__ void window_clear(int cw, bool fin, uint32_t* cnt, uint32_t words, uint64_t& bal,
                                             uint64_t& unb) {
  if (cw == 4) {
    if (fin) lean_clear<4, true, THREADS>(cnt, words, bal, unb);
    else lean_clear<4, false, THREADS>(cnt, words, bal, unb);
  } else if (cw == 8) {
    if (fin) lean_clear<8, true, THREADS>(cnt, words, bal, unb);
    else lean_clear<8, false, THREADS>(cnt, words, bal, unb);
  } else if (cw == 16) {
    if (fin) lean_clear<16, true, THREADS>(cnt, words, bal, unb);
    else lean_clear<16, false, THREADS>(cnt, words, bal, unb);
  } else {
    if (fin) lean_clear<32, true, THREADS>(cnt, words, bal, unb);
    else lean_clear<32, false, THREADS>(cnt, words, bal, unb);
  }
}

template <int G, bool LIST>
__device__ __forceinline__ void window_walk_dispatch(int cw, bool fin, const uint32_t* __restrict__ col, LaneBatch& b,
                                                     const uint2* src, uint32_t n, uint32_t* next, uint2* slots,
                                                     ListState* ls, const Win& w, uint64_t& bal, uint64_t& unb) {
  if (cw == 4) {
    if (fin) window_walk<G, 4, false, LIST>(col, b, src, n, next, slots, ls, w, bal, unb);
    else window_walk<G, 4, true, LIST>(col, b, src, n, next, slots, ls, w, bal, unb);
  } else if (cw == 8) {
    if (fin) window_walk<G, 8, false, LIST>(col, b, src, n, next, slots, ls, w, bal, unb);
    else window_walk<G, 8, true, LIST>(col, b, src, n, next, slots, ls, w, bal, unb);
  } else if (cw == 16) {
    if (fin) window_walk<G, 16, false, LIST>(col, b, src, n, next, slots, ls, w, bal, unb);
    else window_walk<G, 16, true, LIST>(col, b, src, n, next, slots, ls, w, bal, unb);
  } else {
    if (fin) window_walk<G, 32, false, LIST>(col, b, src, n, next, slots, ls, w, bal, unb);
    else window_walk<G, 32, true, LIST>(col, b, src, n, next, slots, ls, w, bal, unb);
  }
}

// Every window of a cursor-mode item, in rank order. On entry the L cursors
// are written and the block is synchronised, and both window counters nbn[0]
// and nbn[1] are zero (they are again on return). Each window ends with two
// barriers: after the first, every count and cursor of the window is final,
// so the warps fetch their first batch of the next window (cursors and first
// chunks) and only then clear the counters, which hides that load latency
// behind the clear.
// THREADS and WORDS: the CTA's threads and counter words.
template <int G, int THREADS = kSweepThreads, uint32_t WORDS = kSweepWords>
__device__ __forceinline__ void sweep_cursor_item(const uint32_t* __restrict__ col, uint32_t L, uint2* cur,
                                                  const ItemWindows& iw, bool fin, uint32_t sbase, uint32_t* cnt_words,
                                                  uint32_t* nbn, uint64_t& bal, uint64_t& unb) {
  const uint32_t R = iw.count();
  LaneBatch b;
  batch_fetch<G>(col, cur, L, &nbn[0], b);
  for (uint32_t r = 0; r < R; r++) {
    uint32_t lo, hi;
    int cw;
    iw.window(r, lo, hi, cw);
    const Win w = make_win<WORDS>(cw, lo, hi, sbase);
    window_walk_dispatch<G, false>(cw, fin, col, b, cur, L, &nbn[r & 1], cur, nullptr, w, bal, unb);
    __syncthreads();
    if (r + 1 < R) batch_fetch<G>(col, cur, L, &nbn[(r + 1) & 1], b);
    window_clear<THREADS>(cw, fin, cnt_words, w.words, bal, unb);
    if (threadIdx.x == 0) nbn[r & 1] = 0u;
    __syncthreads();
  }
}

template <int THREADS = kSweepThreads, uint32_t WORDS = kSweepWords>
__device__ __forceinline__ void sweep_cursor_item_dispatch(int group_log, const uint32_t* __restrict__ col,
                                                           uint32_t L, uint2* cur, const ItemWindows& iw, bool fin,
                                                           uint32_t sbase, uint32_t* cnt_words, uint32_t* nbn,
                                                           uint64_t& bal, uint64_t& unb) {
  switch (group_log) {
    case 0: sweep_cursor_item<1, THREADS, WORDS>(col, L, cur, iw, fin, sbase, cnt_words, nbn, bal, unb); break;
    case 2: sweep_cursor_item<4, THREADS, WORDS>(col, L, cur, iw, fin, sbase, cnt_words, nbn, bal, unb); break;
    case 3: sweep_cursor_item<8, THREADS, WORDS>(col, L, cur, iw, fin, sbase, cnt_words, nbn, bal, unb); break;
    case 4: sweep_cursor_item<16, THREADS, WORDS>(col, L, cur, iw, fin, sbase, cnt_words, nbn, bal, unb); break;
    default: sweep_cursor_item<32, THREADS, WORDS>(col, L, cur, iw, fin, sbase, cnt_words, nbn, bal, unb); break;
  }
}

// A list-mode item (see ListState): consecutive spans of at most Rsub windows,
// whose Rsub lists plus two overflow lists of L slots fit the CTA's list_cap
// slots in `lists`. Each neighbour's row is searched once per item (for its
// first entry at or after the item's first rank); a neighbour whose next entry
// lies past the current span waits in an overflow list and is queued when its
// span starts. Windows end as in sweep_cursor_item. Returns the visits
// (listed neighbours), counted by thread 0.
template <int G>
__device__ __forceinline__ uint64_t sweep_list_item(const CsrView& g, const SweepItem& item, const PivotGeom& q,
                                                    uint2* lists, int64_t list_cap, ListState& ls, uint32_t sbase,
                                                    uint32_t* cnt_words, uint32_t* nbn, uint64_t& bal, uint64_t& unb) {
  const int tid = threadIdx.x;
  const ItemWindows iw(item);
  const uint32_t R = iw.count();
  const bool fin = (item.flags & kItemFinalize) != 0;
  const int64_t per_nb = list_cap / (int64_t)q.L;
  const uint32_t Rsub = (uint32_t)(per_nb - 2 < kListMaxWindows ? per_nb - 2 : kListMaxWindows);
  uint64_t visits = 0;
  int in_buf = 0;  // the overflow list that feeds the next span
  // entries of list r (checked builds: at most its L slots)
  auto listed = [&](uint32_t r) {
    const uint32_t n = (uint32_t)ls.cnt[r];
    return DBBC_CHECK(n <= q.L) ? n : q.L;
  };
  for (uint32_t s0 = 0; s0 < R; s0 += Rsub) {
    const uint32_t nwin = min(Rsub, R - s0);
    uint32_t span_lo, span_hi, wlo, whi;
    int cw;
    iw.window(s0, span_lo, whi, cw);
    iw.window(s0 + nwin - 1, wlo, span_hi, cw);
    uint2* over_in = lists + (size_t)(Rsub + in_buf) * q.L;
    uint32_t n_in = s0 == 0 ? 0u : (uint32_t)ls.ocnt;  // final since the last barrier of the previous span
    if (!DBBC_CHECK(n_in <= q.L)) n_in = q.L;
    __syncthreads();  // every thread has read ls.ocnt
    if (tid == 0) {
      ls.lists = lists;
      ls.over = lists + (size_t)(Rsub + (in_buf ^ 1)) * q.L;
      ls.ocnt = 0;
      ls.L = q.L;
      ls.nwin = nwin;
      ls.iw = iw;
      ls.s0 = s0;
      ls.hl = span_hi << 1;
      ls.item_hl = item.hi << 1;
    }
    if (tid < kListMaxWindows) ls.cnt[tid] = 0;
    __syncthreads();
    if (s0 == 0) {  // each neighbour joins the list of the window of its first entry
      for (uint32_t i = tid; i < q.L; i += kSweepThreads) {
        uint32_t b, en, s1;
        lean_cursor_start(g, q, i, (item.flags & kItemFirst) ? 0u : item.lo, b, en, s1);
        if (b < en) list_queue(ls, g.col[b], b, en, s1);
      }
    } else {  // the neighbours that waited for this span
      for (uint32_t j = tid; j < n_in; j += kSweepThreads) {
        const uint2 e = over_in[j];
        const uint32_t c = e.x, en = e.x + (e.y & 0x7FFFFFFFu);
        if (DBBC_CHECK(c < en && (int64_t)en <= g.nnz)) list_queue(ls, g.col[c], c, en, e.y >> 31);
      }
    }
    __syncthreads();
    LaneBatch b;
    batch_fetch<G>(g.col, lists, listed(0), &nbn[0], b);
    for (uint32_t r = 0; r < nwin; r++) {
      iw.window(s0 + r, wlo, whi, cw);
      const Win w = make_win(cw, wlo, whi, sbase);
      const uint32_t n = listed(r);
      window_walk_dispatch<G, true>(cw, fin, g.col, b, lists + (size_t)r * q.L, n, &nbn[r & 1], nullptr, &ls, w,
                                    bal, unb);
      visits += tid == 0 ? n : 0;
      __syncthreads();  // also publishes the appends to later windows' lists
      if (r + 1 < nwin)
        batch_fetch<G>(g.col, lists + (size_t)(r + 1) * q.L, listed(r + 1), &nbn[(r + 1) & 1], b);
      window_clear(cw, fin, cnt_words, w.words, bal, unb);
      if (tid == 0) nbn[r & 1] = 0u;
      __syncthreads();
    }
    in_buf ^= 1;
  }
  return visits;
}

__device__ __forceinline__ uint64_t sweep_list_item_dispatch(const CsrView& g, const SweepItem& item,
                                                             const PivotGeom& q, uint2* lists, int64_t list_cap,
                                                             ListState& ls, uint32_t sbase, uint32_t* cnt_words,
                                                             uint32_t* nbn, uint64_t& bal, uint64_t& unb) {
  switch (item.group_log) {
    case 0: return sweep_list_item<1>(g, item, q, lists, list_cap, ls, sbase, cnt_words, nbn, bal, unb);
    case 2: return sweep_list_item<4>(g, item, q, lists, list_cap, ls, sbase, cnt_words, nbn, bal, unb);
    case 3: return sweep_list_item<8>(g, item, q, lists, list_cap, ls, sbase, cnt_words, nbn, bal, unb);
    case 4: return sweep_list_item<16>(g, item, q, lists, list_cap, ls, sbase, cnt_words, nbn, bal, unb);
    default: return sweep_list_item<32>(g, item, q, lists, list_cap, ls, sbase, cnt_words, nbn, bal, unb);
  }
}

}  // namespace dbbc
