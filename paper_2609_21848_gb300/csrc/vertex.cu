// Butterflies containing each vertex (the "tip" input of the paper's
// applications) and each edge (the "wing" input), computed with the same
// tiers as the totals. Once the buckets of a pivot u are complete (a pivot's
// hash table, or one window of a hub):
//   * every endpoint w and u itself are in C(p,2) + C(q,2) balanced and p*q
//     unbalanced butterflies of u, where (p, q) are w's symmetric and
//     asymmetric bucket counts (Algorithm 1, Lemma 1);
//   * a symmetric wedge u-v-w pairs with the p - 1 other symmetric wedges to w
//     (balanced) and the q asymmetric ones (unbalanced); an asymmetric wedge
//     with q - 1 and p. Each pairing is one butterfly through the middle v and
//     through both edges (u, v) and (v, w) of the wedge.
// The middles and edges need a second walk of the same wedges after the counts
// are final. Vertex results are accumulated per CSR row and mapped to unified
// ids at the end; edge results per CSR position (an edge has one position in
// each of its two rows), summed over both positions when an edge is queried.
#include "count_device.cuh"

namespace dbbc {

struct TipOut {
  unsigned long long* vb = nullptr;  // [n] per row (vertex counts)
  unsigned long long* vu = nullptr;
  unsigned long long* eb = nullptr;  // [nnz] per CSR position (edge counts)
  unsigned long long* eu = nullptr;
  int64_t n = 0, nnz = 0;            // their lengths
};

// Counter of endpoint w in a shared hash table (the key must be present).
__device__ __forceinline__ unsigned long long hash_find(const uint32_t* keys, const unsigned long long* vals,
                                                        int log_h, uint32_t w) {
  const uint32_t mask = (1u << log_h) - 1u;
  uint32_t h = hash_slot(w, log_h);
  for (uint32_t probe = 0; probe <= mask; probe++) {
    if (keys[h] == w) return vals[h];
    if (keys[h] == kEmptyKey) break;
    h = (h + 1u) & mask;
  }
  return 0ull;
}

// Butterflies one wedge is in, from its endpoint's buckets (p, q) packed as
// (q << 32) | p: the other wedges of its own class close balanced ones, the
// wedges of the other class unbalanced ones.
__device__ __forceinline__ void wedge_pairs(unsigned long long packed, bool sym, uint64_t& bal, uint64_t& unb) {
  const uint64_t p = packed & 0xFFFFFFFFull, q = packed >> 32;
  bal = sym ? p - 1 : q - 1;
  unb = sym ? q : p;
}

__device__ __forceinline__ void endpoint_contrib(unsigned long long packed, uint64_t& bal, uint64_t& unb) {
  const uint64_t p = packed & 0xFFFFFFFFull, q = packed >> 32;
  bal += (p * (p - (p > 0)) >> 1) + (q * (q - (q > 0)) >> 1);
  unb += p * q;
}

__device__ __forceinline__ void add_pair(unsigned long long* b, unsigned long long* u, int64_t i, uint64_t x,
                                         uint64_t y) {
  if (x) atomicAdd(&b[i], (unsigned long long)x);
  if (y) atomicAdd(&u[i], (unsigned long long)y);
}

// Per-row (vertex) and per-CSR-position (edge) sums; checked builds test the
// position first.
__device__ __forceinline__ void add_vertex(const TipOut& o, int64_t r, uint64_t x, uint64_t y) {
  if (DBBC_CHECK(r >= 0 && r < o.n)) add_pair(o.vb, o.vu, r, x, y);
}
__device__ __forceinline__ void add_edge(const TipOut& o, int64_t j, uint64_t x, uint64_t y) {
  if (DBBC_CHECK(j >= 0 && j < o.nnz)) add_pair(o.eb, o.eu, j, x, y);
}

// The second walk over a pivot's wedges (lower-neighbour positions [a, b),
// `step` apart in groups of 32 per warp): each lane credits the far edge
// (v, w) of its wedge; the warp sums v's wedges and one lane credits the
// middle v and the near edge (u, v).
template <bool VERT, bool EDGE, typename Lookup>
__device__ __forceinline__ void warp_second_walk(const CsrView& g, const PivotGeom& q, uint32_t a, uint32_t b,
                                                 uint32_t step, Lookup&& lookup, const TipOut& o) {
  const unsigned lane = lane_id();
  for (uint32_t i0 = a; i0 < b; i0 += step) {
    uint32_t e = 0;
    int64_t vb0 = 0, ve = 0;
    if (i0 + lane < b) {
      e = g.col[q.rb + i0 + lane];
      const int64_t vrow = q.base + (e >> 1);
      vb0 = g.row_ptr[vrow];
      ve = g.row_ptr[vrow + 1];
    }
    const uint32_t cnt = min(32u, b - i0);
    for (uint32_t k = 0; k < cnt; k++) {
      const uint32_t ek = __shfl_sync(kFullMask, e, k);
      const uint32_t s1 = ek & 1u;
      const int64_t jb0 = __shfl_sync(kFullMask, vb0, k);
      const int64_t je = __shfl_sync(kFullMask, ve, k);
      uint64_t sb = 0, su = 0;
      for (int64_t jb = jb0; jb < je; jb += 32) {
        const int64_t j = jb + lane;
        const uint32_t x = j < je ? g.col[j] : 0xFFFFFFFFu;
        const bool ok = x < q.lim;
        if (ok) {
          uint64_t cb, cu;
          wedge_pairs(lookup(x >> 1), ((x ^ s1) & 1u) == 0, cb, cu);
          if (EDGE) add_edge(o, j, cb, cu);
          sb += cb;
          su += cu;
        }
        if (__ballot_sync(kFullMask, !ok)) break;  // rows ascend: nothing accepted beyond
      }
      sb = warp_sum_u64(sb);
      su = warp_sum_u64(su);
      if (lane == 0) {
        if (VERT) add_vertex(o, q.base + (ek >> 1), sb, su);
        if (EDGE) add_edge(o, q.rb + i0 + k, sb, su);
      }
    }
  }
}

// ------------------------------------------------------------------ light / medium
template <bool VERT, bool EDGE>
__global__ void __launch_bounds__(kLightWarps * 32) tips_light_kernel(CsrView g, const int32_t* __restrict__ piv,
                                                                      const uint64_t* __restrict__ work,
                                                                      int64_t n_piv, int hash_mult_log, TipOut o,
                                                                      unsigned* status) {
  extern __shared__ __align__(16) unsigned char light_smem[];
  unsigned long long* vals_all = reinterpret_cast<unsigned long long*>(light_smem);
  uint32_t* keys_all = reinterpret_cast<uint32_t*>(vals_all + kLightWarps * kLightSlots);
  const int w = threadIdx.x >> 5;
  const unsigned lane = lane_id();
  uint32_t* keys = keys_all + w * kLightSlots;
  unsigned long long* vals = vals_all + w * kLightSlots;
  for (int i = lane; i < kLightSlots; i += 32) {
    keys[i] = kEmptyKey;
    vals[i] = 0;
  }
  __syncwarp();
  bool full = false;
  const int64_t nw = (int64_t)gridDim.x * kLightWarps;
  for (int64_t t = (int64_t)blockIdx.x * kLightWarps + w; t < n_piv; t += nw) {
    const int32_t p = piv[t];
    const int log_h = table_log(work[p], 10, hash_mult_log);
    const PivotGeom q = pivot_geom(g, p);
    warp_walk<1>(g, q, 0, q.L, 32, [&](const uint32_t (&x)[1], uint32_t s1) {
      if (x[0] != 0xFFFFFFFFu) {
        unsigned long long old;
        full |= !smem_hash_add(keys, vals, log_h, x[0] >> 1, wedge_inc(x[0], s1), &old);
      }
    });
    __syncwarp();
    if (VERT) {
      const int64_t end_base = p < g.n_u ? 0 : (int64_t)g.n_u;  // endpoints share the pivot's side
      uint64_t pb = 0, pu = 0;
      for (int i = lane; i < (1 << log_h); i += 32) {
        if (keys[i] != kEmptyKey) {
          uint64_t eb = 0, eu = 0;
          endpoint_contrib(vals[i], eb, eu);
          add_vertex(o, end_base + keys[i], eb, eu);
          pb += eb;
          pu += eu;
        }
      }
      pb = warp_sum_u64(pb);
      pu = warp_sum_u64(pu);
      if (lane == 0) add_vertex(o, p, pb, pu);
    }
    warp_second_walk<VERT, EDGE>(g, q, 0, q.L, 32, [&](uint32_t x) { return hash_find(keys, vals, log_h, x); }, o);
    __syncwarp();
    for (int i = lane; i < (1 << log_h); i += 32) {
      keys[i] = kEmptyKey;
      vals[i] = 0;
    }
    __syncwarp();
  }
  if (full) atomicOr(status, DBBC_DEV_HASH_FULL);
}

template <bool VERT, bool EDGE>
__global__ void __launch_bounds__(kMediumThreads) tips_medium_kernel(CsrView g, const int32_t* __restrict__ piv,
                                                                     const uint64_t* __restrict__ work,
                                                                     int64_t n_piv, int hash_mult_log, TipOut o,
                                                                     unsigned* status) {
  extern __shared__ __align__(16) unsigned char med_smem[];
  unsigned long long* vals = reinterpret_cast<unsigned long long*>(med_smem);
  uint32_t* keys = reinterpret_cast<uint32_t*>(vals + kMediumSlots);
  for (int i = threadIdx.x; i < kMediumSlots; i += kMediumThreads) {
    keys[i] = kEmptyKey;
    vals[i] = 0;
  }
  __syncthreads();
  const int w = threadIdx.x >> 5;
  bool full = false;
  for (int64_t t = blockIdx.x; t < n_piv; t += gridDim.x) {
    const int32_t p = piv[t];
    const int log_h = table_log(work[p], 13, hash_mult_log);
    const PivotGeom q = pivot_geom(g, p);
    warp_walk<2>(g, q, (uint32_t)w * 32u, q.L, kMediumWarps * 32u, [&](const uint32_t (&x)[2], uint32_t s1) {
#pragma unroll
      for (int u = 0; u < 2; u++) {
        if (x[u] != 0xFFFFFFFFu) {
          unsigned long long old;
          full |= !smem_hash_add(keys, vals, log_h, x[u] >> 1, wedge_inc(x[u], s1), &old);
        }
      }
    });
    __syncthreads();
    if (VERT) {
      const int64_t end_base = p < g.n_u ? 0 : (int64_t)g.n_u;
      uint64_t pb = 0, pu = 0;
      for (int i = threadIdx.x; i < (1 << log_h); i += kMediumThreads) {
        if (keys[i] != kEmptyKey) {
          uint64_t eb = 0, eu = 0;
          endpoint_contrib(vals[i], eb, eu);
          add_vertex(o, end_base + keys[i], eb, eu);
          pb += eb;
          pu += eu;
        }
      }
      pb = warp_sum_u64(pb);
      pu = warp_sum_u64(pu);
      if (lane_id() == 0) add_vertex(o, p, pb, pu);
    }
    warp_second_walk<VERT, EDGE>(g, q, (uint32_t)w * 32u, q.L, kMediumWarps * 32u,
                                 [&](uint32_t x) { return hash_find(keys, vals, log_h, x); }, o);
    __syncthreads();
    for (int i = threadIdx.x; i < (1 << log_h); i += kMediumThreads) {
      keys[i] = kEmptyKey;
      vals[i] = 0;
    }
    __syncthreads();
  }
  if (full) atomicOr(status, DBBC_DEV_HASH_FULL);
}

// ------------------------------------------------------------------ hub windows
// Counter k of a window of width CW (see add_wedge) as (asym << 32) | sym.
template <int CW>
__device__ __forceinline__ unsigned long long window_value(const uint32_t* c16, const unsigned long long* c32,
                                                           uint32_t k) {
  if (CW == 8) {
    const uint32_t v = (c16[k >> 1] >> ((k & 1u) << 4)) & 0xFFFFu;
    return ((unsigned long long)(v >> 8) << 32) | (v & 0xFFu);
  }
  if (CW == 16) {
    const uint32_t v = c16[k];
    return ((unsigned long long)(v >> 16) << 32) | (v & 0xFFFFu);
  }
  return c32[k];
}

// One window of a hub item, in three passes over the item's lower
// neighbours (lane groups of G as in the counting sweep, moving in warp
// lockstep): count the window's wedges (each neighbour's cursor moves past
// the window, its old value kept in `prev`), credit endpoints and the pivot
// from the complete window, then walk every neighbour's segment
// [prev, cursor) again for the middles and edges.
template <int G, int CW, bool VERT, bool EDGE>
__device__ __forceinline__ void tips_window(const CsrView& g, const PivotGeom& q, uint32_t* cur, uint32_t* prev, uint32_t lo,
                            uint32_t hi, uint32_t* c16, unsigned long long* c32, const TipOut& o, uint64_t& pb,
                            uint64_t& pu) {
  const uint32_t hl = hi << 1, lo2 = lo << 1;
  const int gl = threadIdx.x & (G - 1);
  const uint32_t gid = threadIdx.x / G;
  constexpr uint32_t groups = kSweepThreads / G;
  const uint32_t* col = g.col;
  uint64_t unused_b = 0, unused_u = 0;
  for (uint32_t i = gid; __any_sync(kFullMask, i < q.L); i += groups) {
    const bool active = i < q.L;
    const uint32_t c = active ? cur[2 * i] : 0u, en = active ? cur[2 * i + 1] : 0u;
    const uint32_t s1 = active ? col[q.rb + i] & 1u : 0u;
    uint32_t x[kSweepUnroll];
    load_chunk<G>(col, c, en, gl, x);
    const uint32_t cn = walk_segment<G, CW>(col, c, en, s1, x, lo2, hl, gl, active, c16, c32, unused_b, unused_u);
    if (active && gl == 0) {
      prev[i] = c;
      cur[2 * i] = cn;
    }
  }
  __syncthreads();
  if (VERT) {
    const int64_t end_base = q.base == 0 ? (int64_t)g.n_u : 0;  // endpoints share the pivot's side
    for (uint32_t k = threadIdx.x; k < hi - lo; k += kSweepThreads) {
      const unsigned long long v = window_value<CW>(c16, c32, k);
      if (v) {
        uint64_t eb = 0, eu = 0;
        endpoint_contrib(v, eb, eu);
        add_vertex(o, end_base + lo + k, eb, eu);
        pb += eb;
        pu += eu;
      }
    }
  }
  for (uint32_t i = gid; __any_sync(kFullMask, i < q.L); i += groups) {
    const bool active = i < q.L;
    const uint32_t c0 = active ? prev[i] : 0u, c1 = active ? cur[2 * i] : 0u;
    const uint32_t e = active ? col[q.rb + i] : 0u;
    const uint32_t s1 = e & 1u;
    const uint32_t trips = __reduce_max_sync(kFullMask, (c1 - c0 + G - 1) / G);
    uint64_t sb = 0, su = 0;
    for (uint32_t t = 0; t < trips; t++) {
      const uint32_t pos = c0 + t * G + gl;
      if (pos < c1) {
        const uint32_t xx = col[pos];
        uint64_t cb, cu;
        wedge_pairs(window_value<CW>(c16, c32, (xx - lo2) >> 1), ((xx ^ s1) & 1u) == 0, cb, cu);
        if (EDGE) add_edge(o, pos, cb, cu);
        sb += cb;
        su += cu;
      }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {  // sum over the group's lanes
      sb += __shfl_xor_sync(kFullMask, sb, off);
      su += __shfl_xor_sync(kFullMask, su, off);
    }
    if (active && gl == 0) {
      if (VERT) add_vertex(o, q.base + (e >> 1), sb, su);
      if (EDGE) add_edge(o, q.rb + i, sb, su);
    }
  }
  __syncthreads();
  zero_words(c16, window_words<CW>(hi - lo));
  __syncthreads();
}

template <int CW, bool VERT, bool EDGE>
__device__ __forceinline__ void tips_window_dispatch(int group_log, const CsrView& g, const PivotGeom& q,
                                                     uint32_t* cur, uint32_t* prev, uint32_t lo, uint32_t hi,
                                                     uint32_t* c16, unsigned long long* c32, const TipOut& o,
                                                     uint64_t& pb, uint64_t& pu) {
  switch (group_log) {
    case 0: tips_window<1, CW, VERT, EDGE>(g, q, cur, prev, lo, hi, c16, c32, o, pb, pu); break;
    case 2: tips_window<4, CW, VERT, EDGE>(g, q, cur, prev, lo, hi, c16, c32, o, pb, pu); break;
    case 3: tips_window<8, CW, VERT, EDGE>(g, q, cur, prev, lo, hi, c16, c32, o, pb, pu); break;
    case 4: tips_window<16, CW, VERT, EDGE>(g, q, cur, prev, lo, hi, c16, c32, o, pb, pu); break;
    default: tips_window<32, CW, VERT, EDGE>(g, q, cur, prev, lo, hi, c16, c32, o, pb, pu); break;
  }
}

template <bool VERT, bool EDGE>
__global__ void __launch_bounds__(kSweepThreads, 1) tips_sweep_kernel(CsrView g, const SweepItem* __restrict__ items,
                                                                   int64_t n_items, int* next_item,
                                                                   uint32_t* __restrict__ cursors, int64_t cur_cap,
                                                                   TipOut o) {
  extern __shared__ __align__(16) unsigned char sweep_smem[];
  uint32_t* c16 = reinterpret_cast<uint32_t*>(sweep_smem);
  unsigned long long* c32 = reinterpret_cast<unsigned long long*>(sweep_smem);
  __shared__ int item_sh;
  __shared__ unsigned long long red[2][kSweepThreads / 32];
  const int tid = threadIdx.x;
  zero_words(c16, kSweepWindow16);
  uint32_t* cur = cursors + (int64_t)blockIdx.x * cur_cap * 3;  // [cur_cap][2] cursor and row end
  uint32_t* prev = cur + 2 * cur_cap;                              // [cur_cap] cursor before the window
  for (;;) {
    if (tid == 0) item_sh = atomicAdd(next_item, 1);
    __syncthreads();
    const int64_t it = item_sh;
    __syncthreads();
    if (it >= n_items) break;
    const SweepItem item = items[it];
    PivotGeom q = pivot_geom(g, item.row);
    if (!DBBC_CHECK((int64_t)q.L <= cur_cap)) q.L = 0;  // checked builds: cursor capacity
    const ItemWindows iw(item, false);  // this sweep has no 4-bit counters
    for (uint32_t i = tid; i < q.L; i += kSweepThreads) {
      uint32_t b, en;
      init_cursor(g, q, i, (item.flags & kItemFirst) ? 0u : item.lo, cur, b, en);
    }
    __syncthreads();
    uint64_t pb = 0, pu = 0;
    for (uint32_t r = 0; r < iw.count(); r++) {
      uint32_t lo, hi;
      int cw;
      iw.window(r, lo, hi, cw);
      if (cw == 8) tips_window_dispatch<8, VERT, EDGE>(item.group_log, g, q, cur, prev, lo, hi, c16, c32, o, pb, pu);
      else if (cw == 16) tips_window_dispatch<16, VERT, EDGE>(item.group_log, g, q, cur, prev, lo, hi, c16, c32, o, pb, pu);
      else tips_window_dispatch<32, VERT, EDGE>(item.group_log, g, q, cur, prev, lo, hi, c16, c32, o, pb, pu);
    }
    if (VERT) {  // the pivot's share of this item
      pb = warp_sum_u64(pb);
      pu = warp_sum_u64(pu);
      if (lane_id() == 0) {
        red[0][tid >> 5] = pb;
        red[1][tid >> 5] = pu;
      }
      __syncthreads();
      if (tid < 32) {
        uint64_t x = tid < kSweepThreads / 32 ? red[0][tid] : 0, y = tid < kSweepThreads / 32 ? red[1][tid] : 0;
        x = warp_sum_u64(x);
        y = warp_sum_u64(y);
        if (tid == 0) add_vertex(o, item.row, x, y);
      }
      __syncthreads();
    }
  }
}

__global__ void rows_to_ids_kernel(const int32_t* __restrict__ vertex, int64_t n, const unsigned long long* rb,
                                   const unsigned long long* ru, unsigned long long* ob, unsigned long long* ou) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    ob[vertex[r]] = rb[r];
    ou[vertex[r]] = ru[r];
  }
}

__global__ void row_of_id_kernel(const int32_t* __restrict__ vertex, int64_t n, int32_t* __restrict__ row_of) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    row_of[vertex[r]] = (int32_t)r;
}

// Position in [b, e) of a row whose entry has side rank r, or -1 (rows are
// sorted by entry, and an entry is (side rank << 1) | negative).
__device__ __forceinline__ int64_t find_in_row(const uint32_t* col, int64_t b, int64_t e, uint32_t r) {
  const uint32_t key = r << 1;
  const int64_t end = e;
  while (b < e) {
    const int64_t mid = (b + e) >> 1;
    if (col[mid] < key) b = mid + 1; else e = mid;
  }
  return b < end && (col[b] >> 1) == r ? b : -1;
}

// Per queried pair (U id, V id): the sum of the counts at the edge's two CSR
// positions, or zeros when the pair is not an edge; ids out of range set err.
__global__ void edge_query_kernel(CsrView g, const int32_t* __restrict__ row_of, const int32_t* __restrict__ qu,
                                  const int32_t* __restrict__ qv, int64_t k, const unsigned long long* eb,
                                  const unsigned long long* eu, unsigned long long* ob, unsigned long long* ou,
                                  unsigned* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = qu[i], b = qv[i];
    unsigned long long xb = 0, xu = 0;
    if (a < 0 || a >= g.n_u || b < 0 || (int64_t)b >= g.n - g.n_u) {
      atomicOr(err, 1u);
    } else {
      const int64_t ru = row_of[a], rv = row_of[(int64_t)g.n_u + b];
      const int64_t p1 = find_in_row(g.col, g.row_ptr[ru], g.row_ptr[ru + 1], (uint32_t)(rv - g.n_u));
      const int64_t p2 = find_in_row(g.col, g.row_ptr[rv], g.row_ptr[rv + 1], (uint32_t)ru);
      if (p1 >= 0 && p2 >= 0) {
        xb = eb[p1] + eb[p2];
        xu = eu[p1] + eu[p2];
      }
    }
    ob[i] = xb;
    ou[i] = xu;
  }
}

template <bool VERT, bool EDGE>
void enqueue_tips(const dbbc_graph* g, cudaStream_t s, const TipOut& o, unsigned* d_status, Scratch& sc) {
  if (g->n_piv == 0) return;
  const CsrView view{g->row_ptr, g->col, g->lower, g->n_u, g->n, g->nnz};
  const int sms = num_sms();
  if (g->n_light > 0) {
    auto fn = tips_light_kernel<VERT, EDGE>;
    const size_t smem = (size_t)kLightWarps * kLightSlots * 12;
    DBBC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t want = ceil_div<int64_t>(g->n_light, kLightWarps);
    const int64_t cap = (int64_t)sms * blocks_per_sm((const void*)fn, kLightWarps * 32, smem);
    fn<<<(unsigned)std::min(want, cap), kLightWarps * 32, smem, s>>>(
        view, g->order + g->n_hub + g->n_medium, g->work, g->n_light, g->tune.hash_mult_log, o, d_status);
    DBBC_LAUNCH_CHECK();
  }
  if (g->n_medium > 0) {
    auto fn = tips_medium_kernel<VERT, EDGE>;
    const size_t smem = (size_t)kMediumSlots * 12;
    DBBC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t cap = (int64_t)sms * blocks_per_sm((const void*)fn, kMediumThreads, smem);
    fn<<<(unsigned)std::min<int64_t>(g->n_medium, cap), kMediumThreads, smem, s>>>(
        view, g->order + g->n_hub, g->work, g->n_medium, g->tune.hash_mult_log, o, d_status);
    DBBC_LAUNCH_CHECK();
  }
  if (g->n_hub > 0) {
    auto fn = tips_sweep_kernel<VERT, EDGE>;
    const size_t smem = (size_t)kSweepWindow16 * 4;
    DBBC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = sms * blocks_per_sm((const void*)fn, kSweepThreads, smem);
    uint32_t* cursors = sc.get<uint32_t>((size_t)grid * (size_t)g->sweep_max_lower * 3);
    int* next = sc.get<int>(1);
    DBBC_CUDA(cudaMemsetAsync(next, 0, sizeof(int), s));
    fn<<<grid, kSweepThreads, smem, s>>>(view, g->sweep_items, g->n_sweep_items, next, cursors, g->sweep_max_lower,
                                         o);
    DBBC_LAUNCH_CHECK();
  }
}

inline unsigned grid_1d(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
}

}  // namespace dbbc

using namespace dbbc;

extern "C" dbbc_status dbbc_count_vertices(const dbbc_graph* g, void* cuda_stream, uint64_t* balanced_v,
                                           uint64_t* unbalanced_v) {
  if (!g || (g->n > 0 && (!balanced_v || !unbalanced_v))) return DBBC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  try {
    if (g->n == 0) return DBBC_OK;
    Scratch sc(s);
    const int64_t n = g->n;
    unsigned long long* rows = sc.get<unsigned long long>((size_t)(4 * n));  // row sums, then per-id output
    unsigned* d_status = sc.get<unsigned>(1);
    DBBC_CUDA(cudaMemsetAsync(rows, 0, (size_t)(2 * n) * 8, s));
    DBBC_CUDA(cudaMemsetAsync(d_status, 0, sizeof(unsigned), s));
    TipOut o;
    o.vb = rows;
    o.vu = rows + n;
    o.n = n;
    enqueue_tips<true, false>(g, s, o, d_status, sc);
    unsigned long long* ob = rows + 2 * n;
    unsigned long long* ou = rows + 3 * n;
    rows_to_ids_kernel<<<grid_1d(n), 256, 0, s>>>(g->vertex, n, o.vb, o.vu, ob, ou);
    DBBC_LAUNCH_CHECK();
    DBBC_CUDA(cudaMemcpyAsync(balanced_v, ob, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    DBBC_CUDA(cudaMemcpyAsync(unbalanced_v, ou, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    unsigned h = 0;
    DBBC_CUDA(cudaMemcpyAsync(&h, d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
    DBBC_CUDA(cudaStreamSynchronize(s));
    raise_device_status(h);
  } catch (const Error& e) {
    return e.status;
  } catch (...) {
    return DBBC_EINTERNAL;
  }
  return DBBC_OK;
}

extern "C" dbbc_status dbbc_count_edges(const dbbc_graph* g, void* cuda_stream, const int32_t* qu, const int32_t* qv,
                                        int64_t k, uint32_t flags, uint64_t* balanced_e, uint64_t* unbalanced_e) {
  if (!g || k < 0 || (flags & ~(uint32_t)DBBC_INPUT_DEVICE) != 0) return DBBC_EINVAL;
  if (k == 0) return DBBC_OK;
  if (!qu || !qv || !balanced_e || !unbalanced_e) return DBBC_EINVAL;
  if (g->n_u == 0 || g->n == g->n_u) return DBBC_EINVAL;  // no pair is in range
  const bool on_device = (flags & DBBC_INPUT_DEVICE) != 0;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  try {
    Scratch sc(s);
    const int64_t n = g->n, nnz = g->nnz;
    unsigned long long* acc = sc.get<unsigned long long>((size_t)(2 * nnz));
    unsigned* d_status = sc.get<unsigned>(2);  // [0] device checks, [1] ids out of range
    int32_t* row_of = sc.get<int32_t>((size_t)n);
    DBBC_CUDA(cudaMemsetAsync(acc, 0, (size_t)(2 * nnz) * 8, s));
    DBBC_CUDA(cudaMemsetAsync(d_status, 0, 2 * sizeof(unsigned), s));
    TipOut o;
    o.eb = acc;
    o.eu = acc + nnz;
    o.nnz = nnz;
    enqueue_tips<false, true>(g, s, o, d_status, sc);
    row_of_id_kernel<<<grid_1d(n), 256, 0, s>>>(g->vertex, n, row_of);
    DBBC_LAUNCH_CHECK();
    const int32_t* dqu = qu;
    const int32_t* dqv = qv;
    unsigned long long* ob = reinterpret_cast<unsigned long long*>(balanced_e);
    unsigned long long* ou = reinterpret_cast<unsigned long long*>(unbalanced_e);
    if (!on_device) {
      int32_t* q = sc.get<int32_t>((size_t)(2 * k));
      DBBC_CUDA(cudaMemcpyAsync(q, qu, (size_t)k * 4, cudaMemcpyHostToDevice, s));
      DBBC_CUDA(cudaMemcpyAsync(q + k, qv, (size_t)k * 4, cudaMemcpyHostToDevice, s));
      dqu = q;
      dqv = q + k;
      ob = sc.get<unsigned long long>((size_t)(2 * k));
      ou = ob + k;
    }
    const CsrView view{g->row_ptr, g->col, g->lower, g->n_u, g->n, g->nnz};
    edge_query_kernel<<<grid_1d(k), 256, 0, s>>>(view, row_of, dqu, dqv, k, o.eb, o.eu, ob, ou, d_status + 1);
    DBBC_LAUNCH_CHECK();
    if (!on_device) {
      DBBC_CUDA(cudaMemcpyAsync(balanced_e, ob, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
      DBBC_CUDA(cudaMemcpyAsync(unbalanced_e, ou, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
    }
    unsigned h[2] = {0, 0};
    DBBC_CUDA(cudaMemcpyAsync(h, d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
    DBBC_CUDA(cudaStreamSynchronize(s));
    if (h[1]) return DBBC_EINVAL;
    raise_device_status(h[0]);
  } catch (const Error& e) {
    return e.status;
  } catch (...) {
    return DBBC_EINTERNAL;
  }
  return DBBC_OK;
}
