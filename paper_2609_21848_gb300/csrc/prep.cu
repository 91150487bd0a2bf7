// Graph build on the device: validate, keep-latest deduplication, degrees,
// Def. 3 priority ranks, sign-packed CSR sorted by priority, accepted-wedge
// work per pivot (Algorithm 1's inner loop bounds), and the counting tiers.
#include <algorithm>
#include <cstring>

#include "internal.h"
#include "radix.cuh"

namespace dbbc {

// Components of a disjoint union as seen by the kernels: component c owns the
// side ids (and, after ranking, the side ranks) [uoff[c], uoff[c+1]) of U and
// [voff[c], voff[c+1]) of V. A plain graph is one component.
struct UnionView {
  const int64_t* uoff;
  const int64_t* voff;
  int32_t n_graphs;
};

__device__ __forceinline__ int32_t component_of(const int64_t* off, int32_t n_graphs, int64_t side_id) {
  int64_t lo = 0, hi = (int64_t)n_graphs + 1;  // upper_bound over off[0 .. n_graphs]
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (off[mid] <= side_id) lo = mid + 1; else hi = mid;
  }
  return (int32_t)(lo - 1);
}

// ------------------------------------------------------------------ kernels
template <typename T>
__device__ __forceinline__ int64_t lower_bound_dev(const T* a, int64_t n, T x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
template <typename T>
__device__ __forceinline__ int64_t upper_bound_dev(const T* a, int64_t n, T x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void validate_kernel(const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                const int8_t* __restrict__ s, int64_t m, int32_t n_u, int32_t n_v, unsigned* err) {
  unsigned e = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = u[i], b = v[i];
    const int8_t c = s[i];
    if (a < 0 || a >= n_u) e |= 1u;
    if (b < 0 || b >= n_v) e |= 2u;
    if (c != 1 && c != -1) e |= 4u;
  }
  e = __reduce_or_sync(kFullMask, e);
  if (lane_id() == 0 && e) atomicOr(err, e);
}

__global__ void edge_keys_kernel(const int32_t* __restrict__ u, const int32_t* __restrict__ v, int64_t m, int bits_v,
                                 uint64_t* __restrict__ key, uint32_t* __restrict__ idx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    key[i] = ((uint64_t)(uint32_t)u[i] << bits_v) | (uint32_t)v[i];
    idx[i] = (uint32_t)i;
  }
}

// flag[i] = 1 iff i is the last occurrence of its key (keys sorted stably, so
// the last of a run is the latest input occurrence).
__global__ void run_last_kernel(const uint64_t* __restrict__ key, int64_t m, uint32_t* __restrict__ flag,
                                unsigned* dup) {
  bool any_dup = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const bool last = (i == m - 1) || (key[i] != key[i + 1]);
    flag[i] = last ? 1u : 0u;
    any_dup |= !last;
  }
  if (__any_sync(kFullMask, any_dup) && lane_id() == 0) atomicOr(dup, 8u);
}

__global__ void compact_edges_kernel(const uint64_t* __restrict__ key, const uint32_t* __restrict__ idx,
                                     const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                                     const int8_t* __restrict__ sign, int64_t m, int bits_v,
                                     int32_t* __restrict__ eu, int32_t* __restrict__ ev, int8_t* __restrict__ es) {
  const uint64_t mask_v = (bits_v >= 64) ? ~0ull : ((1ull << bits_v) - 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[i]) continue;
    const uint32_t j = pos[i];
    const uint64_t k = key[i];
    eu[j] = (int32_t)(k >> bits_v);
    ev[j] = (int32_t)(k & mask_v);
    es[j] = sign[idx[i]];
  }
}

// deg[id] += 1 for every lane with ok, as one atomic per run of equal ids in
// consecutive lanes (edges that arrive grouped by an endpoint form long runs).
__device__ __forceinline__ void add_runs(int32_t* __restrict__ deg, int32_t id, bool ok) {
  const unsigned lane = lane_id();
  const int32_t x = ok ? id : -1;
  const int32_t prev = __shfl_up_sync(kFullMask, x, 1);
  const bool head = lane == 0 || prev != x;
  const unsigned heads = __ballot_sync(kFullMask, head);
  const unsigned later = lane == 31 ? 0u : heads & (~0u << (lane + 1));
  const int len = (later ? __ffs(later) - 1 : 32) - (int)lane;
  if (ok && head) atomicAdd(&deg[x], len);
}

// Degrees over unified ids (V ids follow the U ids).
__global__ void degree_kernel(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev, int64_t m,
                              int32_t n_u, int32_t* __restrict__ deg) {
  constexpr int kRound = 4;  // edges per thread per round, their loads in flight together
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (m + stride - 1) / stride;  // the same for every lane: the warp votes together
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t it = 0; it < iters; it += kRound) {
    int32_t a[kRound], b[kRound];
#pragma unroll
    for (int j = 0; j < kRound; j++) {
      const int64_t i = (it + j) * stride + t0;
      a[j] = i < m ? eu[i] : 0;
      b[j] = i < m ? n_u + ev[i] : 0;
    }
#pragma unroll
    for (int j = 0; j < kRound; j++) {
      const bool ok = (it + j) * stride + t0 < m;
      add_runs(deg, a[j], ok);
      add_runs(deg, b[j], ok);
    }
  }
}

// Sort key per vertex: (side, component, degree, id within the component).
// Ascending order is the Def. 3 priority within each side of each component
// (V ids follow U ids in the unified space); components occupy contiguous
// rank ranges, which keeps a component's accepted endpoints together.
__global__ void vertex_keys_kernel(const int32_t* __restrict__ deg, int64_t n, int32_t n_u, int bits_comp,
                                   int bits_deg, int bits_id, UnionView un, uint64_t* __restrict__ key) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t side = x >= n_u ? 1 : 0;
    const int64_t sid = side ? x - n_u : x;
    const int64_t* off = side ? un.voff : un.uoff;
    const int32_t c = component_of(off, un.n_graphs, sid);
    const uint64_t local = (uint64_t)(sid - off[c]);
    key[x] = (side << (bits_comp + bits_deg + bits_id)) | ((uint64_t)c << (bits_deg + bits_id)) |
             ((uint64_t)deg[x] << bits_id) | local;
  }
}

__global__ void ranks_kernel(const uint64_t* __restrict__ skey, int64_t n, int32_t n_u, int bits_comp, int bits_deg,
                             int bits_id, UnionView un, int32_t* __restrict__ vertex, int32_t* __restrict__ side_rank,
                             int32_t* __restrict__ rowdeg) {
  const uint64_t id_mask = (1ull << bits_id) - 1, deg_mask = (1ull << bits_deg) - 1;
  const uint64_t comp_mask = (1ull << bits_comp) - 1;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = skey[r];
    const bool side = (k >> (bits_comp + bits_deg + bits_id)) & 1;
    const int32_t c = bits_comp ? (int32_t)((k >> (bits_deg + bits_id)) & comp_mask) : 0;
    const int64_t local = (int64_t)(k & id_mask);
    const int32_t x = side ? (int32_t)(n_u + un.voff[c] + local) : (int32_t)(un.uoff[c] + local);
    if (!DBBC_CHECK(x >= 0 && x < n)) continue;
    vertex[r] = x;
    side_rank[x] = side ? (int32_t)(r - n_u) : (int32_t)r;
    rowdeg[r] = (int32_t)((k >> bits_id) & deg_mask);
  }
}

// CSR keys in two sorts. The U rows are the edges sorted by
// ku = (U rank << (bits_v + 1)) | (V rank << 1) | negative; the V rows are the
// same list re-sorted stably by V rank alone, as
// kv = (V rank << (bits_u + 1)) | (U rank << 1) | negative, which keeps every
// V row ascending by U rank.
__global__ void csr_u_keys_kernel(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                                  const int8_t* __restrict__ es, int64_t m, int32_t n_u,
                                  const int32_t* __restrict__ side_rank, int bits_v, uint64_t* __restrict__ ku) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t ru = (uint32_t)side_rank[eu[i]];
    const uint64_t rv = (uint32_t)side_rank[n_u + ev[i]];
    ku[i] = (ru << (bits_v + 1)) | (rv << 1) | (es[i] < 0 ? 1u : 0u);
  }
}

// V keys of the U-sorted list, each with its U position (the edge's position
// in its U row) as the value the V sort carries along.
__global__ void csr_v_keys_kernel(const uint64_t* __restrict__ ku, int64_t m, int bits_u, int bits_v,
                                  uint64_t* __restrict__ kv, uint32_t* __restrict__ upos) {
  const uint64_t mask_v = (1ull << bits_v) - 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = ku[i];
    const uint64_t ru = k >> (bits_v + 1), rv = (k >> 1) & mask_v;
    kv[i] = (rv << (bits_u + 1)) | (ru << 1) | (k & 1u);
    upos[i] = (uint32_t)i;
  }
}

// Flags a repeated (u, v) pair: U-sorted keys that agree in everything but the
// sign bit are adjacent.
__global__ void adjacent_dup_kernel(const uint64_t* __restrict__ key, int64_t m, unsigned* dup) {
  bool any = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i + 1 < m; i += (int64_t)gridDim.x * blockDim.x)
    any |= (key[i] >> 1) == (key[i + 1] >> 1);
  if (__any_sync(kFullMask, any) && lane_id() == 0) atomicOr(dup, 1u);
}

// Row and entry of CSR position i: the first m positions are the U rows, the
// next m the V rows.
struct CsrKeys {
  const uint64_t* ku;
  const uint64_t* kv;
  const uint32_t* upos;  // upos[k]: the U position of the edge at V position m + k
  int64_t m;
  int32_t n_u;
  int bits_u, bits_v;
  __device__ __forceinline__ int64_t row(int64_t i) const {
    return i < m ? (int64_t)(ku[i] >> (bits_v + 1)) : (int64_t)n_u + (int64_t)(kv[i - m] >> (bits_u + 1));
  }
  __device__ __forceinline__ uint32_t entry(int64_t i) const {
    return i < m ? (uint32_t)(ku[i] & ((2ull << bits_v) - 1)) : (uint32_t)(kv[i - m] & ((2ull << bits_u) - 1));
  }
};

__global__ void csr_cols_kernel(CsrKeys ck, int64_t nnz, uint32_t* __restrict__ col) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x)
    col[i] = ck.entry(i);
}

// lower[r] = neighbours of row r with lower Def. 3 priority. A U vertex of
// degree d is above a V vertex iff deg(v) < d (equal degree: the V id is
// larger); a V vertex of degree d is above a U vertex iff deg(u) <= d.
// Neighbours lie in the row's own component, whose other-side ranks ascend by
// degree, and rows list neighbours by ascending side rank, so the lower ones
// are a prefix.
__global__ void lower_kernel(const int64_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
                             const int32_t* __restrict__ rowdeg, int64_t n, int32_t n_u, UnionView un,
                             uint32_t* __restrict__ lower) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = rowdeg[r];
    int64_t t;  // side rank threshold in the other side
    if (r < n_u) {
      const int32_t c = component_of(un.uoff, un.n_graphs, r);
      const int64_t b = un.voff[c], e = un.voff[c + 1];
      t = b + lower_bound_dev<int32_t>(rowdeg + n_u + b, e - b, d);
    } else {
      const int32_t c = component_of(un.voff, un.n_graphs, r - n_u);
      const int64_t b = un.uoff[c], e = un.uoff[c + 1];
      t = b + upper_bound_dev<int32_t>(rowdeg + b, e - b, d);
    }
    const int64_t b = row_ptr[r];
    lower[r] = (uint32_t)lower_bound_dev<uint32_t>(col + b, row_ptr[r + 1] - b, (uint32_t)(t << 1));
  }
}

// work[p] = sum over lower neighbours v of p of |{w in row(v) : rank(w) < rank(p)}|,
// i.e. the wedges Algorithm 1 accepts at pivot p. Every edge appears as the
// entry at V position m + k (row v, index idx_v in it) and at U position
// upos[k] (row u, index idx_u); rows ascend by rank, so idx_v entries of
// row(v) rank below u and idx_u entries of row(u) rank below v. A lower
// neighbour v of u (idx_u < lower[u]) thus adds idx_v to work[u], and a lower
// neighbour u of v (idx_v < lower[v]) adds idx_u to work[v]. Edges are taken
// in V order, 32 consecutive ones per warp: the V rows' sums are merged by a
// segmented warp sum, the U rows' go to their rows directly.
__global__ void work_kernel(CsrKeys ck, const int64_t* __restrict__ row_ptr, const uint32_t* __restrict__ lower,
                            unsigned long long* __restrict__ work) {
  constexpr int kRound = 4;  // edges per thread per round, their loads in flight together
  const int64_t m = ck.m;
  const uint64_t mask_u = (1ull << ck.bits_u) - 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (m + stride - 1) / stride;  // the same for every lane: the warp shuffles together
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = lane_id();
  for (int64_t it = 0; it < iters; it += kRound) {
    uint64_t key[kRound];
    uint32_t up[kRound];
#pragma unroll
    for (int j = 0; j < kRound; j++) {
      const int64_t k = (it + j) * stride + t0;
      key[j] = k < m ? ck.kv[k] : 0;
      up[j] = k < m ? ck.upos[k] : 0;
    }
    int64_t v[kRound], ru[kRound];
    uint64_t idx_v[kRound], idx_u[kRound];
    uint32_t low_u[kRound], low_v[kRound];
#pragma unroll
    for (int j = 0; j < kRound; j++) {
      const int64_t k = (it + j) * stride + t0;
      ru[j] = (int64_t)((key[j] >> 1) & mask_u);
      v[j] = -1;
      idx_v[j] = idx_u[j] = 0;
      low_u[j] = low_v[j] = 0;
      if (k < m) {
        v[j] = (int64_t)ck.n_u + (int64_t)(key[j] >> (ck.bits_u + 1));
        idx_v[j] = (uint64_t)(m + k - row_ptr[v[j]]);
        idx_u[j] = (uint64_t)((int64_t)up[j] - row_ptr[ru[j]]);
        low_u[j] = lower[ru[j]];
        low_v[j] = lower[v[j]];
      }
    }
#pragma unroll
    for (int j = 0; j < kRound; j++) {
      if (v[j] >= 0 && idx_u[j] < low_u[j] && idx_v[j]) atomicAdd(&work[ru[j]], (unsigned long long)idx_v[j]);
      uint64_t acc = (v[j] >= 0 && idx_v[j] < low_v[j]) ? idx_u[j] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_down_sync(kFullMask, acc, o);
        const int64_t v2 = __shfl_down_sync(kFullMask, v[j], o);
        if (lane + o < 32 && v2 == v[j]) acc += y;
      }
      const int64_t vp = __shfl_up_sync(kFullMask, v[j], 1);
      if (v[j] >= 0 && acc && (lane == 0 || vp != v[j])) atomicAdd(&work[v[j]], (unsigned long long)acc);
    }
  }
}

struct PrepStats {
  unsigned long long wedges, wedges_hub, wedges_medium, wedges_light, max_work;
  unsigned long long n_piv, n_hub, n_medium;
  unsigned long long lower_hub, lower_medium, lower_light;
};

// Pivots that can close a butterfly: at least two lower neighbours and at
// least one accepted wedge. (A pivot with a single lower neighbour v reaches
// every endpoint w at most once, so all its buckets stay below 2.)
__global__ void pivot_flags_kernel(const uint64_t* __restrict__ work, const uint32_t* __restrict__ lower, int64_t n,
                                   uint64_t light_max, uint64_t medium_max, uint32_t* __restrict__ flag,
                                   PrepStats* st) {
  uint64_t w_all = 0, w_hub = 0, w_med = 0, w_light = 0, mx = 0, np = 0, nh = 0, nm = 0;
  uint64_t l_hub = 0, l_med = 0, l_light = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t w = work[r];
    w_all += w;
    const bool piv = lower[r] >= 2 && w > 0;
    flag[r] = piv ? 1u : 0u;
    if (piv) {
      np++;
      mx = w > mx ? w : mx;
      const uint64_t L = lower[r];
      if (w > medium_max) { nh++; w_hub += w; l_hub += L; }
      else if (w > light_max) { nm++; w_med += w; l_med += L; }
      else { w_light += w; l_light += L; }
    }
  }
  w_all = warp_sum_u64(w_all);
  w_hub = warp_sum_u64(w_hub);
  w_med = warp_sum_u64(w_med);
  w_light = warp_sum_u64(w_light);
  np = warp_sum_u64(np);
  nh = warp_sum_u64(nh);
  nm = warp_sum_u64(nm);
  l_hub = warp_sum_u64(l_hub);
  l_med = warp_sum_u64(l_med);
  l_light = warp_sum_u64(l_light);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t y = __shfl_xor_sync(kFullMask, mx, o);
    mx = y > mx ? y : mx;
  }
  if (lane_id() == 0) {
    if (w_all) atomicAdd(&st->wedges, (unsigned long long)w_all);
    if (w_hub) atomicAdd(&st->wedges_hub, (unsigned long long)w_hub);
    if (w_med) atomicAdd(&st->wedges_medium, (unsigned long long)w_med);
    if (w_light) atomicAdd(&st->wedges_light, (unsigned long long)w_light);
    if (mx) atomicMax(&st->max_work, (unsigned long long)mx);
    if (np) atomicAdd(&st->n_piv, (unsigned long long)np);
    if (nh) atomicAdd(&st->n_hub, (unsigned long long)nh);
    if (nm) atomicAdd(&st->n_medium, (unsigned long long)nm);
    if (l_hub) atomicAdd(&st->lower_hub, (unsigned long long)l_hub);
    if (l_med) atomicAdd(&st->lower_medium, (unsigned long long)l_med);
    if (l_light) atomicAdd(&st->lower_light, (unsigned long long)l_light);
  }
}

// Descending-work sort key for pivot rows: (2^bits - 1 - work) ascending.
__global__ void pivot_keys_kernel(const uint64_t* __restrict__ work, const uint32_t* __restrict__ flag,
                                  const uint32_t* __restrict__ pos, int64_t n, int bits, uint64_t* __restrict__ key,
                                  uint32_t* __restrict__ row) {
  const uint64_t top = bits >= 64 ? ~0ull : ((1ull << bits) - 1);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[r]) continue;
    const uint32_t j = pos[r];
    key[j] = top - work[r];
    row[j] = (uint32_t)r;
  }
}

// Per side, how many vertices have degree below each of four limits (ranks
// ascend by degree within a side): out[2k] for U, out[2k + 1] for V.
struct DegreeLimits {
  int32_t d[4];
};
__global__ void narrow_ranks_kernel(const int32_t* __restrict__ rowdeg, int64_t n, int32_t n_u, DegreeLimits lim,
                                    int64_t* out) {
  const int t = threadIdx.x;
  if (t < 8) {
    const bool u = (t & 1) == 0;
    out[t] = u ? lower_bound_dev<int32_t>(rowdeg, n_u, lim.d[t >> 1])
               : lower_bound_dev<int32_t>(rowdeg + n_u, n - n_u, lim.d[t >> 1]);
  }
}

// Union of several graphs: graph i's local ids are validated against its own
// sides and shifted by the sizes of the graphs before it.
__global__ void union_ids_kernel(const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                 const int8_t* __restrict__ s, const int64_t* __restrict__ eoff,
                                 const int32_t* __restrict__ nu, const int32_t* __restrict__ nv,
                                 const int64_t* __restrict__ uoff, const int64_t* __restrict__ voff, int32_t n_graphs,
                                 int32_t* __restrict__ ou, int32_t* __restrict__ ov, int8_t* __restrict__ os,
                                 unsigned* err) {
  unsigned e = 0;
  for (int32_t gi = blockIdx.x; gi < n_graphs; gi += gridDim.x) {
    const int64_t e0 = eoff[gi], e1 = eoff[gi + 1];
    const int32_t a = nu[gi], b = nv[gi];
    const int32_t du = (int32_t)uoff[gi], dv = (int32_t)voff[gi];
    for (int64_t i = e0 + threadIdx.x; i < e1; i += blockDim.x) {
      const int32_t x = u[i], y = v[i];
      const int8_t c = s[i];
      if (x < 0 || x >= a) e |= 1u;
      if (y < 0 || y >= b) e |= 2u;
      if (c != 1 && c != -1) e |= 4u;
      ou[i] = x + du;
      ov[i] = y + dv;
      os[i] = c;
    }
  }
  e = __reduce_or_sync(kFullMask, e);
  if (lane_id() == 0 && e) atomicOr(err, e);
}

// Component of every row of a union: the graph whose id range holds the
// row's vertex.
__global__ void component_kernel(const int32_t* __restrict__ vertex, int64_t n, int32_t n_u_total,
                                 const int64_t* __restrict__ uoff, const int64_t* __restrict__ voff, int32_t n_graphs,
                                 int32_t* __restrict__ comp) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = vertex[r];
    const bool is_u = x < n_u_total;
    const int64_t key = is_u ? x : (int64_t)x - n_u_total;
    const int64_t* off = is_u ? uoff : voff;
    comp[r] = (int32_t)upper_bound_dev<int64_t>(off, (int64_t)n_graphs + 1, key) - 1;
  }
}

__global__ void gather_u32_kernel(const uint32_t* __restrict__ src, const uint32_t* __restrict__ idx, int64_t n,
                                  uint32_t* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}
__global__ void gather_u64_kernel(const uint64_t* __restrict__ src, const uint32_t* __restrict__ idx, int64_t n,
                                  uint64_t* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

// ------------------------------------------------------------------ host
static unsigned grid_for(int64_t n, int threads = 256) {
  int64_t b = ceil_div<int64_t>(n > 0 ? n : 1, threads);
  const int64_t cap = (int64_t)kNumSMs * 16;
  return (unsigned)(b < cap ? b : cap);
}

void* graph_alloc(dbbc_graph* g, size_t bytes) {
  void* p = dev_alloc(bytes ? bytes : 16, g->stream);
  if (!p) throw Error{DBBC_ENOMEM, "graph_alloc"};
  g->allocations.push_back(p);
  g->device_bytes += bytes;
  return p;
}

void free_graph_memory(dbbc_graph* g) {
  for (void* p : g->allocations) dev_free(p, g->stream);
  g->allocations.clear();
  g->device_bytes = 0;
}

template <typename T>
static T read_back(const T* d, cudaStream_t s) {
  T h;
  DBBC_CUDA(cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, s));
  DBBC_CUDA(cudaStreamSynchronize(s));
  return h;
}

static void plan_hubs(dbbc_graph* g, cudaStream_t s, const UnionSpec& un) {
  if (g->n_hub == 0) return;
  std::vector<uint32_t> rows((size_t)g->n_hub), lows((size_t)g->n_hub);
  std::vector<uint64_t> works((size_t)g->n_hub);
  {
    Scratch sc(s);
    uint32_t* d_low = sc.get<uint32_t>((size_t)g->n_hub);
    uint64_t* d_work = sc.get<uint64_t>((size_t)g->n_hub);
    const uint32_t* d_rows = reinterpret_cast<const uint32_t*>(g->order);
    gather_u32_kernel<<<grid_for(g->n_hub), 256, 0, s>>>(g->lower, d_rows, g->n_hub, d_low);
    DBBC_LAUNCH_CHECK();
    gather_u64_kernel<<<grid_for(g->n_hub), 256, 0, s>>>(g->work, d_rows, g->n_hub, d_work);
    DBBC_LAUNCH_CHECK();
    DBBC_CUDA(cudaMemcpyAsync(rows.data(), d_rows, rows.size() * 4, cudaMemcpyDeviceToHost, s));
    DBBC_CUDA(cudaMemcpyAsync(lows.data(), d_low, lows.size() * 4, cudaMemcpyDeviceToHost, s));
    DBBC_CUDA(cudaMemcpyAsync(works.data(), d_work, works.size() * 8, cudaMemcpyDeviceToHost, s));
    DBBC_CUDA(cudaStreamSynchronize(s));
  }
  // Split each hub's accepted ranks [0, sp) into items of roughly equal work.
  // Ranks below the side's first endpoint of degree >= 2^16 use narrow
  // counters (16-bit halves) unless the hub has < 2^16 lower neighbours, in
  // which case every count fits 16 bits. An item that does not start at rank
  // 0 pays one binary search per lower neighbour, so items stay large against
  // the hub's lower-neighbour count.
  struct Planned {
    SweepItem it;
    uint64_t est;
  };
  std::vector<Planned> plan;
  int64_t max_lower = 1;
  for (size_t h = 0; h < rows.size(); h++) {
    const int32_t row = (int32_t)rows[h];
    const uint32_t L = lows[h];
    const uint64_t W = works[h];
    const bool is_u = row < g->n_u;
    const uint64_t sp = is_u ? (uint64_t)row : (uint64_t)(row - g->n_u);
    // the hub's accepted endpoints are the ranks of its own component below it
    const std::vector<int64_t>& off = is_u ? un.uoff : un.voff;
    const uint64_t start =
        (uint64_t)off[(size_t)(std::upper_bound(off.begin(), off.end(), (int64_t)sp) - off.begin() - 1)];
    // counter widths by the counts they must hold: a count never exceeds the
    // endpoint's degree nor the hub's lower-neighbour count L. Ranks ascend by
    // degree, so quarter (4-bit halves) counters serve the ranks below the
    // side's first endpoint of degree >= 2^4, tiny (8-bit) ones those below
    // degree 2^8 and narrow (16-bit) ones those below degree 2^16; for a union,
    // whose ranks are component-major, only L bounds the counts. Endpoints of
    // degree 0 (the lowest ranks) are in no row, so the windows start after
    // them.
    auto clamp_rank = [&](int64_t x) {
      return std::max<uint64_t>(start, std::min<uint64_t>(sp, (uint64_t)std::max<int64_t>(x, 0)));
    };
    const bool plain = un.n_graphs == 1;
    const uint64_t first = plain ? clamp_rank(is_u ? g->zero_ranks_u : g->zero_ranks_v) : start;
    const uint64_t quarter_end = L < (uint32_t)kQuarterCountLimit ? sp
                                 : plain ? std::max<uint64_t>(first, clamp_rank(is_u ? g->quarter_ranks_u
                                                                                     : g->quarter_ranks_v))
                                         : first;
    const uint64_t tiny_end = L < (uint32_t)kTinyCountLimit ? sp
                              : plain ? std::max<uint64_t>(quarter_end, clamp_rank(is_u ? g->tiny_ranks_u
                                                                                        : g->tiny_ranks_v))
                                      : quarter_end;
    const uint64_t narrow_end =
        L < (uint32_t)kNarrowCountLimit ? sp
        : plain ? std::max<uint64_t>(tiny_end, clamp_rank(is_u ? g->narrow_ranks_u : g->narrow_ranks_v))
                : tiny_end;
    const uint64_t H4 = 4ull * kSweepWindow16, H8 = 2ull * kSweepWindow16;
    const uint64_t Rq = (quarter_end - first + H4 - 1) / H4;
    const uint64_t Rt = (tiny_end - quarter_end + H8 - 1) / H8;
    const uint64_t Rn = (narrow_end - tiny_end + kSweepWindow16 - 1) / kSweepWindow16;
    const uint64_t Rw = (sp - narrow_end + kSweepWindow32 - 1) / kSweepWindow32;
    const uint64_t target = std::max<uint64_t>(g->tune.hub_item_work, 64ull * L);
    max_lower = std::max<int64_t>(max_lower, L);
    // lanes per (neighbour, window) segment from the hub's mean segment length
    const double density = (double)W / ((double)L * (double)std::max<uint64_t>(1, Rq + Rt + Rn + Rw));
    const double* gd = g->tune.group_density;
    const int16_t dense_log = density >= gd[0] ? 5 : density >= gd[1] ? 4 : density >= gd[2] ? 3 : density >= gd[3] ? 2 : 0;
    // sparse hubs sweep in list mode: one item per hub, run in spans of at
    // most Rsub windows whose lists (plus two overflow lists of L slots) fit
    // the per-CTA list scratch
    const uint64_t per_nb = (uint64_t)kListCapEntries / std::max<uint32_t>(L, 1);
    const uint64_t Rsub = per_nb >= 3 ? std::min<uint64_t>(kListMaxWindows, per_nb - 2) : 0;
    const uint64_t R_all = Rq + Rt + Rn + Rw;
    const bool listed = density < g->tune.list_density && Rsub >= 1 && R_all >= 2;
    // the first rank of window w of the hub (windows numbered in rank order
    // over the quarter, tiny, narrow and wide parts)
    auto window_start = [&](uint64_t w) -> uint64_t {
      if (w < Rq) return first + w * H4;
      if (w < Rq + Rt) return quarter_end + (w - Rq) * H8;
      if (w < Rq + Rt + Rn) return tiny_end + (w - Rq - Rt) * kSweepWindow16;
      return std::min<uint64_t>(sp, narrow_end + (w - Rq - Rt - Rn) * kSweepWindow32);
    };
    // items of roughly `target` wedges over consecutive windows (one item in
    // list mode); an item crosses width boundaries freely
    const uint64_t spans = listed ? 1 : std::max<uint64_t>(1, std::min<uint64_t>(R_all, W / target));
    for (uint64_t k = 0; k < spans && R_all > 0; k++) {
      const uint64_t w0 = R_all * k / spans, w1 = R_all * (k + 1) / spans;
      if (w1 <= w0) continue;
      Planned p;
      p.it.row = row;
      p.it.lo = (uint32_t)window_start(w0);
      p.it.hi = (uint32_t)(w1 == R_all ? sp : window_start(w1));
      p.it.q_end = (uint32_t)quarter_end;
      p.it.t_end = (uint32_t)tiny_end;
      p.it.n_end = (uint32_t)narrow_end;
      // list-mode items take list_group_log lanes per segment, at least 8 when
      // their mean segment reaches list_wide_density
      const int16_t list_log = (int16_t)(density >= g->tune.list_wide_density
                                             ? std::max<int32_t>(3, g->tune.list_group_log)
                                             : g->tune.list_group_log);
      p.it.group_log = listed ? list_log : dense_log;
      p.it.flags = listed ? kItemList : 0;
      // dense items: finalise each window from its counters when clearing it
      if ((double)W / (double)R_all >= (double)g->tune.finalize_window_wedges) p.it.flags |= kItemFinalize;
      if (w0 == 0) p.it.flags |= kItemFirst;
      p.est = std::max<uint64_t>(1, W / spans);
      plan.push_back(p);
      const int64_t R = (int64_t)(w1 - w0);
      g->hub_cursor_inits += L;
      if (listed)
        g->sweep_list_cap = std::max<int64_t>(g->sweep_list_cap, (std::min<int64_t>(R, (int64_t)Rsub) + 2) * (int64_t)L);
      else g->hub_cursor_steps += (int64_t)L * R;
    }
  }
  std::stable_sort(plan.begin(), plan.end(), [](const Planned& a, const Planned& b) { return a.est > b.est; });
  std::vector<SweepItem> items(plan.size());
  g->sweep_est_host.resize(plan.size());
  for (size_t i = 0; i < plan.size(); i++) {
    items[i] = plan[i].it;
    g->sweep_est_host[i] = plan[i].est;
  }
  g->sweep_items_host = items;
  g->n_sweep_items = (int64_t)items.size();
  g->sweep_max_lower = max_lower;
  g->sweep_items = static_cast<SweepItem*>(graph_alloc(g, items.size() * sizeof(SweepItem)));
  DBBC_CUDA(cudaMemcpyAsync(g->sweep_items, items.data(), items.size() * sizeof(SweepItem), cudaMemcpyHostToDevice,
                            s));
  DBBC_CUDA(cudaStreamSynchronize(s));
}

void build_graph_multi(dbbc_graph* g, const int32_t* u, const int32_t* v, const int8_t* sgn,
                       const int64_t* edge_offsets, const int32_t* n_u, const int32_t* n_v, int32_t n_graphs,
                       bool on_device, bool reject_duplicates, cudaStream_t s) {
  // host metadata: edge ranges and the id shift of every graph
  std::vector<int64_t> uoff((size_t)n_graphs + 1, 0), voff((size_t)n_graphs + 1, 0);
  for (int32_t i = 0; i < n_graphs; i++) {
    if (n_u[i] < 0 || n_v[i] < 0 || edge_offsets[i + 1] < edge_offsets[i])
      throw Error{DBBC_EINVAL, "bad component sizes or edge offsets"};
    uoff[(size_t)i + 1] = uoff[(size_t)i] + n_u[i];
    voff[(size_t)i + 1] = voff[(size_t)i] + n_v[i];
  }
  const int64_t m = edge_offsets[n_graphs] - edge_offsets[0];
  if (edge_offsets[0] != 0 || m >= (int64_t{1} << 31) || uoff.back() + voff.back() >= (int64_t{1} << 31))
    throw Error{DBBC_EINVAL, "union too large"};
  g->n_u = (int32_t)uoff.back();
  g->n_v = (int32_t)voff.back();
  Scratch sc(s);
  const int32_t* du = u;
  const int32_t* dv = v;
  const int8_t* ds = sgn;
  if (!on_device && m > 0) {
    int32_t* tu = sc.get<int32_t>((size_t)m);
    int32_t* tv = sc.get<int32_t>((size_t)m);
    int8_t* ts = sc.get<int8_t>((size_t)m);
    DBBC_CUDA(cudaMemcpyAsync(tu, u, (size_t)m * 4, cudaMemcpyHostToDevice, s));
    DBBC_CUDA(cudaMemcpyAsync(tv, v, (size_t)m * 4, cudaMemcpyHostToDevice, s));
    DBBC_CUDA(cudaMemcpyAsync(ts, sgn, (size_t)m, cudaMemcpyHostToDevice, s));
    du = tu;
    dv = tv;
    ds = ts;
  }
  int64_t* d_meta = sc.get<int64_t>((size_t)3 * (n_graphs + 1));
  int32_t* d_n = sc.get<int32_t>((size_t)2 * n_graphs + 2);
  std::vector<int32_t> nn((size_t)2 * n_graphs + 2, 0);
  std::copy(n_u, n_u + n_graphs, nn.begin());
  std::copy(n_v, n_v + n_graphs, nn.begin() + n_graphs);
  DBBC_CUDA(cudaMemcpyAsync(d_meta, edge_offsets, (size_t)(n_graphs + 1) * 8, cudaMemcpyHostToDevice, s));
  DBBC_CUDA(cudaMemcpyAsync(d_meta + n_graphs + 1, uoff.data(), uoff.size() * 8, cudaMemcpyHostToDevice, s));
  DBBC_CUDA(cudaMemcpyAsync(d_meta + 2 * (n_graphs + 1), voff.data(), voff.size() * 8, cudaMemcpyHostToDevice, s));
  DBBC_CUDA(cudaMemcpyAsync(d_n, nn.data(), nn.size() * 4, cudaMemcpyHostToDevice, s));
  int32_t* ou = sc.get<int32_t>((size_t)std::max<int64_t>(m, 1));
  int32_t* ov = sc.get<int32_t>((size_t)std::max<int64_t>(m, 1));
  int8_t* os = sc.get<int8_t>((size_t)std::max<int64_t>(m, 1));
  unsigned* d_err = sc.get<unsigned>(1);
  DBBC_CUDA(cudaMemsetAsync(d_err, 0, sizeof(unsigned), s));
  if (n_graphs > 0 && m > 0) {
    union_ids_kernel<<<(unsigned)std::min<int32_t>(n_graphs, 65535), 256, 0, s>>>(
        du, dv, ds, d_meta, d_n, d_n + n_graphs, d_meta + n_graphs + 1, d_meta + 2 * (n_graphs + 1), n_graphs, ou, ov,
        os, d_err);
    DBBC_LAUNCH_CHECK();
    if (read_back(d_err, s) != 0) throw Error{DBBC_EINVAL, "invalid edge id or sign"};
  }
  UnionSpec un;
  un.n_graphs = std::max<int32_t>(n_graphs, 1);
  un.uoff = n_graphs > 0 ? uoff : std::vector<int64_t>{0, 0};
  un.voff = n_graphs > 0 ? voff : std::vector<int64_t>{0, 0};
  un.d_uoff = n_graphs > 0 ? d_meta + n_graphs + 1 : nullptr;
  un.d_voff = n_graphs > 0 ? d_meta + 2 * (n_graphs + 1) : nullptr;
  for (int32_t i = 0; i < n_graphs; i++) un.max_side = std::max<int64_t>(un.max_side, std::max(n_u[i], n_v[i]));
  if (n_graphs == 0) {
    int64_t* d = sc.get<int64_t>(4);
    DBBC_CUDA(cudaMemsetAsync(d, 0, 32, s));
    un.d_uoff = d;
    un.d_voff = d + 2;
  }
  build_graph(g, ou, ov, os, m, true, reject_duplicates, s, &un);
  g->n_components = n_graphs;
  g->component = static_cast<int32_t*>(graph_alloc(g, (size_t)std::max<int64_t>(g->n, 1) * 4));
  if (g->n > 0) {
    component_kernel<<<grid_for(g->n), 256, 0, s>>>(g->vertex, g->n, g->n_u, d_meta + n_graphs + 1,
                                                    d_meta + 2 * (n_graphs + 1), n_graphs, g->component);
    DBBC_LAUNCH_CHECK();
  }
  DBBC_CUDA(cudaStreamSynchronize(s));
}

void build_graph(dbbc_graph* g, const int32_t* u_in, const int32_t* v_in, const int8_t* s_in, int64_t m,
                 bool on_device, bool reject_duplicates, cudaStream_t s, const UnionSpec* union_spec) {
  const int32_t n_u = g->n_u, n_v = g->n_v;
  const int64_t n = (int64_t)n_u + n_v;
  g->n = n;
  g->m_input = m;
  g->tune = current_tuning();
  Scratch sc(s);
  // a plain graph is a union of one component
  UnionSpec plain;
  const UnionSpec* un = union_spec;
  if (!un) {
    plain.uoff = {0, (int64_t)n_u};
    plain.voff = {0, (int64_t)n_v};
    plain.max_side = std::max<int64_t>(n_u, n_v);
    int64_t* d = sc.get<int64_t>(4);
    DBBC_CUDA(cudaMemcpyAsync(d, plain.uoff.data(), 16, cudaMemcpyHostToDevice, s));
    DBBC_CUDA(cudaMemcpyAsync(d + 2, plain.voff.data(), 16, cudaMemcpyHostToDevice, s));
    plain.d_uoff = d;
    plain.d_voff = d + 2;
    un = &plain;
  }
  const UnionView uv{un->d_uoff, un->d_voff, un->n_graphs};

  // ---- inputs on the device
  const int32_t* du = u_in;
  const int32_t* dv = v_in;
  const int8_t* ds = s_in;
  if (!on_device && m > 0) {
    int32_t* tu = sc.get<int32_t>((size_t)m);
    int32_t* tv = sc.get<int32_t>((size_t)m);
    int8_t* ts = sc.get<int8_t>((size_t)m);
    DBBC_CUDA(cudaMemcpyAsync(tu, u_in, (size_t)m * 4, cudaMemcpyHostToDevice, s));
    DBBC_CUDA(cudaMemcpyAsync(tv, v_in, (size_t)m * 4, cudaMemcpyHostToDevice, s));
    DBBC_CUDA(cudaMemcpyAsync(ts, s_in, (size_t)m, cudaMemcpyHostToDevice, s));
    du = tu;
    dv = tv;
    ds = ts;
  }
  unsigned* d_flags = sc.get<unsigned>(4);
  DBBC_CUDA(cudaMemsetAsync(d_flags, 0, 4 * sizeof(unsigned), s));

  // ---- a1: validate
  if (m > 0) {
    validate_kernel<<<grid_for(m), 256, 0, s>>>(du, dv, ds, m, n_u, n_v, d_flags);
    DBBC_LAUNCH_CHECK();
    if (read_back(d_flags, s) != 0) throw Error{DBBC_EINVAL, "invalid edge id or sign"};
  }

  const int bits_u = bits_for(n_u > 0 ? (uint64_t)(n_u - 1) : 0);
  const int bits_v = bits_for(n_v > 0 ? (uint64_t)(n_v - 1) : 0);
  // rank keys: (side, component, degree, id within the component)
  const int bits_comp = un->n_graphs > 1 ? bits_for((uint64_t)(un->n_graphs - 1)) : 0;
  const int bits_lid = std::max(1, bits_for(un->max_side > 0 ? (uint64_t)(un->max_side - 1) : 0));
  const int bits_deg = std::max(1, bits_for((uint64_t)un->max_side));
  if (1 + bits_comp + bits_deg + bits_lid > 64) throw Error{DBBC_EINVAL, "union too large for 64-bit rank keys"};
  int32_t* deg = sc.get<int32_t>((size_t)n);
  int32_t* side_rank = sc.get<int32_t>((size_t)n);
  int32_t* rowdeg = sc.get<int32_t>((size_t)n);
  uint64_t* vk0 = sc.get<uint64_t>((size_t)n);
  uint64_t* vk1 = sc.get<uint64_t>((size_t)n);
  uint64_t* ck0 = sc.get<uint64_t>((size_t)(2 * m));
  uint64_t* ck1 = sc.get<uint64_t>((size_t)(2 * m));
  g->vertex = static_cast<int32_t*>(graph_alloc(g, (size_t)n * 4));
  g->row_ptr = static_cast<int64_t*>(graph_alloc(g, (size_t)(n + 1) * 8));

  // a2 + a3 for an edge list: degrees, Def. 3 ranks per side, and the CSR
  // keys of both sides (CsrKeys: U rows sorted by (U rank, V rank), V rows
  // by (V rank, U rank)) with the sign in bit 0. Returns the keys and whether
  // any (u, v) pair occurs twice (adjacent U keys).
  auto csr_from_edges = [&](const int32_t* eu, const int32_t* ev, const int8_t* es, int64_t me,
                            bool* dup) -> CsrKeys {
    DBBC_CUDA(cudaMemsetAsync(deg, 0, (size_t)n * 4, s));
    if (me > 0) {
      degree_kernel<<<grid_for(me), 256, 0, s>>>(eu, ev, me, n_u, deg);
      DBBC_LAUNCH_CHECK();
    }
    if (n > 0) {
      vertex_keys_kernel<<<grid_for(n), 256, 0, s>>>(deg, n, n_u, bits_comp, bits_deg, bits_lid, uv, vk0);
      DBBC_LAUNCH_CHECK();
      // keys are generated in (side, component, local id) order, so a stable
      // sort on (side, component, degree) alone leaves equal degrees by id
      const bool alt = radix_sort<uint64_t, uint32_t, false>(vk0, vk1, nullptr, nullptr, n, bits_lid,
                                                             1 + bits_comp + bits_deg + bits_lid, s, sc);
      ranks_kernel<<<grid_for(n), 256, 0, s>>>(alt ? vk1 : vk0, n, n_u, bits_comp, bits_deg, bits_lid, uv,
                                               g->vertex, side_rank, rowdeg);
      DBBC_LAUNCH_CHECK();
    }
    *dup = false;
    CsrKeys k{ck0, ck0 + me, nullptr, me, n_u, bits_u, bits_v};
    if (me == 0) return k;
    // the halves of ck0 / ck1 hold the U keys and the V keys; the sorts skip
    // bit 0 (the sign), so repeated pairs stay in input order
    csr_u_keys_kernel<<<grid_for(me), 256, 0, s>>>(eu, ev, es, me, n_u, side_rank, bits_v, ck0);
    DBBC_LAUNCH_CHECK();
    const bool alt_u = radix_sort<uint64_t, uint32_t, false>(ck0, ck1, nullptr, nullptr, me, 1, 1 + bits_v + bits_u,
                                                             s, sc);
    k.ku = alt_u ? ck1 : ck0;
    DBBC_CUDA(cudaMemsetAsync(d_flags + 3, 0, sizeof(unsigned), s));
    adjacent_dup_kernel<<<grid_for(me), 256, 0, s>>>(k.ku, me, d_flags + 3);
    DBBC_LAUNCH_CHECK();
    uint32_t* up0 = sc.get<uint32_t>((size_t)me);
    uint32_t* up1 = sc.get<uint32_t>((size_t)me);
    csr_v_keys_kernel<<<grid_for(me), 256, 0, s>>>(k.ku, me, bits_u, bits_v, ck0 + me, up0);
    DBBC_LAUNCH_CHECK();
    const bool alt_v = radix_sort<uint64_t, uint32_t, true>(ck0 + me, ck1 + me, up0, up1, me, 1 + bits_u,
                                                            1 + bits_u + bits_v, s, sc);
    k.kv = alt_v ? ck1 + me : ck0 + me;
    k.upos = alt_v ? up1 : up0;
    *dup = read_back(d_flags + 3, s) != 0;
    return k;
  };

  // ---- a1-a3: build straight from the input; only when some (u, v) pair
  // repeats, drop all but its latest occurrence (stable sort on (u, v), keep
  // the last of every run) and build again from the distinct edges.
  bool dup = false;
  int64_t mu = m;
  CsrKeys ck = csr_from_edges(du, dv, ds, m, &dup);
  if (dup) {
    if (reject_duplicates) throw Error{DBBC_EINVAL, "duplicate edge under DBBC_DUP_REJECT"};
    uint64_t* k0 = ck0;  // reuse the CSR key buffers (2m entries each) for the (u, v) sort
    uint64_t* k1 = ck1;
    uint32_t* i0 = sc.get<uint32_t>((size_t)m);
    uint32_t* i1 = sc.get<uint32_t>((size_t)m);
    edge_keys_kernel<<<grid_for(m), 256, 0, s>>>(du, dv, m, bits_v, k0, i0);
    DBBC_LAUNCH_CHECK();
    const bool alt = radix_sort<uint64_t, uint32_t, true>(k0, k1, i0, i1, m, 0, bits_u + bits_v, s, sc);
    const uint64_t* ks = alt ? k1 : k0;
    const uint32_t* is = alt ? i1 : i0;
    uint32_t* flag = alt ? i0 : i1;  // the free index buffer
    uint32_t* pos = sc.get<uint32_t>((size_t)m);
    run_last_kernel<<<grid_for(m), 256, 0, s>>>(ks, m, flag, d_flags + 1);
    DBBC_LAUNCH_CHECK();
    exclusive_scan<uint32_t, uint32_t>(flag, pos, m, s, sc, reinterpret_cast<uint32_t*>(d_flags + 2));
    mu = read_back(d_flags + 2, s);
    int32_t* eu = sc.get<int32_t>((size_t)mu);
    int32_t* ev = sc.get<int32_t>((size_t)mu);
    int8_t* es = sc.get<int8_t>((size_t)mu);
    compact_edges_kernel<<<grid_for(m), 256, 0, s>>>(ks, is, flag, pos, ds, m, bits_v, eu, ev, es);
    DBBC_LAUNCH_CHECK();
    ck = csr_from_edges(eu, ev, es, mu, &dup);
    if (dup) throw Error{DBBC_EINTERNAL, "duplicates left after deduplication"};
  }
  g->m = mu;
  g->nnz = 2 * mu;
  g->col = static_cast<uint32_t*>(graph_alloc(g, (size_t)g->nnz * 4));
  g->lower = static_cast<uint32_t*>(graph_alloc(g, (size_t)n * 4));
  g->work = static_cast<uint64_t*>(graph_alloc(g, (size_t)n * 8));
  exclusive_scan<int32_t, int64_t>(rowdeg, g->row_ptr, n, s, sc, g->row_ptr + n);
  DBBC_CUDA(cudaMemsetAsync(g->work, 0, (size_t)n * 8, s));
  if (g->nnz > 0) {
    csr_cols_kernel<<<grid_for(g->nnz), 256, 0, s>>>(ck, g->nnz, g->col);
    DBBC_LAUNCH_CHECK();
  }
  if (n > 0) {
    lower_kernel<<<grid_for(n), 256, 0, s>>>(g->row_ptr, g->col, rowdeg, n, n_u, uv, g->lower);
    DBBC_LAUNCH_CHECK();
  }

  // ---- a4: accepted wedges per pivot and the counting tiers
  if (g->nnz > 0) {
    work_kernel<<<grid_for(g->m), 256, 0, s>>>(ck, g->row_ptr, g->lower,
                                               reinterpret_cast<unsigned long long*>(g->work));
    DBBC_LAUNCH_CHECK();
  }
  PrepStats* d_st = sc.get<PrepStats>(1);
  DBBC_CUDA(cudaMemsetAsync(d_st, 0, sizeof(PrepStats), s));
  uint32_t* pflag = sc.get<uint32_t>((size_t)std::max<int64_t>(n, 1));
  if (n > 0) {
    pivot_flags_kernel<<<grid_for(n), 256, 0, s>>>(g->work, g->lower, n, g->tune.light_max_work,
                                                   g->tune.medium_max_work, pflag, d_st);
    DBBC_LAUNCH_CHECK();
  }
  const PrepStats st = read_back(d_st, s);
  g->wedges = st.wedges;
  g->wedges_hub = st.wedges_hub;
  g->wedges_medium = st.wedges_medium;
  g->wedges_light = st.wedges_light;
  g->n_piv = (int64_t)st.n_piv;
  g->n_hub = (int64_t)st.n_hub;
  g->n_medium = (int64_t)st.n_medium;
  g->n_light = g->n_piv - g->n_hub - g->n_medium;
  g->lower_hub = (int64_t)st.lower_hub;
  g->lower_medium = (int64_t)st.lower_medium;
  g->lower_light = (int64_t)st.lower_light;
  g->order = static_cast<int32_t*>(graph_alloc(g, (size_t)std::max<int64_t>(g->n_piv, 1) * 4));
  if (g->n_piv > 0) {
    uint32_t* ppos = sc.get<uint32_t>((size_t)n);
    exclusive_scan<uint32_t, uint32_t>(pflag, ppos, n, s, sc);
    const int wbits = std::max(1, bits_for(st.max_work));
    uint64_t* pk0 = sc.get<uint64_t>((size_t)g->n_piv);
    uint64_t* pk1 = sc.get<uint64_t>((size_t)g->n_piv);
    uint32_t* pr0 = reinterpret_cast<uint32_t*>(g->order);
    uint32_t* pr1 = sc.get<uint32_t>((size_t)g->n_piv);
    pivot_keys_kernel<<<grid_for(n), 256, 0, s>>>(g->work, pflag, ppos, n, wbits, pk0, pr0);
    DBBC_LAUNCH_CHECK();
    const bool alt = radix_sort<uint64_t, uint32_t, true>(pk0, pk1, pr0, pr1, g->n_piv, 0, wbits, s, sc);
    if (alt)
      DBBC_CUDA(cudaMemcpyAsync(pr0, pr1, (size_t)g->n_piv * 4, cudaMemcpyDeviceToDevice, s));
  }
  // per side: how many vertices have degree < 2^16, < 2^8, < 2^4 and 0
  // (ranks ascend by degree)
  {
    int64_t* d_t = sc.get<int64_t>(8);
    const DegreeLimits lim{{kNarrowCountLimit, kTinyCountLimit, kQuarterCountLimit, 1}};
    narrow_ranks_kernel<<<1, 32, 0, s>>>(rowdeg, n, n_u, lim, d_t);
    DBBC_LAUNCH_CHECK();
    int64_t ht[8];
    DBBC_CUDA(cudaMemcpyAsync(ht, d_t, sizeof(ht), cudaMemcpyDeviceToHost, s));
    DBBC_CUDA(cudaStreamSynchronize(s));
    g->narrow_ranks_u = ht[0];
    g->narrow_ranks_v = ht[1];
    g->tiny_ranks_u = ht[2];
    g->tiny_ranks_v = ht[3];
    g->quarter_ranks_u = ht[4];
    g->quarter_ranks_v = ht[5];
    g->zero_ranks_u = ht[6];
    g->zero_ranks_v = ht[7];
  }
  plan_hubs(g, s, *un);
  DBBC_CUDA(cudaStreamSynchronize(s));
}

}  // namespace dbbc
