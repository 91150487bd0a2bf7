// Signed wedge aggregation (Algorithm 1, Phase 5) and the per-endpoint
// finalisation of Lemma 1, in three tiers chosen by a pivot's accepted wedges:
//
//   light  : one warp per pivot, open-addressing hash in the warp's slice of
//            shared memory (packed u64 counter per endpoint: low 32 bits
//            symmetric wedges B1, high 32 bits asymmetric wedges B2);
//   medium : one CTA per pivot, a larger shared hash shared by its warps;
//   hub    : work items (pivot, range of lower neighbours) spread over all
//            CTAs; a dense global u64 counter array per concurrently counted
//            hub plus a list of touched endpoints for the reset.
//
// Each pivot p walks its lower neighbours v (a prefix of its CSR row) and,
// for each, the prefix of v's row whose entries rank below p, so every wedge
// it reads is accepted.
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

__device__ __forceinline__ int table_log(uint64_t work, int max_log) {
  // smallest 2^k >= 2 * work, at least 32 slots
  int k = 5;
  while (k < max_log && (1ull << k) < 2 * work) k++;
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
  q.rb = g.row_ptr[p];
  q.L = g.lower[p];
  const bool is_u = p < g.n_u;
  q.lim = (is_u ? (uint32_t)p : (uint32_t)(p - g.n_u)) << 1;
  q.base = is_u ? (int64_t)g.n_u : 0;
  return q;
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
      const int64_t vrow = q.base + (e >> 1);
      vb = g.row_ptr[vrow];
      ve = g.row_ptr[vrow + 1];
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

// ------------------------------------------------------------------ light tier
constexpr int kLightWarps = 8;

__global__ void __launch_bounds__(kLightWarps * 32) count_light_kernel(CsrView g, const int32_t* __restrict__ piv,
                                                                       const uint64_t* __restrict__ work, int64_t n_piv,
                                                                       unsigned long long* out, unsigned* status) {
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
  constexpr int max_log = 10;  // log2(kLightSlots)
  uint64_t bal = 0, unb = 0;
  bool full = false;
  const int64_t nw = (int64_t)gridDim.x * kLightWarps;
  for (int64_t t = (int64_t)blockIdx.x * kLightWarps + w; t < n_piv; t += nw) {
    const int32_t p = piv[t];
    const int log_h = table_log(work[p], max_log);
    const PivotGeom q = pivot_geom(g, p);
    warp_walk<1>(g, q, 0, q.L, 32, [&](const uint32_t (&x)[1], uint32_t s1) {
      if (x[0] != 0xFFFFFFFFu) {
        const unsigned long long inc = wedge_inc(x[0], s1);
        unsigned long long old;
        if (smem_hash_add(keys, vals, log_h, x[0] >> 1, inc, &old)) wedge_contrib(old, inc, bal, unb);
        else full = true;
      }
    });
    __syncwarp();
    for (int i = lane; i < (1 << log_h); i += 32) {
      keys[i] = kEmptyKey;
      vals[i] = 0;
    }
    __syncwarp();
  }
  if (full) atomicOr(status, DBBC_DEV_HASH_FULL);
  block_add_pair<kLightWarps * 32>(bal, unb, out);
}

// ------------------------------------------------------------------ medium tier
constexpr int kMediumThreads = 256;
constexpr int kMediumWarps = kMediumThreads / 32;

__global__ void __launch_bounds__(kMediumThreads) count_medium_kernel(CsrView g, const int32_t* __restrict__ piv,
                                                                      const uint64_t* __restrict__ work,
                                                                      int64_t n_piv, unsigned long long* out,
                                                                      unsigned* status) {
  extern __shared__ __align__(16) unsigned char med_smem[];
  unsigned long long* vals = reinterpret_cast<unsigned long long*>(med_smem);
  uint32_t* keys = reinterpret_cast<uint32_t*>(vals + kMediumSlots);
  for (int i = threadIdx.x; i < kMediumSlots; i += kMediumThreads) {
    keys[i] = kEmptyKey;
    vals[i] = 0;
  }
  __syncthreads();
  constexpr int max_log = 13;  // log2(kMediumSlots)
  const int w = threadIdx.x >> 5;
  uint64_t bal = 0, unb = 0;
  bool full = false;
  for (int64_t t = blockIdx.x; t < n_piv; t += gridDim.x) {
    const int32_t p = piv[t];
    const int log_h = table_log(work[p], max_log);
    const PivotGeom q = pivot_geom(g, p);
    warp_walk<2>(g, q, (uint32_t)w * 32u, q.L, kMediumWarps * 32u, [&](const uint32_t (&x)[2], uint32_t s1) {
#pragma unroll
      for (int u = 0; u < 2; u++) {
        if (x[u] != 0xFFFFFFFFu) {
          const unsigned long long inc = wedge_inc(x[u], s1);
          unsigned long long old;
          if (smem_hash_add(keys, vals, log_h, x[u] >> 1, inc, &old)) wedge_contrib(old, inc, bal, unb);
          else full = true;
        }
      }
    });
    __syncthreads();
    for (int i = threadIdx.x; i < (1 << log_h); i += kMediumThreads) {
      keys[i] = kEmptyKey;
      vals[i] = 0;
    }
    __syncthreads();
  }
  if (full) atomicOr(status, DBBC_DEV_HASH_FULL);
  block_add_pair<kMediumThreads>(bal, unb, out);
}

// ------------------------------------------------------------------ hub tier
// Window sweep. A hub pivot's accepted endpoints [0, side_rank(p)) are cut
// into windows of kSweepWindow16 (or kSweepWindow32) consecutive side ranks. A
// work item is one hub and a span of its windows, owned by one CTA, so the
// counts of every endpoint in a window are complete inside that CTA: they live
// in shared memory, and the Lemma 1 contributions come from the value each
// atomic returns. Each lower neighbour v keeps a cursor into its row; rows
// ascend, so sweeping the windows in order moves every cursor forward only.
// Counters pack (asym << 16) | sym when the hub has fewer than 2^16 lower
// neighbours (no count can exceed that), else (asym << 32) | sym.
constexpr int kSweepThreads = DBBC_SWEEP_THREADS;
constexpr int kSweepUnroll = DBBC_SWEEP_UNROLL;

__device__ __forceinline__ void sweep_contrib16(uint32_t old, bool sym, uint64_t& bal, uint64_t& unb) {
  const uint64_t p = old & 0xFFFFu, q = old >> 16;
  bal += sym ? p : q;
  unb += sym ? q : p;
}

// One window of one item: every group of G lanes takes lower neighbours
// gid, gid + groups, ... and walks the neighbour's row from its cursor, G
// consecutive entries at a time, until an entry leaves the window.
template <int G, bool PACK16>
__device__ __forceinline__ void sweep_window(const CsrView& g, const PivotGeom& q, int64_t* cur, uint32_t lo,
                                             uint32_t hl, uint32_t* c16, unsigned long long* c32, uint64_t& bal,
                                             uint64_t& unb) {
  const int tid = threadIdx.x;
  const int gl = tid & (G - 1);
  const uint32_t gid = (uint32_t)tid / G;
  constexpr uint32_t groups = kSweepThreads / G;
  const unsigned lane = lane_id();
  const unsigned gmask = G == 32 ? kFullMask : (((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));
  const uint32_t lo2 = lo << 1;
  // the next neighbour's cursor and edge sign are loaded while this one is walked
  int64_t c_nx = 0, en_nx = 0;
  uint32_t s1_nx = 0;
  if (gid < q.L) {
    c_nx = cur[2 * gid];
    en_nx = cur[2 * gid + 1];
    s1_nx = g.col[q.rb + gid] & 1u;
  }
  for (uint32_t i = gid; i < q.L; i += groups) {
    int64_t c = c_nx;
    const int64_t en = en_nx;
    const uint32_t s1 = s1_nx;
    const uint32_t i_nx = i + groups;
    if (i_nx < q.L) {
      c_nx = cur[2 * i_nx];
      en_nx = cur[2 * i_nx + 1];
      s1_nx = g.col[q.rb + i_nx] & 1u;
    }
    for (;;) {
      uint32_t x[kSweepUnroll];
#pragma unroll
      for (int u = 0; u < kSweepUnroll; u++) {
        const int64_t pos = c + u * G + gl;
        x[u] = pos < en ? g.col[pos] : 0xFFFFFFFFu;
      }
      int n_ok = 0;
#pragma unroll
      for (int u = 0; u < kSweepUnroll; u++) {
        const bool ok = x[u] < hl;
        if (ok) {
          const bool sym = ((x[u] ^ s1) & 1u) == 0;
          const uint32_t k = (x[u] - lo2) >> 1;
          if (PACK16) {
            sweep_contrib16(atomicAdd(&c16[k], sym ? 1u : 0x10000u), sym, bal, unb);
          } else {
            const unsigned long long inc = sym ? 1ull : (1ull << 32);
            wedge_contrib(atomicAdd(&c32[k], inc), inc, bal, unb);
          }
        }
        n_ok += __popc(__ballot_sync(gmask, ok));  // accepted entries are a prefix
      }
      c += n_ok;
      if (n_ok < G * kSweepUnroll) break;
    }
    if (gl == 0) cur[2 * i] = c;
  }
}

template <bool PACK16>
__device__ __forceinline__ void sweep_window_dispatch(int group_log, const CsrView& g, const PivotGeom& q,
                                                      int64_t* cur, uint32_t lo, uint32_t hl, uint32_t* c16,
                                                      unsigned long long* c32, uint64_t& bal, uint64_t& unb) {
  switch (group_log) {
    case 0: sweep_window<1, PACK16>(g, q, cur, lo, hl, c16, c32, bal, unb); break;
    case 2: sweep_window<4, PACK16>(g, q, cur, lo, hl, c16, c32, bal, unb); break;
    case 3: sweep_window<8, PACK16>(g, q, cur, lo, hl, c16, c32, bal, unb); break;
    case 4: sweep_window<16, PACK16>(g, q, cur, lo, hl, c16, c32, bal, unb); break;
    default: sweep_window<32, PACK16>(g, q, cur, lo, hl, c16, c32, bal, unb); break;
  }
}

__global__ void __launch_bounds__(kSweepThreads) hub_sweep_kernel(CsrView g, const SweepItem* __restrict__ items,
                                                                      int64_t n_items, int* next_item,
                                                                      int64_t* __restrict__ cursors, int64_t cur_cap,
                                                                      unsigned long long* out) {
  extern __shared__ __align__(16) unsigned char sweep_smem[];
  uint32_t* c16 = reinterpret_cast<uint32_t*>(sweep_smem);
  unsigned long long* c32 = reinterpret_cast<unsigned long long*>(sweep_smem);
  __shared__ int item_sh;
  const int tid = threadIdx.x;
  for (int i = tid; i < (int)kSweepWindow16; i += kSweepThreads) c16[i] = 0u;
  int64_t* cur = cursors + (int64_t)blockIdx.x * cur_cap * 2;
  uint64_t bal = 0, unb = 0;
  for (;;) {
    if (tid == 0) item_sh = atomicAdd(next_item, 1);
    __syncthreads();  // also orders the zeroing above / below before reuse
    const int64_t it = item_sh;
    __syncthreads();
    if (it >= n_items) break;
    const SweepItem item = items[it];
    const PivotGeom q = pivot_geom(g, item.row);
    const bool wide = item.wide != 0;
    const uint32_t H = wide ? kSweepWindow32 : kSweepWindow16;
    // cursors: first entry at or after rank item.lo, and the row end
    const uint32_t first = item.lo << 1;
    for (uint32_t i = tid; i < q.L; i += kSweepThreads) {
      const uint32_t e = g.col[q.rb + i];
      const int64_t vrow = q.base + (e >> 1);
      int64_t b = g.row_ptr[vrow];
      const int64_t en = g.row_ptr[vrow + 1];
      if (first) {  // lower_bound of `first` in the row
        int64_t lo = b, hi = en;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (g.col[mid] < first) lo = mid + 1; else hi = mid;
        }
        b = lo;
      }
      cur[2 * i] = b;
      cur[2 * i + 1] = en;
    }
    __syncthreads();
    for (uint32_t lo = item.lo; lo < item.hi; lo += H) {
      const uint32_t hi = min(lo + H, item.hi);
      if (wide) sweep_window_dispatch<false>(item.group_log, g, q, cur, lo, hi << 1, c16, c32, bal, unb);
      else sweep_window_dispatch<true>(item.group_log, g, q, cur, lo, hi << 1, c16, c32, bal, unb);
      __syncthreads();
      const uint32_t words = wide ? 2 * (hi - lo) : (hi - lo);  // 32-bit words to clear
      for (uint32_t j = tid; j < words; j += kSweepThreads) c16[j] = 0u;
      __syncthreads();
    }
  }
  block_add_pair<kSweepThreads>(bal, unb, out);
}

// ------------------------------------------------------------------ host
static int blocks_per_sm(const void* fn, int threads, size_t smem) {
  int b = 0;
  DBBC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem));
  return b > 0 ? b : 1;
}

static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    DBBC_CUDA(cudaGetDevice(&dev));
    DBBC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (sms <= 0) sms = kNumSMs;
  }
  return sms;
}

cudaEvent_t CountProfiler::begin(cudaStream_t s) {
  cudaEvent_t a;
  DBBC_CUDA(cudaEventCreate(&a));
  DBBC_CUDA(cudaEventRecord(a, s));
  return a;
}

void CountProfiler::end(int tier, cudaEvent_t a, cudaStream_t s) {
  cudaEvent_t b;
  DBBC_CUDA(cudaEventCreate(&b));
  DBBC_CUDA(cudaEventRecord(b, s));
  marks.push_back(Mark{tier, a, b});
}

void CountProfiler::summarize(dbbc_count_profile* out) {
  float ms[NTIERS] = {0, 0, 0, 0, 0};
  for (const Mark& mk : marks) {
    float t = 0;
    DBBC_CUDA(cudaEventElapsedTime(&t, mk.a, mk.b));
    ms[mk.tier] += t;
  }
  uint64_t touched = 0;
  for (uint32_t x : hub_touched) touched += x;
  out->ms_light = ms[LIGHT];
  out->ms_medium = ms[MEDIUM];
  out->ms_hub_aggregate = ms[HUB_AGG];
  out->ms_hub_finalize = ms[HUB_FIN];
  out->ms_total = ms[TOTAL];
  out->launches_light = launches[LIGHT];
  out->launches_medium = launches[MEDIUM];
  out->launches_hub_aggregate = launches[HUB_AGG];
  out->launches_hub_finalize = launches[HUB_FIN];
  out->hub_touched = touched;
}

CountProfiler::~CountProfiler() {
  for (const Mark& mk : marks) {
    cudaEventDestroy(mk.a);
    cudaEventDestroy(mk.b);
  }
}

void enqueue_count(const dbbc_graph* g, cudaStream_t s, unsigned long long* d_out, unsigned* d_status,
                   Scratch& sc, CountProfiler* prof) {
  if (g->n_piv == 0) return;
  const CsrView view{g->row_ptr, g->col, g->lower, g->n_u, g->n};
  const int sms = num_sms();
  cudaEvent_t t_all = prof ? prof->begin(s) : nullptr;
  cudaEvent_t t0 = nullptr;

  if (g->n_light > 0) {
    if (prof) t0 = prof->begin(s);
    const size_t smem = (size_t)kLightWarps * kLightSlots * 12;
    DBBC_CUDA(cudaFuncSetAttribute(count_light_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t want = ceil_div<int64_t>(g->n_light, kLightWarps);
    const int64_t cap = (int64_t)sms * blocks_per_sm((const void*)count_light_kernel, kLightWarps * 32, smem);
    count_light_kernel<<<(unsigned)std::min(want, cap), kLightWarps * 32, smem, s>>>(
        view, g->order + g->n_hub + g->n_medium, g->work, g->n_light, d_out, d_status);
    DBBC_LAUNCH_CHECK();
    if (prof) {
      prof->end(CountProfiler::LIGHT, t0, s);
      prof->launches[CountProfiler::LIGHT]++;
    }
  }
  if (g->n_medium > 0) {
    if (prof) t0 = prof->begin(s);
    const size_t smem = (size_t)kMediumSlots * 12;
    DBBC_CUDA(cudaFuncSetAttribute(count_medium_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t cap = (int64_t)sms * blocks_per_sm((const void*)count_medium_kernel, kMediumThreads, smem);
    count_medium_kernel<<<(unsigned)std::min<int64_t>(g->n_medium, cap), kMediumThreads, smem, s>>>(
        view, g->order + g->n_hub, g->work, g->n_medium, d_out, d_status);
    DBBC_LAUNCH_CHECK();
    if (prof) {
      prof->end(CountProfiler::MEDIUM, t0, s);
      prof->launches[CountProfiler::MEDIUM]++;
    }
  }
  if (g->n_hub > 0) {
    const size_t smem = (size_t)kSweepWindow16 * 4;
    DBBC_CUDA(cudaFuncSetAttribute(hub_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = sms * blocks_per_sm((const void*)hub_sweep_kernel, kSweepThreads, smem);
    int64_t* cursors = sc.get<int64_t>((size_t)grid * (size_t)g->sweep_max_lower * 2);
    int* next = sc.get<int>(1);
    DBBC_CUDA(cudaMemsetAsync(next, 0, sizeof(int), s));
    if (prof) t0 = prof->begin(s);
    hub_sweep_kernel<<<grid, kSweepThreads, smem, s>>>(view, g->sweep_items, g->n_sweep_items, next, cursors,
                                                       g->sweep_max_lower, d_out);
    DBBC_LAUNCH_CHECK();
    if (prof) {
      prof->end(CountProfiler::HUB_AGG, t0, s);
      prof->launches[CountProfiler::HUB_AGG]++;
    }
  }
  if (prof) prof->end(CountProfiler::TOTAL, t_all, s);
}

}  // namespace dbbc

namespace dbbc {

// The kernels of enqueue_count with all device scratch supplied by the caller:
// d_status (one word) and d_next (one int) are cleared here, and the hub
// sweep keeps its per-CTA cursors in `cursors` (cursor_bytes long), which
// bounds how many CTAs it can run. Throws DBBC_EOVERFLOW when not even one
// CTA's cursors fit.
void enqueue_count_prealloc(const dbbc_graph* g, cudaStream_t s, unsigned long long* d_out, unsigned* d_status,
                            int* d_next, int64_t* cursors, size_t cursor_bytes) {
  DBBC_CUDA(cudaMemsetAsync(d_status, 0, sizeof(unsigned), s));
  DBBC_CUDA(cudaMemsetAsync(d_out, 0, 2 * sizeof(unsigned long long), s));
  if (g->n_piv == 0) return;
  const CsrView view{g->row_ptr, g->col, g->lower, g->n_u, g->n};
  const int sms = num_sms();
  int64_t hub_grid = 0;
  if (g->n_hub > 0) {
    const size_t per_cta = (size_t)g->sweep_max_lower * 2 * sizeof(int64_t);
    hub_grid = (int64_t)(cursor_bytes / per_cta);
    if (hub_grid < 1) throw Error{DBBC_EOVERFLOW, "hub cursors exceed the fixed scratch"};
  }
  if (g->n_light > 0) {
    const size_t smem = (size_t)kLightWarps * kLightSlots * 12;
    DBBC_CUDA(cudaFuncSetAttribute(count_light_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t want = ceil_div<int64_t>(g->n_light, kLightWarps);
    const int64_t cap = (int64_t)sms * blocks_per_sm((const void*)count_light_kernel, kLightWarps * 32, smem);
    count_light_kernel<<<(unsigned)std::min(want, cap), kLightWarps * 32, smem, s>>>(
        view, g->order + g->n_hub + g->n_medium, g->work, g->n_light, d_out, d_status);
    DBBC_LAUNCH_CHECK();
  }
  if (g->n_medium > 0) {
    const size_t smem = (size_t)kMediumSlots * 12;
    DBBC_CUDA(cudaFuncSetAttribute(count_medium_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t cap = (int64_t)sms * blocks_per_sm((const void*)count_medium_kernel, kMediumThreads, smem);
    count_medium_kernel<<<(unsigned)std::min<int64_t>(g->n_medium, cap), kMediumThreads, smem, s>>>(
        view, g->order + g->n_hub, g->work, g->n_medium, d_out, d_status);
    DBBC_LAUNCH_CHECK();
  }
  if (g->n_hub > 0) {
    const size_t smem = (size_t)kSweepWindow16 * 4;
    DBBC_CUDA(cudaFuncSetAttribute(hub_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t full = (int64_t)sms * blocks_per_sm((const void*)hub_sweep_kernel, kSweepThreads, smem);
    const int grid = (int)std::min<int64_t>(full, hub_grid);
    DBBC_CUDA(cudaMemsetAsync(d_next, 0, sizeof(int), s));
    hub_sweep_kernel<<<grid, kSweepThreads, smem, s>>>(view, g->sweep_items, g->n_sweep_items, d_next, cursors,
                                                       g->sweep_max_lower, d_out);
    DBBC_LAUNCH_CHECK();
  }
}

}  // namespace dbbc
