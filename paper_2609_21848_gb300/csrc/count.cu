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

__device__ __forceinline__ uint32_t hash_slot(uint32_t w, int log_h) {
  return (w * 2654435769u) >> (32 - log_h);
}

// Insert / find endpoint w in a shared table of 2^log_h slots and add inc.
// Returns false if the probe sequence ran past the table (cannot happen when
// the table has more slots than the pivot's accepted wedges).
__device__ __forceinline__ bool smem_hash_add(uint32_t* keys, unsigned long long* vals, int log_h, uint32_t w,
                                              unsigned long long inc) {
  const uint32_t mask = (1u << log_h) - 1u;
  uint32_t h = hash_slot(w, log_h);
  for (uint32_t probe = 0; probe <= mask; probe++) {
    uint32_t cur = *reinterpret_cast<volatile uint32_t*>(&keys[h]);
    if (cur == kEmptyKey) cur = atomicCAS(&keys[h], kEmptyKey, w);
    if (cur == kEmptyKey || cur == w) {
      atomicAdd(&vals[h], inc);
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
// 32 (`step` = distance between this warp's groups, in positions) and calls
// visit(w, inc) for every accepted wedge, lanes striding over each v's row.
template <typename Visit>
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
      for (int64_t jb = jb0; jb < je; jb += 32) {
        const int64_t j = jb + lane;
        const uint32_t x = j < je ? g.col[j] : 0xFFFFFFFFu;
        const bool ok = x < q.lim;
        if (ok) visit(x >> 1, wedge_inc(x, s1));
        if (__ballot_sync(kFullMask, !ok)) break;  // rows ascend: nothing accepted beyond
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
    warp_walk(g, q, 0, q.L, 32, [&](uint32_t x, unsigned long long inc) {
      full |= !smem_hash_add(keys, vals, log_h, x, inc);
    });
    __syncwarp();
    for (int i = lane; i < (1 << log_h); i += 32) {
      if (keys[i] != kEmptyKey) {
        pair_contrib(vals[i], bal, unb);
        keys[i] = kEmptyKey;
        vals[i] = 0;
      }
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
    warp_walk(g, q, (uint32_t)w * 32u, q.L, kMediumWarps * 32u, [&](uint32_t x, unsigned long long inc) {
      full |= !smem_hash_add(keys, vals, log_h, x, inc);
    });
    __syncthreads();
    for (int i = threadIdx.x; i < (1 << log_h); i += kMediumThreads) {
      if (keys[i] != kEmptyKey) {
        pair_contrib(vals[i], bal, unb);
        keys[i] = kEmptyKey;
        vals[i] = 0;
      }
    }
    __syncthreads();
  }
  if (full) atomicOr(status, DBBC_DEV_HASH_FULL);
  block_add_pair<kMediumThreads>(bal, unb, out);
}

// ------------------------------------------------------------------ hub tier
constexpr int kHubThreads = 256;
constexpr int kHubWarps = kHubThreads / 32;

// Pull (hub, lower-neighbour range) items and add every accepted wedge to the
// hub's dense counter array; the first increment of an endpoint appends it to
// the slot's touched list.
__global__ void __launch_bounds__(kHubThreads) hub_aggregate_kernel(CsrView g, const HubItem* __restrict__ items,
                                                                    int64_t n_items, unsigned long long* __restrict__ ctr,
                                                                    uint32_t* __restrict__ touched, int64_t stride,
                                                                    uint32_t* __restrict__ tcount, int* next_item) {
  __shared__ int item_sh;
  const int w = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) item_sh = atomicAdd(next_item, 1);
    __syncthreads();
    const int64_t it = item_sh;
    __syncthreads();
    if (it >= n_items) break;
    const HubItem item = items[it];
    const PivotGeom q = pivot_geom(g, item.row);
    unsigned long long* c = ctr + (int64_t)item.slot * stride;
    uint32_t* tl = touched + (int64_t)item.slot * stride;
    uint32_t* tc = tcount + item.slot;
    warp_walk(g, q, item.a + (uint32_t)w * 32u, item.b, kHubWarps * 32u, [&](uint32_t x, unsigned long long inc) {
      const unsigned long long old = atomicAdd(&c[x], inc);
      if (old == 0ull) tl[atomicAdd(tc, 1u)] = x;
    });
  }
}

// Finalise one wave: every touched endpoint of every slot adds its Lemma 1
// contribution and its counter is cleared for the next wave.
__global__ void __launch_bounds__(kHubThreads) hub_finalize_kernel(unsigned long long* __restrict__ ctr,
                                                                   const uint32_t* __restrict__ touched,
                                                                   int64_t stride, const uint32_t* __restrict__ tcount,
                                                                   unsigned long long* out) {
  const int slot = blockIdx.y;
  const uint32_t cnt = tcount[slot];
  unsigned long long* c = ctr + (int64_t)slot * stride;
  const uint32_t* tl = touched + (int64_t)slot * stride;
  uint64_t bal = 0, unb = 0;
  for (uint32_t i = blockIdx.x * kHubThreads + threadIdx.x; i < cnt; i += gridDim.x * kHubThreads) {
    const uint32_t x = tl[i];
    pair_contrib(c[x], bal, unb);
    c[x] = 0;
  }
  block_add_pair<kHubThreads>(bal, unb, out);
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
    const int64_t slots = g->hub_slots, stride = g->hub_stride;
    const int64_t waves = (int64_t)g->hub_wave_begin.size() - 1;
    unsigned long long* ctr = sc.get<unsigned long long>((size_t)(slots * stride));
    uint32_t* touched = sc.get<uint32_t>((size_t)(slots * stride));
    uint32_t* tcount = sc.get<uint32_t>((size_t)(waves * slots));
    int* next = sc.get<int>((size_t)waves);
    DBBC_CUDA(cudaMemsetAsync(ctr, 0, (size_t)(slots * stride) * 8, s));
    DBBC_CUDA(cudaMemsetAsync(tcount, 0, (size_t)(waves * slots) * 4, s));
    DBBC_CUDA(cudaMemsetAsync(next, 0, (size_t)waves * 4, s));
    const int agg_blocks = sms * blocks_per_sm((const void*)hub_aggregate_kernel, kHubThreads, 0);
    const unsigned fin_x = (unsigned)std::max<int64_t>(1, (int64_t)sms * 4 / slots);
    for (int64_t wv = 0; wv < waves; wv++) {
      const int64_t i0 = g->hub_wave_begin[(size_t)wv], i1 = g->hub_wave_begin[(size_t)wv + 1];
      const int64_t n_items = i1 - i0;
      const unsigned blocks = (unsigned)std::min<int64_t>(n_items, agg_blocks);
      if (prof) t0 = prof->begin(s);
      hub_aggregate_kernel<<<blocks, kHubThreads, 0, s>>>(view, g->hub_items + i0, n_items, ctr, touched, stride,
                                                         tcount + wv * slots, next + wv);
      DBBC_LAUNCH_CHECK();
      if (prof) {
        prof->end(CountProfiler::HUB_AGG, t0, s);
        prof->launches[CountProfiler::HUB_AGG]++;
        t0 = prof->begin(s);
      }
      const int64_t wave_slots = std::min<int64_t>(slots, g->n_hub - wv * slots);
      hub_finalize_kernel<<<dim3(fin_x, (unsigned)wave_slots), kHubThreads, 0, s>>>(ctr, touched, stride,
                                                                                    tcount + wv * slots, d_out);
      DBBC_LAUNCH_CHECK();
      if (prof) {
        prof->end(CountProfiler::HUB_FIN, t0, s);
        prof->launches[CountProfiler::HUB_FIN]++;
      }
    }
    if (prof) {
      prof->hub_touched.resize((size_t)(waves * slots));
      DBBC_CUDA(cudaMemcpyAsync(prof->hub_touched.data(), tcount, (size_t)(waves * slots) * 4,
                                cudaMemcpyDeviceToHost, s));
    }
  }
  if (prof) prof->end(CountProfiler::TOTAL, t_all, s);
}

}  // namespace dbbc
