// Signed wedge aggregation (Algorithm 1, Phase 5) and the per-endpoint
// finalisation of Lemma 1, in three tiers chosen by a pivot's accepted wedges:
//
//   light  : one warp per pivot, open-addressing hash in the warp's slice of
//            shared memory (packed u64 counter per endpoint: low 32 bits
//            symmetric wedges B1, high 32 bits asymmetric wedges B2);
//   medium : one CTA per pivot, a larger shared hash shared by its warps;
//   hub    : window sweep: a work item is a hub and a range of its endpoint
//            ranks, owned by one CTA, whose counters for one window of ranks
//            live in shared memory while per-neighbour cursors walk the rows.
//
// Each pivot p walks its lower neighbours v (a prefix of its CSR row) and,
// for each, the prefix of v's row whose entries rank below p, so every wedge
// it reads is accepted.
#include "sweep_device.cuh"

namespace dbbc {

// ------------------------------------------------------------------ light tier
// Each warp's table has 2^slots_log slots (at most kLightSlots).
__global__ void __launch_bounds__(kLightWarps * 32) count_light_kernel(CsrView g, const int32_t* __restrict__ piv,
                                                                       const uint64_t* __restrict__ work, int64_t n_piv,
                                                                       int hash_mult_log, int slots_log,
                                                                       unsigned long long* out, unsigned* status) {
  extern __shared__ __align__(16) unsigned char light_smem[];
  const int slots = 1 << slots_log;
  unsigned long long* vals_all = reinterpret_cast<unsigned long long*>(light_smem);
  uint32_t* keys_all = reinterpret_cast<uint32_t*>(vals_all + kLightWarps * slots);
  const int w = threadIdx.x >> 5;
  const unsigned lane = lane_id();
  uint32_t* keys = keys_all + w * slots;
  unsigned long long* vals = vals_all + w * slots;
  for (int i = lane; i < slots; i += 32) {
    keys[i] = kEmptyKey;
    vals[i] = 0;
  }
  __syncwarp();
  const int max_log = slots_log;
  uint64_t bal = 0, unb = 0;
  bool full = false;
  const int64_t nw = (int64_t)gridDim.x * kLightWarps;
  for (int64_t t = (int64_t)blockIdx.x * kLightWarps + w; t < n_piv; t += nw) {
    const int32_t p = piv[t];
    const int log_h = table_log(work[p], max_log, hash_mult_log);
    const PivotGeom q = pivot_geom(g, p);
    full |= !hash_walk_dispatch(hash_group_log(work[p], q.L, 5), lane, 32u, g, q, keys, vals, log_h, bal, unb);
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
// The CTA's table has 2^slots_log slots (at most kMediumSlots).
__global__ void __launch_bounds__(kMediumThreads) count_medium_kernel(CsrView g, const int32_t* __restrict__ piv,
                                                                      const uint64_t* __restrict__ work,
                                                                      int64_t n_piv, int hash_mult_log, int slots_log,
                                                                      unsigned long long* out, unsigned* status) {
  extern __shared__ __align__(16) unsigned char med_smem[];
  const int slots = 1 << slots_log;
  unsigned long long* vals = reinterpret_cast<unsigned long long*>(med_smem);
  uint32_t* keys = reinterpret_cast<uint32_t*>(vals + slots);
  for (int i = threadIdx.x; i < slots; i += kMediumThreads) {
    keys[i] = kEmptyKey;
    vals[i] = 0;
  }
  __syncthreads();
  const int max_log = slots_log;
  uint64_t bal = 0, unb = 0;
  bool full = false;
  for (int64_t t = blockIdx.x; t < n_piv; t += gridDim.x) {
    const int32_t p = piv[t];
    const int log_h = table_log(work[p], max_log, hash_mult_log);
    const PivotGeom q = pivot_geom(g, p);
    full |= !hash_walk_dispatch(hash_group_log(work[p], q.L, 5), threadIdx.x, (uint32_t)kMediumThreads, g, q, keys,
                                vals, log_h, bal, unb);
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
// Items are pulled dynamically in descending estimated work (LPT). An item in
// list mode (sweep_device.cuh) uses per-window neighbour lists in `lists`
// (list_cap slots per CTA); with no room for them (list_cap below three slots
// per lower neighbour) it is swept by cursors like every other item, which
// gives the same counts.
__global__ void __launch_bounds__(kSweepThreads) hub_sweep_kernel(CsrView g, const SweepItem* __restrict__ items,
                                                                      int64_t n_items, int* next_item,
                                                                      uint2* __restrict__ cursors, int64_t cur_cap,
                                                                      uint2* __restrict__ lists, int64_t list_cap,
                                                                      unsigned long long* out,
                                                                      unsigned long long* visits) {
  extern __shared__ __align__(16) unsigned char sweep_smem[];
  uint32_t* cnt_words = reinterpret_cast<uint32_t*>(sweep_smem);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sweep_smem);
  __shared__ int item_sh;
  __shared__ ListState ls;
  __shared__ uint32_t nbn[2];
  const int tid = threadIdx.x;
  zero_words(cnt_words, kSweepWords);
  if (tid < 2) nbn[tid] = 0u;
  uint2* cur = cursors + (int64_t)blockIdx.x * cur_cap;
  uint2* my_lists = lists ? lists + (int64_t)blockIdx.x * list_cap : nullptr;
  uint64_t bal = 0, unb = 0, n_visits = 0;
  for (;;) {
    if (tid == 0) item_sh = atomicAdd(next_item, 1);
    __syncthreads();  // also orders the clearing above / below before reuse
    const int64_t it = item_sh;
    __syncthreads();
    if (it >= n_items) break;
    const SweepItem item = items[it];
    const PivotGeom q = pivot_geom(g, item.row);
    const int64_t per_nb = q.L ? list_cap / (int64_t)q.L : 0;
    if ((item.flags & kItemList) != 0 && my_lists != nullptr && per_nb >= 3) {
      n_visits += sweep_list_item_dispatch(g, item, q, my_lists, list_cap, ls, sbase, cnt_words, nbn, bal, unb);
      continue;
    }
    const uint32_t L = DBBC_CHECK((int64_t)q.L <= cur_cap) ? q.L : 0u;  // checked builds: cursor capacity
    for (uint32_t i = tid; i < L; i += kSweepThreads) {
      uint32_t b, en, s1;
      lean_cursor_start(g, q, i, (item.flags & kItemFirst) ? 0u : item.lo, b, en, s1);
      cur[i] = lean_slot(b, en, s1);
    }
    __syncthreads();
    sweep_cursor_item_dispatch(item.group_log, g.col, L, cur, ItemWindows(item), (item.flags & kItemFinalize) != 0,
                               sbase, cnt_words, nbn, bal, unb);
  }
  block_add_pair<kSweepThreads>(bal, unb, out);
  if (visits && tid == 0 && n_visits) atomicAdd(visits, (unsigned long long)n_visits);
}

// ------------------------------------------------------------------ host
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
  if (d_visits) DBBC_CUDA(cudaMemcpy(&list_visits, d_visits, sizeof(list_visits), cudaMemcpyDeviceToHost));
  out->ms_light = ms[LIGHT];
  out->ms_medium = ms[MEDIUM];
  out->ms_hub_aggregate = ms[HUB_AGG];
  out->ms_hub_finalize = ms[HUB_FIN];
  out->ms_total = ms[TOTAL];
  out->launches_light = launches[LIGHT];
  out->launches_medium = launches[MEDIUM];
  out->launches_hub_aggregate = launches[HUB_AGG];
  out->launches_hub_finalize = launches[HUB_FIN];
  out->hub_list_visits = list_visits;
}

CountProfiler::~CountProfiler() {
  for (const Mark& mk : marks) {
    cudaEventDestroy(mk.a);
    cudaEventDestroy(mk.b);
  }
}

// Launches of the three tiers, shared by enqueue_count and
// enqueue_count_prealloc.
static void launch_light(const dbbc_graph* g, const CsrView& view, cudaStream_t s, unsigned long long* d_out,
                         unsigned* d_status) {
  const int slots_log = tier_slots_log(g->tune.light_max_work, g->tune.hash_mult_log, 10);
  const size_t smem = (size_t)kLightWarps * ((size_t)1 << slots_log) * 12;
  DBBC_CUDA(cudaFuncSetAttribute(count_light_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)kLightWarps * kLightSlots * 12)));
  const int64_t want = ceil_div<int64_t>(g->n_light, kLightWarps);
  const int64_t cap = (int64_t)num_sms() * blocks_per_sm((const void*)count_light_kernel, kLightWarps * 32, smem);
  count_light_kernel<<<(unsigned)std::min(want, cap), kLightWarps * 32, smem, s>>>(
      view, g->order + g->n_hub + g->n_medium, g->work, g->n_light, g->tune.hash_mult_log, slots_log, d_out,
      d_status);
  DBBC_LAUNCH_CHECK();
}

static void launch_medium(const dbbc_graph* g, const CsrView& view, cudaStream_t s, unsigned long long* d_out,
                          unsigned* d_status) {
  const int slots_log = tier_slots_log(g->tune.medium_max_work, g->tune.hash_mult_log, 13);
  const size_t smem = ((size_t)1 << slots_log) * 12;
  DBBC_CUDA(cudaFuncSetAttribute(count_medium_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)kMediumSlots * 12)));
  const int64_t cap = (int64_t)num_sms() * blocks_per_sm((const void*)count_medium_kernel, kMediumThreads, smem);
  count_medium_kernel<<<(unsigned)std::min<int64_t>(g->n_medium, cap), kMediumThreads, smem, s>>>(
      view, g->order + g->n_hub, g->work, g->n_medium, g->tune.hash_mult_log, slots_log, d_out, d_status);
  DBBC_LAUNCH_CHECK();
}

// CTAs the hub sweep can keep resident (one per SM: its counters fill the
// SM's shared memory).
static int64_t hub_full_grid() {
  DBBC_CUDA(cudaFuncSetAttribute(hub_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmem));
  return (int64_t)num_sms() * blocks_per_sm((const void*)hub_sweep_kernel, kSweepThreads, kSweepSmem);
}

// The hub sweep on `grid` CTAs with per-CTA cursors (sweep_max_lower each)
// and, if `lists` is given, per-CTA list scratch (sweep_list_cap slots each);
// `next` is the item counter, cleared here.
static void launch_hub(const dbbc_graph* g, const CsrView& view, cudaStream_t s, int grid, int* next,
                       uint2* cursors, uint2* lists, unsigned long long* d_out, unsigned long long* visits) {
  DBBC_CUDA(cudaMemsetAsync(next, 0, sizeof(int), s));
  hub_sweep_kernel<<<grid, kSweepThreads, kSweepSmem, s>>>(view, g->sweep_items, g->n_sweep_items, next, cursors,
                                                           g->sweep_max_lower, lists,
                                                           lists ? g->sweep_list_cap : 0, d_out, visits);
  DBBC_LAUNCH_CHECK();
}

void enqueue_count(const dbbc_graph* g, cudaStream_t s, unsigned long long* d_out, unsigned* d_status,
                   Scratch& sc, CountProfiler* prof) {
  if (g->n_piv == 0) return;
  const CsrView view{g->row_ptr, g->col, g->lower, g->n_u, g->n, g->nnz};
  cudaEvent_t t_all = prof ? prof->begin(s) : nullptr;
  cudaEvent_t t0 = nullptr;
  if (g->n_light > 0) {
    if (prof) t0 = prof->begin(s);
    launch_light(g, view, s, d_out, d_status);
    if (prof) {
      prof->end(CountProfiler::LIGHT, t0, s);
      prof->launches[CountProfiler::LIGHT]++;
    }
  }
  if (g->n_medium > 0) {
    if (prof) t0 = prof->begin(s);
    launch_medium(g, view, s, d_out, d_status);
    if (prof) {
      prof->end(CountProfiler::MEDIUM, t0, s);
      prof->launches[CountProfiler::MEDIUM]++;
    }
  }
  if (g->n_hub > 0) {
    const int grid = (int)hub_full_grid();
    uint2* cursors = sc.get<uint2>((size_t)grid * (size_t)g->sweep_max_lower);
    uint2* lists = g->sweep_list_cap > 0 ? sc.get<uint2>((size_t)grid * (size_t)g->sweep_list_cap) : nullptr;
    int* next = sc.get<int>(1);
    if (prof) {
      prof->d_visits = sc.get<unsigned long long>(1);
      DBBC_CUDA(cudaMemsetAsync(prof->d_visits, 0, sizeof(unsigned long long), s));
      t0 = prof->begin(s);
    }
    launch_hub(g, view, s, grid, next, cursors, lists, d_out, prof ? prof->d_visits : nullptr);
    if (prof) {
      prof->end(CountProfiler::HUB_AGG, t0, s);
      prof->launches[CountProfiler::HUB_AGG]++;
    }
  }
  if (prof) prof->end(CountProfiler::TOTAL, t_all, s);
}

// The kernels of enqueue_count with all device scratch supplied by the caller:
// d_status (one word) and d_next (one int) are cleared here, and the hub
// sweep keeps its per-CTA cursors (8 bytes per lower neighbour of the largest
// hub) in `cursors` (cursor_bytes long, 8-byte aligned), which bounds how many
// CTAs it can run; it runs without list scratch (cursor mode for every item,
// same counts). Throws DBBC_EOVERFLOW when not even one CTA's cursors fit.
void enqueue_count_prealloc(const dbbc_graph* g, cudaStream_t s, unsigned long long* d_out, unsigned* d_status,
                            int* d_next, uint32_t* cursors, size_t cursor_bytes) {
  DBBC_CUDA(cudaMemsetAsync(d_status, 0, sizeof(unsigned), s));
  DBBC_CUDA(cudaMemsetAsync(d_out, 0, 2 * sizeof(unsigned long long), s));
  if (g->n_piv == 0) return;
  const CsrView view{g->row_ptr, g->col, g->lower, g->n_u, g->n, g->nnz};
  int64_t hub_grid = 0;
  if (g->n_hub > 0) {
    const size_t per_cta = (size_t)g->sweep_max_lower * sizeof(uint2);
    hub_grid = (int64_t)(cursor_bytes / per_cta);
    if (hub_grid < 1) throw Error{DBBC_EOVERFLOW, "hub cursors exceed the fixed scratch"};
  }
  if (g->n_light > 0) launch_light(g, view, s, d_out, d_status);
  if (g->n_medium > 0) launch_medium(g, view, s, d_out, d_status);
  if (g->n_hub > 0) {
    const int grid = (int)std::min<int64_t>(hub_full_grid(), hub_grid);
    launch_hub(g, view, s, grid, d_next, reinterpret_cast<uint2*>(cursors), nullptr, d_out, nullptr);
  }
}

}  // namespace dbbc
