// Batched counting of many resident graphs. A batch plan concatenates the
// graphs' light and medium pivot lists and their hub items (the latter in
// descending estimated work across all graphs, i.e. LPT order) into one work
// list; one light, one medium and one hub-sweep kernel then serve every
// graph, each adding its sums into that graph's output pair. The sequence is
// captured into a CUDA graph on the first count and replayed afterwards, so a
// batch count costs one graph launch however many graphs it holds.
#include <algorithm>
#include <numeric>

#include "sweep_device.cuh"

namespace dbbc {

struct GraphDesc {
  const int64_t* row_ptr;
  const uint32_t* col;
  const uint32_t* lower;
  const uint64_t* work;
  int64_t n;
  int64_t nnz;
  int32_t n_u;
  int32_t hash_mult_log;
};

struct BatchPivot {
  int32_t graph;
  int32_t row;
};

struct BatchHubItem {
  int32_t graph;
  int32_t pad;
  SweepItem it;
};

struct GatherJob {
  const int32_t* order;
  int64_t n_hub, n_medium, n_light;
  int64_t medium_off, light_off;
};

__device__ __forceinline__ CsrView view_of(const GraphDesc& d) { return CsrView{d.row_ptr, d.col, d.lower, d.n_u, d.n, d.nnz}; }

// One CTA per graph copies its medium and light pivots into the batch lists.
__global__ void gather_pivots_kernel(const GatherJob* __restrict__ jobs, BatchPivot* __restrict__ med,
                                     BatchPivot* __restrict__ light) {
  const int gi = blockIdx.x;
  const GatherJob j = jobs[gi];
  for (int64_t i = threadIdx.x; i < j.n_medium; i += blockDim.x)
    med[j.medium_off + i] = BatchPivot{gi, j.order[j.n_hub + i]};
  for (int64_t i = threadIdx.x; i < j.n_light; i += blockDim.x)
    light[j.light_off + i] = BatchPivot{gi, j.order[j.n_hub + j.n_medium + i]};
}

// Pivots of a disjoint union, tagged with their component.
__global__ void gather_component_pivots_kernel(const int32_t* __restrict__ order, int64_t n_hub, int64_t n_medium,
                                               int64_t n_light, const int32_t* __restrict__ comp,
                                               BatchPivot* __restrict__ med, BatchPivot* __restrict__ light) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_medium + n_light; i += stride) {
    const int32_t row = order[n_hub + i];
    const BatchPivot bp{comp[row], row};
    if (i < n_medium) med[i] = bp;
    else light[i - n_medium] = bp;
  }
}

__global__ void gather_rows_kernel(const int32_t* __restrict__ comp, const int32_t* __restrict__ rows, int64_t n,
                                   int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = comp[rows[i]];
}

__device__ __forceinline__ void warp_flush(int graph, uint64_t& bal, uint64_t& unb, unsigned long long* out) {
  const uint64_t b = warp_sum_u64(bal), u = warp_sum_u64(unb);
  if (lane_id() == 0 && graph >= 0) {
    if (b) atomicAdd(&out[2 * graph], (unsigned long long)b);
    if (u) atomicAdd(&out[2 * graph + 1], (unsigned long long)u);
  }
  bal = 0;
  unb = 0;
}

// Light tier over all graphs: warps pull chunks of 32 consecutive pivots and
// flush their sums whenever the graph changes.
// Each warp's table has 2^slots_log slots (at most kLightSlots).
__global__ void __launch_bounds__(kLightWarps * 32) count_light_batch_kernel(
    const GraphDesc* __restrict__ desc, const BatchPivot* __restrict__ piv, int64_t n_piv, int* next_chunk,
    int slots_log, unsigned long long* out, unsigned* status) {
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
  int cur_graph = -1;
  CsrView g{};
  const uint64_t* work = nullptr;
  int mult_log = 1;
  for (;;) {
    int chunk = 0;
    if (lane == 0) chunk = atomicAdd(next_chunk, 1);
    chunk = __shfl_sync(kFullMask, chunk, 0);
    const int64_t t0 = (int64_t)chunk * 32;
    if (t0 >= n_piv) break;
    const int64_t t1 = t0 + 32 < n_piv ? t0 + 32 : n_piv;
    for (int64_t t = t0; t < t1; t++) {
      const BatchPivot bp = piv[t];
      if (bp.graph != cur_graph) {
        warp_flush(cur_graph, bal, unb, out);
        cur_graph = bp.graph;
        const GraphDesc d = desc[bp.graph];
        g = view_of(d);
        work = d.work;
        mult_log = d.hash_mult_log;
      }
      const int log_h = table_log(work[bp.row], max_log, mult_log);
      const PivotGeom q = pivot_geom(g, bp.row);
      full |= !hash_walk_dispatch(hash_group_log(work[bp.row], q.L, 5), lane, 32u, g, q, keys, vals, log_h, bal,
                                  unb);
      __syncwarp();
      for (int i = lane; i < (1 << log_h); i += 32) {
        keys[i] = kEmptyKey;
        vals[i] = 0;
      }
      __syncwarp();
    }
  }
  warp_flush(cur_graph, bal, unb, out);
  if (full) atomicOr(status, DBBC_DEV_HASH_FULL);
}

// Medium tier over all graphs: one CTA per pivot, sums flushed per pivot.
// The CTA's table has 2^slots_log slots (at most kMediumSlots).
__global__ void __launch_bounds__(kMediumThreads) count_medium_batch_kernel(const GraphDesc* __restrict__ desc,
                                                                            const BatchPivot* __restrict__ piv,
                                                                            int64_t n_piv, int slots_log,
                                                                            unsigned long long* out,
                                                                            unsigned* status) {
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
  bool full = false;
  for (int64_t t = blockIdx.x; t < n_piv; t += gridDim.x) {
    const BatchPivot bp = piv[t];
    const GraphDesc d = desc[bp.graph];
    const CsrView g = view_of(d);
    const int log_h = table_log(d.work[bp.row], max_log, d.hash_mult_log);
    const PivotGeom q = pivot_geom(g, bp.row);
    uint64_t bal = 0, unb = 0;
    full |= !hash_walk_dispatch(hash_group_log(d.work[bp.row], q.L, 5), threadIdx.x, (uint32_t)kMediumThreads, g, q,
                                keys, vals, log_h, bal, unb);
    __syncthreads();
    for (int i = threadIdx.x; i < (1 << log_h); i += kMediumThreads) {
      keys[i] = kEmptyKey;
      vals[i] = 0;
    }
    block_add_pair<kMediumThreads>(bal, unb, out + 2 * bp.graph);  // contains __syncthreads
  }
  if (full) atomicOr(status, DBBC_DEV_HASH_FULL);
}

// Hub sweep over all graphs' hub items (see hub_sweep_kernel); sums are
// flushed per item. Two shapes: wide CTAs (kSweepThreads threads, the full
// window) for large items, and narrow ones (kNarrowThreads threads, a window
// of kNarrowWords words, eight CTAs per SM) for the many small items of
// small graphs, whose per-item barriers, cursor set-up and sums would
// otherwise occupy a whole SM each. Measured on GB300 (4,096-graph batch):
// 64-, 96- and 128-thread narrow CTAs within 1% of each other, 256 threads
// 12% slower, 512 threads 34% slower.
#ifndef DBBC_NARROW_THREADS
#define DBBC_NARROW_THREADS 128
#endif
#ifndef DBBC_NARROW_WORDS
#define DBBC_NARROW_WORDS (6656 + 4)
#endif
constexpr int kNarrowThreads = DBBC_NARROW_THREADS;
constexpr uint32_t kNarrowWords = DBBC_NARROW_WORDS;
constexpr size_t kNarrowSmem = (size_t)kNarrowWords * 4;
static_assert(kNarrowWords % 4 == 0, "window buffers are cleared 16 bytes at a time");
// items above this many estimated wedges stay on wide CTAs (a long item on a
// narrow CTA would finish last)
#ifndef DBBC_NARROW_ITEM_WORK
#define DBBC_NARROW_ITEM_WORK (1u << 20)
#endif
constexpr uint64_t kNarrowItemWork = DBBC_NARROW_ITEM_WORK;

template <int THREADS, uint32_t WORDS>
__global__ void __launch_bounds__(THREADS) hub_sweep_batch_kernel(const GraphDesc* __restrict__ desc,
                                                                  const BatchHubItem* __restrict__ items,
                                                                  int64_t n_items, int* next_item,
                                                                  uint2* __restrict__ cursors, int64_t cur_cap,
                                                                  unsigned long long* out) {
  extern __shared__ __align__(16) unsigned char sweep_smem[];
  uint32_t* cnt_words = reinterpret_cast<uint32_t*>(sweep_smem);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sweep_smem);
  __shared__ int item_sh;
  __shared__ uint32_t nbn[2];
  const int tid = threadIdx.x;
  zero_words<THREADS>(cnt_words, WORDS);
  if (tid < 2) nbn[tid] = 0u;
  uint2* cur = cursors + (int64_t)blockIdx.x * cur_cap;
  for (;;) {
    if (tid == 0) item_sh = atomicAdd(next_item, 1);
    __syncthreads();
    const int64_t it = item_sh;
    __syncthreads();
    if (it >= n_items) break;
    const BatchHubItem bi = items[it];
    const SweepItem item = bi.it;
    const CsrView g = view_of(desc[bi.graph]);
    const PivotGeom q = pivot_geom(g, item.row);
    const uint32_t L = DBBC_CHECK((int64_t)q.L <= cur_cap) ? q.L : 0u;  // checked builds: cursor capacity
    for (uint32_t i = tid; i < L; i += THREADS) {
      uint32_t b, en, s1;
      lean_cursor_start(g, q, i, (item.flags & kItemFirst) ? 0u : item.lo, b, en, s1);
      cur[i] = lean_slot(b, en, s1);
    }
    __syncthreads();
    uint64_t bal = 0, unb = 0;
    sweep_cursor_item_dispatch<THREADS, WORDS>(item.group_log, g.col, L, cur, ItemWindows(item),
                                               (item.flags & kItemFinalize) != 0, sbase, cnt_words, nbn, bal, unb);
    block_add_pair<THREADS>(bal, unb, out + 2 * bi.graph);
  }
}

#define DBBC_WIDE_SWEEP hub_sweep_batch_kernel<kSweepThreads, kSweepWords>
#define DBBC_NARROW_SWEEP hub_sweep_batch_kernel<kNarrowThreads, kNarrowWords>

// The largest counter buffer (32-bit words) a window of the item needs, with
// the windows of ItemWindows: the first window of each counter width is its
// widest.
static uint32_t item_window_words(const SweepItem& it) {
  const uint32_t lo = it.lo, hi = it.hi;
  const uint32_t qe = std::min(std::max(it.q_end, lo), hi);
  const uint32_t te = std::min(std::max(it.t_end, qe), hi);
  const uint32_t ne = std::min(std::max(it.n_end, te), hi);
  uint32_t w = 0;
  if (qe > lo) {
    const uint32_t wh = std::min(lo + window_ranks<4>(), qe);
    w = std::max(w, (wh - (lo & ~3u) + 3u) >> 2);
  }
  if (te > qe) {
    const uint32_t wh = std::min(qe + window_ranks<8>(), te);
    w = std::max(w, (wh - (qe & ~1u) + 1u) >> 1);
  }
  if (ne > te) w = std::max(w, std::min(te + window_ranks<16>(), ne) - te);
  if (hi > ne) w = std::max(w, 2u * (std::min(ne + window_ranks<32>(), hi) - ne));
  return w;
}

}  // namespace dbbc

struct dbbc_batch {
  int device = 0;
  cudaStream_t stream = nullptr;   // stream the plan was created on (frees are ordered on it)
  cudaStream_t capture = nullptr;  // private stream used only to capture the CUDA graph
  cudaStream_t side = nullptr;     // second branch of a count (narrow hub items and the medium tier)
  cudaEvent_t fork = nullptr, join = nullptr;
  int32_t n_graphs = 0;
  dbbc::GraphDesc* desc = nullptr;
  dbbc::BatchPivot* light = nullptr;
  dbbc::BatchPivot* medium = nullptr;
  dbbc::BatchHubItem* hub = nullptr;         // items for wide CTAs, then items for narrow ones
  int64_t n_light = 0, n_medium = 0, n_hub_items = 0, max_lower = 1;
  int64_t n_wide = 0, n_narrow = 0;
  unsigned long long* out = nullptr;  // [n_graphs][2]
  uint2* cursors = nullptr;         // wide CTAs'
  uint2* narrow_cursors = nullptr;  // narrow CTAs'
  int* counters = nullptr;  // [0] light chunks, [1] wide hub items, [2] narrow hub items
  unsigned* status = nullptr;
  int hub_grid = 0, narrow_grid = 0, light_grid = 0, medium_grid = 0;
  int light_log = 10, medium_log = 13;  // log2 of the hash slots of a light / medium table
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels_per_replay = 0;
  std::vector<void*> allocations;
};

namespace dbbc {

static void* batch_alloc(dbbc_batch* b, size_t bytes) {
  void* p = dev_alloc(bytes ? bytes : 16, b->stream);
  if (!p) throw Error{DBBC_ENOMEM, "batch_alloc"};
  b->allocations.push_back(p);
  return p;
}

static void batch_release(dbbc_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  for (void* p : b->allocations) dev_free(p, b->stream);
  b->allocations.clear();
  if (b->capture) cudaStreamDestroy(b->capture);
  b->capture = nullptr;
  if (b->side) cudaStreamDestroy(b->side);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  b->side = nullptr;
  b->fork = b->join = nullptr;
}

static void finish_plan(dbbc_batch* b, std::vector<GraphDesc>& desc, std::vector<BatchHubItem>& items,
                        const std::vector<uint64_t>& est);

// Hash table sizes of the plan's light and medium kernels: the largest any of
// its graphs' tiers needs (each graph's pivots were tiered by its own tuning).
static void plan_table_logs(dbbc_batch* b, const dbbc_graph* const* gs, int32_t n) {
  b->light_log = 5;
  b->medium_log = 5;
  for (int32_t i = 0; i < n; i++) {
    const Tuning& t = gs[i]->tune;
    b->light_log = std::max(b->light_log, tier_slots_log(t.light_max_work, t.hash_mult_log, 10));
    b->medium_log = std::max(b->medium_log, tier_slots_log(t.medium_max_work, t.hash_mult_log, 13));
  }
}
static size_t light_smem_bytes(const dbbc_batch* b) {
  return (size_t)kLightWarps * ((size_t)1 << b->light_log) * 12;
}
static size_t medium_smem_bytes(const dbbc_batch* b) { return ((size_t)1 << b->medium_log) * 12; }

// Plan for the components of one union handle: every component shares the
// union's CSR; pivots and hub items are tagged with their component.
static void plan_components(dbbc_batch* b, const dbbc_graph* g) {
  cudaStream_t s = b->stream;
  std::vector<GraphDesc> desc((size_t)b->n_graphs, GraphDesc{g->row_ptr, g->col, g->lower, g->work, g->n, g->nnz, g->n_u, g->tune.hash_mult_log});
  b->n_medium = g->n_medium;
  b->n_light = g->n_light;
  b->max_lower = std::max<int64_t>(1, g->sweep_max_lower);
  // components of the hub items' rows
  const size_t nh = g->sweep_items_host.size();
  std::vector<int32_t> rows(nh), comps(nh);
  for (size_t k = 0; k < nh; k++) rows[k] = g->sweep_items_host[k].row;
  std::vector<BatchHubItem> items(nh);
  if (nh > 0) {
    Scratch sc(s);
    int32_t* d_rows = sc.get<int32_t>(nh);
    int32_t* d_comp = sc.get<int32_t>(nh);
    DBBC_CUDA(cudaMemcpyAsync(d_rows, rows.data(), nh * 4, cudaMemcpyHostToDevice, s));
    gather_rows_kernel<<<(unsigned)std::min<size_t>((nh + 255) / 256, 4096), 256, 0, s>>>(g->component, d_rows,
                                                                                        (int64_t)nh, d_comp);
    DBBC_LAUNCH_CHECK();
    DBBC_CUDA(cudaMemcpyAsync(comps.data(), d_comp, nh * 4, cudaMemcpyDeviceToHost, s));
    DBBC_CUDA(cudaStreamSynchronize(s));
  }
  // the union's items are already in descending estimated work
  for (size_t k = 0; k < nh; k++) items[k] = BatchHubItem{comps[k], 0, g->sweep_items_host[k]};
  plan_table_logs(b, &g, 1);
  finish_plan(b, desc, items, g->sweep_est_host);
  if (b->n_medium + b->n_light > 0) {
    const int64_t total = b->n_medium + b->n_light;
    gather_component_pivots_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, s>>>(
        g->order, g->n_hub, g->n_medium, g->n_light, g->component, b->medium, b->light);
    DBBC_LAUNCH_CHECK();
  }
  DBBC_CUDA(cudaStreamSynchronize(s));
}

static void plan_batch(dbbc_batch* b, const dbbc_graph* const* gs) {
  const int32_t n = b->n_graphs;
  cudaStream_t s = b->stream;
  std::vector<GraphDesc> desc((size_t)n);
  std::vector<GatherJob> jobs((size_t)n);
  struct HubRef {
    BatchHubItem item;
    uint64_t est;
  };
  std::vector<HubRef> hubs;
  for (int32_t i = 0; i < n; i++) {
    const dbbc_graph* g = gs[i];
    desc[(size_t)i] = GraphDesc{g->row_ptr, g->col, g->lower, g->work, g->n, g->nnz, g->n_u, g->tune.hash_mult_log};
    jobs[(size_t)i] = GatherJob{g->order, g->n_hub, g->n_medium, g->n_light, b->n_medium, b->n_light};
    b->n_medium += g->n_medium;
    b->n_light += g->n_light;
    for (size_t k = 0; k < g->sweep_items_host.size(); k++)
      hubs.push_back(HubRef{BatchHubItem{i, 0, g->sweep_items_host[k]}, g->sweep_est_host[k]});
    if (g->n_hub > 0) b->max_lower = std::max<int64_t>(b->max_lower, g->sweep_max_lower);
  }
  std::stable_sort(hubs.begin(), hubs.end(), [](const HubRef& a, const HubRef& c) { return a.est > c.est; });
  std::vector<BatchHubItem> items(hubs.size());
  std::vector<uint64_t> est(hubs.size());
  for (size_t k = 0; k < hubs.size(); k++) {
    items[k] = hubs[k].item;
    est[k] = hubs[k].est;
  }
  plan_table_logs(b, gs, n);
  finish_plan(b, desc, items, est);
  GatherJob* d_jobs = static_cast<GatherJob*>(batch_alloc(b, jobs.size() * sizeof(GatherJob)));
  DBBC_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(GatherJob), cudaMemcpyHostToDevice, s));
  if (n > 0) {
    gather_pivots_kernel<<<(unsigned)n, 256, 0, s>>>(d_jobs, b->medium, b->light);
    DBBC_LAUNCH_CHECK();
  }
  DBBC_CUDA(cudaStreamSynchronize(s));  // host vectors above must outlive the copies
}

// Allocations, launch shapes and uploads shared by both kinds of plan.
static void finish_plan(dbbc_batch* b, std::vector<GraphDesc>& desc, std::vector<BatchHubItem>& items,
                        const std::vector<uint64_t>& est) {
  cudaStream_t s = b->stream;
  const int32_t n = b->n_graphs;
  // wide items first, then the narrow ones, each in their LPT order; an item
  // goes to a narrow CTA when its windows fit kNarrowWords and its estimated
  // work (est[k], absent: unknown) is small
  {
    std::vector<BatchHubItem> narrow;
    size_t n_wide = 0;
    for (size_t k = 0; k < items.size(); k++) {
      if (k < est.size() && est[k] <= kNarrowItemWork && item_window_words(items[k].it) <= kNarrowWords)
        narrow.push_back(items[k]);
      else
        items[n_wide++] = items[k];
    }
    std::copy(narrow.begin(), narrow.end(), items.begin() + (ptrdiff_t)n_wide);
    b->n_wide = (int64_t)n_wide;
    b->n_narrow = (int64_t)narrow.size();
  }
  b->n_hub_items = (int64_t)items.size();
  b->desc = static_cast<GraphDesc*>(batch_alloc(b, desc.size() * sizeof(GraphDesc)));
  b->light = static_cast<BatchPivot*>(batch_alloc(b, (size_t)b->n_light * sizeof(BatchPivot)));
  b->medium = static_cast<BatchPivot*>(batch_alloc(b, (size_t)b->n_medium * sizeof(BatchPivot)));
  b->hub = static_cast<BatchHubItem*>(batch_alloc(b, items.size() * sizeof(BatchHubItem)));
  b->out = static_cast<unsigned long long*>(batch_alloc(b, (size_t)n * 2 * sizeof(unsigned long long)));
  b->counters = static_cast<int*>(batch_alloc(b, 3 * sizeof(int)));
  b->status = static_cast<unsigned*>(batch_alloc(b, sizeof(unsigned)));
  b->hub_grid = (int)std::min<int64_t>(num_sms() * blocks_per_sm((const void*)DBBC_WIDE_SWEEP, kSweepThreads,
                                                                 kSweepSmem), std::max<int64_t>(b->n_wide, 1));
  b->narrow_grid = (int)std::min<int64_t>(num_sms() * blocks_per_sm((const void*)DBBC_NARROW_SWEEP, kNarrowThreads,
                                                                    kNarrowSmem), std::max<int64_t>(b->n_narrow, 1));
  if (b->n_wide > 0)
    b->cursors = static_cast<uint2*>(batch_alloc(b, (size_t)b->hub_grid * (size_t)b->max_lower * sizeof(uint2)));
  if (b->n_narrow > 0)
    b->narrow_cursors = static_cast<uint2*>(batch_alloc(b, (size_t)b->narrow_grid * (size_t)b->max_lower * sizeof(uint2)));
  {
    const int sms = num_sms();
    const int64_t want = ceil_div<int64_t>(ceil_div<int64_t>(b->n_light, 32), kLightWarps);
    const int64_t cap = (int64_t)sms * blocks_per_sm((const void*)count_light_batch_kernel, kLightWarps * 32,
                                                     light_smem_bytes(b));
    b->light_grid = (int)std::max<int64_t>(1, std::min(want, cap));
    const int64_t mcap = (int64_t)sms * blocks_per_sm((const void*)count_medium_batch_kernel, kMediumThreads,
                                                      medium_smem_bytes(b));
    b->medium_grid = (int)std::max<int64_t>(1, std::min<int64_t>(b->n_medium, mcap));
  }
  if (!b->side) {
    DBBC_CUDA(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
    DBBC_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    DBBC_CUDA(cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming));
  }
  DBBC_CUDA(cudaMemcpyAsync(b->desc, desc.data(), desc.size() * sizeof(GraphDesc), cudaMemcpyHostToDevice, s));
  if (!items.empty())
    DBBC_CUDA(cudaMemcpyAsync(b->hub, items.data(), items.size() * sizeof(BatchHubItem), cudaMemcpyHostToDevice, s));
  DBBC_CUDA(cudaStreamSynchronize(s));  // host vectors must outlive the copies
}

// The batch count: clear outputs and counters, then the tiers on two
// branches that run side by side (every kernel adds into the graphs' output
// pairs with atomics, so their order does not matter): the wide hub items and
// the light tier on `s`, the narrow hub items and the medium tier on the side
// stream. The side branch forks from and joins back into `s`, also when `s`
// is being captured.
static void enqueue_batch(dbbc_batch* b, cudaStream_t s) {
  DBBC_CUDA(cudaMemsetAsync(b->out, 0, (size_t)b->n_graphs * 2 * sizeof(unsigned long long), s));
  DBBC_CUDA(cudaMemsetAsync(b->counters, 0, 3 * sizeof(int), s));
  DBBC_CUDA(cudaMemsetAsync(b->status, 0, sizeof(unsigned), s));
  const bool two = b->side && (b->n_narrow > 0 || b->n_medium > 0) && (b->n_wide > 0 || b->n_light > 0);
  cudaStream_t s2 = two ? b->side : s;
  if (two) {
    DBBC_CUDA(cudaEventRecord(b->fork, s));
    DBBC_CUDA(cudaStreamWaitEvent(s2, b->fork, 0));
  }
  if (b->n_narrow > 0) {
    DBBC_NARROW_SWEEP<<<b->narrow_grid, kNarrowThreads, kNarrowSmem, s2>>>(
        b->desc, b->hub + b->n_wide, b->n_narrow, b->counters + 2, b->narrow_cursors, b->max_lower, b->out);
    DBBC_LAUNCH_CHECK();
  }
  if (b->n_medium > 0) {
    count_medium_batch_kernel<<<(unsigned)b->medium_grid, kMediumThreads, medium_smem_bytes(b), s2>>>(
        b->desc, b->medium, b->n_medium, b->medium_log, b->out, b->status);
    DBBC_LAUNCH_CHECK();
  }
  if (b->n_wide > 0) {
    DBBC_WIDE_SWEEP<<<b->hub_grid, kSweepThreads, kSweepSmem, s>>>(b->desc, b->hub, b->n_wide, b->counters + 1,
                                                                  b->cursors, b->max_lower, b->out);
    DBBC_LAUNCH_CHECK();
  }
  if (b->n_light > 0) {
    count_light_batch_kernel<<<(unsigned)b->light_grid, kLightWarps * 32, light_smem_bytes(b), s>>>(
        b->desc, b->light, b->n_light, b->counters, b->light_log, b->out, b->status);
    DBBC_LAUNCH_CHECK();
  }
  if (two) {
    DBBC_CUDA(cudaEventRecord(b->join, s2));
    DBBC_CUDA(cudaStreamWaitEvent(s, b->join, 0));
  }
}

static void set_batch_attributes() {
  DBBC_CUDA(cudaFuncSetAttribute(count_light_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)kLightWarps * kLightSlots * 12)));
  DBBC_CUDA(cudaFuncSetAttribute(count_medium_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)kMediumSlots * 12)));
  DBBC_CUDA(cudaFuncSetAttribute(DBBC_WIDE_SWEEP, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmem));
  DBBC_CUDA(cudaFuncSetAttribute(DBBC_NARROW_SWEEP, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNarrowSmem));
}

static void check_batch_status(const dbbc_batch* b, cudaStream_t s) {
  unsigned h = 0;
  DBBC_CUDA(cudaMemcpyAsync(&h, b->status, sizeof(h), cudaMemcpyDeviceToHost, s));
  DBBC_CUDA(cudaStreamSynchronize(s));
  raise_device_status(h);
}

template <typename F>
static dbbc_status batch_guard(F&& f) {
  try {
    f();
    return DBBC_OK;
  } catch (const Error& e) {
    return e.status;
  } catch (const std::bad_alloc&) {
    return DBBC_ENOMEM;
  } catch (...) {
    return DBBC_EINTERNAL;
  }
}

// Counts of one graph restricted to some of its pivots: a one-graph plan
// over the given medium and light pivot rows and hub items.
void count_subset(const dbbc_graph* g, cudaStream_t s, const std::vector<int32_t>& medium_rows,
                  const std::vector<int32_t>& light_rows, const std::vector<SweepItem>& hub_items, uint64_t* balanced,
                  uint64_t* unbalanced) {
  dbbc_batch plan;
  dbbc_batch* b = &plan;
  b->stream = s;
  b->n_graphs = 1;
  uint64_t h[2] = {0, 0};
  try {
    DBBC_CUDA(cudaGetDevice(&b->device));
    set_batch_attributes();
    std::vector<GraphDesc> desc(1, GraphDesc{g->row_ptr, g->col, g->lower, g->work, g->n, g->nnz, g->n_u,
                                              g->tune.hash_mult_log});
    b->n_medium = (int64_t)medium_rows.size();
    b->n_light = (int64_t)light_rows.size();
    b->max_lower = std::max<int64_t>(1, g->sweep_max_lower);
    std::vector<BatchHubItem> items(hub_items.size());
    for (size_t k = 0; k < hub_items.size(); k++) items[k] = BatchHubItem{0, 0, hub_items[k]};
    plan_table_logs(b, &g, 1);
    finish_plan(b, desc, items, {});  // work unknown: every item on wide CTAs
    std::vector<BatchPivot> med(medium_rows.size()), light(light_rows.size());
    for (size_t k = 0; k < medium_rows.size(); k++) med[k] = BatchPivot{0, medium_rows[k]};
    for (size_t k = 0; k < light_rows.size(); k++) light[k] = BatchPivot{0, light_rows[k]};
    if (!med.empty())
      DBBC_CUDA(cudaMemcpyAsync(b->medium, med.data(), med.size() * sizeof(BatchPivot), cudaMemcpyHostToDevice, s));
    if (!light.empty())
      DBBC_CUDA(cudaMemcpyAsync(b->light, light.data(), light.size() * sizeof(BatchPivot), cudaMemcpyHostToDevice,
                                s));
    enqueue_batch(b, s);
    DBBC_CUDA(cudaMemcpyAsync(h, b->out, sizeof(h), cudaMemcpyDeviceToHost, s));
    check_batch_status(b, s);  // synchronizes (the host vectors outlive the copies)
  } catch (...) {
    batch_release(b);
    throw;
  }
  batch_release(b);
  if (balanced) *balanced = h[0];
  if (unbalanced) *unbalanced = h[1];
}

}  // namespace dbbc

using namespace dbbc;

extern "C" {

dbbc_status dbbc_batch_create(const dbbc_graph* const* gs, int32_t n_graphs, void* cuda_stream, dbbc_batch** out) {
  if (!out || n_graphs < 0 || (n_graphs > 0 && !gs)) return DBBC_EINVAL;
  for (int32_t i = 0; i < n_graphs; i++)
    if (!gs[i]) return DBBC_EINVAL;
  dbbc_batch* b = nullptr;
  try {
    b = new dbbc_batch();
  } catch (...) {
    return DBBC_ENOMEM;
  }
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->n_graphs = n_graphs;
  const dbbc_status st = batch_guard([&] {
    DBBC_CUDA(cudaGetDevice(&b->device));
    set_batch_attributes();
    plan_batch(b, gs);
  });
  if (st != DBBC_OK) {
    batch_release(b);
    (void)cudaStreamSynchronize(b->stream);
    delete b;
    return st;
  }
  *out = b;
  return DBBC_OK;
}

dbbc_status dbbc_batch_count_async(dbbc_batch* b, void* cuda_stream, uint64_t* d_out) {
  if (!b) return DBBC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return batch_guard([&] {
    if (!b->exec) {
      // capture on a private stream (the caller's may be the legacy stream,
      // which cannot be captured), replay on the caller's stream
      if (!b->capture) DBBC_CUDA(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
      cudaGraph_t graph = nullptr;
      DBBC_CUDA(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
      const uint64_t before = launches_so_far();
      try {
        enqueue_batch(b, b->capture);
      } catch (...) {
        cudaStreamEndCapture(b->capture, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      b->kernels_per_replay = launches_so_far() - before;
      note_launches((uint64_t)0 - b->kernels_per_replay);  // captured, not yet run
      DBBC_CUDA(cudaStreamEndCapture(b->capture, &graph));
      const cudaError_t e = cudaGraphInstantiate(&b->exec, graph, 0);
      cudaGraphDestroy(graph);
      DBBC_CUDA(e);
    }
    DBBC_CUDA(cudaGraphLaunch(b->exec, s));
    note_launches(b->kernels_per_replay);
    if (d_out)
      DBBC_CUDA(cudaMemcpyAsync(d_out, b->out, (size_t)b->n_graphs * 2 * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                                s));
  });
}

dbbc_status dbbc_batch_count(dbbc_batch* b, void* cuda_stream, uint64_t* balanced, uint64_t* unbalanced) {
  if (!b || (b->n_graphs > 0 && (!balanced || !unbalanced))) return DBBC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  std::vector<uint64_t> h((size_t)b->n_graphs * 2);
  dbbc_status st = dbbc_batch_count_async(b, cuda_stream, nullptr);
  if (st != DBBC_OK) return st;
  st = batch_guard([&] {
    DBBC_CUDA(cudaMemcpyAsync(h.data(), b->out, h.size() * 8, cudaMemcpyDeviceToHost, s));
    check_batch_status(b, s);
  });
  if (st != DBBC_OK) return st;
  for (int32_t i = 0; i < b->n_graphs; i++) {
    balanced[i] = h[2 * (size_t)i];
    unbalanced[i] = h[2 * (size_t)i + 1];
  }
  return DBBC_OK;
}

dbbc_status dbbc_count_components(const dbbc_graph* g, void* cuda_stream, uint64_t* balanced,
                                  uint64_t* unbalanced) {
  if (!g || !balanced || !unbalanced) return DBBC_EINVAL;
  if (!g->component) return dbbc_count(g, cuda_stream, balanced, unbalanced);
  const int32_t n = g->n_components;
  if (n == 0) return DBBC_OK;
  dbbc_batch* b = nullptr;
  try {
    b = new dbbc_batch();
  } catch (...) {
    return DBBC_ENOMEM;
  }
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->n_graphs = n;
  std::vector<uint64_t> h((size_t)n * 2);
  const dbbc_status st = batch_guard([&] {
    DBBC_CUDA(cudaGetDevice(&b->device));
    set_batch_attributes();
    plan_components(b, g);
    enqueue_batch(b, b->stream);
    DBBC_CUDA(cudaMemcpyAsync(h.data(), b->out, h.size() * 8, cudaMemcpyDeviceToHost, b->stream));
    check_batch_status(b, b->stream);
  });
  dbbc_batch_free(b);
  if (st != DBBC_OK) return st;
  for (int32_t i = 0; i < n; i++) {
    balanced[i] = h[2 * (size_t)i];
    unbalanced[i] = h[2 * (size_t)i + 1];
  }
  return DBBC_OK;
}

void dbbc_batch_free(dbbc_batch* b) {
  if (!b) return;
  batch_release(b);
  delete b;
}

// One-shot forms over a temporary plan (no graph capture).
dbbc_status dbbc_count_batch_async(const dbbc_graph* const* gs, int32_t n_graphs, void* cuda_stream,
                                   uint64_t* d_out) {
  if (n_graphs < 0 || (n_graphs > 0 && (!gs || !d_out))) return DBBC_EINVAL;
  if (n_graphs == 0) return DBBC_OK;
  dbbc_batch* b = nullptr;
  dbbc_status st = dbbc_batch_create(gs, n_graphs, cuda_stream, &b);
  if (st != DBBC_OK) return st;
  st = batch_guard([&] {
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    enqueue_batch(b, s);
    DBBC_CUDA(cudaMemcpyAsync(d_out, b->out, (size_t)n_graphs * 2 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  });
  dbbc_batch_free(b);  // frees are stream-ordered after the copy
  return st;
}

dbbc_status dbbc_count_batch(const dbbc_graph* const* gs, int32_t n_graphs, void* cuda_stream, uint64_t* balanced,
                             uint64_t* unbalanced) {
  if (n_graphs < 0 || (n_graphs > 0 && (!gs || !balanced || !unbalanced))) return DBBC_EINVAL;
  for (int32_t i = 0; i < n_graphs; i++)
    if (!gs[i]) return DBBC_EINVAL;
  if (n_graphs == 0) return DBBC_OK;
  dbbc_batch* b = nullptr;
  dbbc_status st = dbbc_batch_create(gs, n_graphs, cuda_stream, &b);
  if (st != DBBC_OK) return st;
  std::vector<uint64_t> h((size_t)n_graphs * 2);
  st = batch_guard([&] {
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    enqueue_batch(b, s);
    DBBC_CUDA(cudaMemcpyAsync(h.data(), b->out, h.size() * 8, cudaMemcpyDeviceToHost, s));
    check_batch_status(b, s);
  });
  dbbc_batch_free(b);
  if (st != DBBC_OK) return st;
  for (int32_t i = 0; i < n_graphs; i++) {
    balanced[i] = h[2 * (size_t)i];
    unbalanced[i] = h[2 * (size_t)i + 1];
  }
  return DBBC_OK;
}

}  // extern "C"
