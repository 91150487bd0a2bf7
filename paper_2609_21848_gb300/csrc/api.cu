// C ABI of the dbbc library (see include/dbbc.h for the contract of every
// entry point). Each entry point converts internal errors into a status; no
// C++ exception crosses the interface.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>

#include "internal.h"
#include "common.cuh"

namespace dbbc {

namespace {
std::atomic<uint64_t> g_launches{0};
void* (*g_alloc_fn)(size_t, void*, void*) = nullptr;
void (*g_free_fn)(void*, void*, void*) = nullptr;
void* g_alloc_ctx = nullptr;
}  // namespace

// The tuning new builds take; builder threads read it while another thread
// may set it, so both sides hold the lock.
namespace {
std::mutex g_tuning_mu;
Tuning g_tuning;
}  // namespace
Tuning current_tuning() {
  std::lock_guard<std::mutex> lock(g_tuning_mu);
  return g_tuning;
}

// Flag words of the translation units of a checked build (see common.cuh).
namespace {
std::mutex g_checked_mu;
std::vector<unsigned (*)()>& checked_units() {
  static std::vector<unsigned (*)()> units;
  return units;
}
}  // namespace

void checked_register(unsigned (*take)()) {
  std::lock_guard<std::mutex> lock(g_checked_mu);
  checked_units().push_back(take);
}

unsigned checked_take_all() {
  if (!DBBC_CHECKED) return 0u;
  DBBC_CUDA(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lock(g_checked_mu);
  unsigned f = 0;
  for (unsigned (*take)() : checked_units()) f |= take();
  return f;
}

void raise_device_status(unsigned h) {
  h |= checked_take_all();
  if (h & DBBC_DEV_RANGE) throw Error{DBBC_EINTERNAL, "index out of range (checked build)"};
  if (h & DBBC_DEV_HASH_FULL) throw Error{DBBC_EINTERNAL, "shared hash table overflow"};
  if (h) throw Error{DBBC_EINTERNAL, "device status"};
}

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// Device memory comes from one stream-ordered pool per device owned by the
// library. The pool keeps up to kPoolKeepBytes of freed memory mapped across
// synchronizations (the default pool would unmap all of it at every
// synchronize, and the next build or count would map it again); what it holds
// beyond that goes back to the device. A 300M-edge build and count peak near
// 20 GB of scratch and graph, so the pool keeps 32 GB.
#ifndef DBBC_POOL_KEEP_GB
#define DBBC_POOL_KEEP_GB 32
#endif
constexpr uint64_t kPoolKeepBytes = uint64_t{DBBC_POOL_KEEP_GB} << 30;

static cudaMemPool_t library_pool(int dev) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    (void)cudaGetLastError();
    pool = nullptr;  // fall back to the device's default pool
  } else {
    uint64_t keep = kPoolKeepBytes;
    (void)cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  pools[dev] = pool;
  return pool;
}

void* dev_alloc(size_t bytes, cudaStream_t s) {
  if (g_alloc_fn) return g_alloc_fn(bytes, (void*)s, g_alloc_ctx);
  void* p = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  const cudaMemPool_t pool = library_pool(dev);
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void* p, cudaStream_t s) {
  if (!p) return;
  if (g_free_fn) {
    g_free_fn(p, (void*)s, g_alloc_ctx);
    return;
  }
  if (cudaFreeAsync(p, s) != cudaSuccess) (void)cudaGetLastError();
}

template <typename F>
static dbbc_status guarded(F&& f) {
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

static void check_status_word(const unsigned* d_status, cudaStream_t s) {
  unsigned h = 0;
  DBBC_CUDA(cudaMemcpyAsync(&h, d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
  DBBC_CUDA(cudaStreamSynchronize(s));
  raise_device_status(h);
}

}  // namespace dbbc

using namespace dbbc;

extern "C" {

const char* dbbc_version(void) { return DBBC_CHECKED ? "0.1.0+checked" : "0.1.0"; }

int dbbc_is_checked(void) { return DBBC_CHECKED ? 1 : 0; }

dbbc_status dbbc_checked_flags(uint32_t* flags) {
  if (!flags) return DBBC_EINVAL;
  return guarded([&] { *flags = checked_take_all(); });
}

const char* dbbc_status_string(dbbc_status s) {
  switch (s) {
    case DBBC_OK: return "ok";
    case DBBC_EINVAL: return "invalid argument or input graph";
    case DBBC_ENOMEM: return "device allocation failed";
    case DBBC_ECUDA: return "CUDA runtime error";
    case DBBC_ETIMEOUT: return "bounded device wait gave up";
    case DBBC_EOVERFLOW: return "count or capacity overflow";
    case DBBC_EINTERNAL: return "internal consistency check failed";
  }
  return "unknown status";
}

dbbc_status dbbc_set_tuning(const dbbc_tuning* t) {
  if (!t) {
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    g_tuning = Tuning();
    return DBBC_OK;
  }
  if (t->light_max_work < 1 || t->light_max_work > kLightMaxWork || t->medium_max_work < t->light_max_work ||
      t->medium_max_work > kMediumMaxWork || t->hub_item_work < 1024 || t->hash_mult_log < 1 ||
      t->hash_mult_log > 3 || !(t->list_density >= 0) || t->list_group_log < 0 || t->list_group_log > 5 ||
      t->list_group_log == 1 || !(t->list_wide_density >= 0))
    return DBBC_EINVAL;
  for (int i = 0; i < 4; i++)
    if (!(t->group_density[i] >= 0) || (i > 0 && t->group_density[i] > t->group_density[i - 1])) return DBBC_EINVAL;
  Tuning n;
  n.light_max_work = t->light_max_work;
  n.medium_max_work = t->medium_max_work;
  n.hub_item_work = t->hub_item_work;
  for (int i = 0; i < 4; i++) n.group_density[i] = t->group_density[i];
  n.hash_mult_log = t->hash_mult_log;
  n.list_density = t->list_density;
  n.list_group_log = t->list_group_log;
  n.finalize_window_wedges = t->finalize_window_wedges;
  n.list_wide_density = t->list_wide_density;
  std::lock_guard<std::mutex> lock(g_tuning_mu);
  g_tuning = n;
  return DBBC_OK;
}

void dbbc_get_tuning(dbbc_tuning* t) {
  if (!t) return;
  const Tuning c = current_tuning();
  t->light_max_work = c.light_max_work;
  t->medium_max_work = c.medium_max_work;
  t->hub_item_work = c.hub_item_work;
  for (int i = 0; i < 4; i++) t->group_density[i] = c.group_density[i];
  t->hash_mult_log = c.hash_mult_log;
  t->list_density = c.list_density;
  t->list_group_log = c.list_group_log;
  t->finalize_window_wedges = c.finalize_window_wedges;
  t->list_wide_density = c.list_wide_density;
}

void dbbc_set_allocator(void* (*alloc_fn)(size_t, void*, void*), void (*free_fn)(void*, void*, void*), void* ctx) {
  if (alloc_fn && free_fn) {
    g_alloc_fn = alloc_fn;
    g_free_fn = free_fn;
    g_alloc_ctx = ctx;
  } else {
    g_alloc_fn = nullptr;
    g_free_fn = nullptr;
    g_alloc_ctx = nullptr;
  }
}

dbbc_status dbbc_graph_from_coo(const int32_t* u, const int32_t* v, const int8_t* sign, int64_t m, int32_t n_u,
                                int32_t n_v, uint32_t flags, void* cuda_stream, dbbc_graph** out) {
  if (!out || m < 0 || m >= (int64_t{1} << 31) || n_u < 0 || n_v < 0 ||
      (int64_t)n_u + (int64_t)n_v >= (int64_t{1} << 31) || (flags & ~3u) != 0)
    return DBBC_EINVAL;
  if (m > 0 && (!u || !v || !sign)) return DBBC_EINVAL;
  dbbc_graph* g = nullptr;
  try {
    g = new dbbc_graph();
  } catch (...) {
    return DBBC_ENOMEM;
  }
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  g->n_u = n_u;
  g->n_v = n_v;
  const dbbc_status st = guarded([&] {
    DBBC_CUDA(cudaGetDevice(&g->device));
    build_graph(g, u, v, sign, m, (flags & DBBC_INPUT_DEVICE) != 0, (flags & DBBC_DUP_REJECT) != 0, g->stream);
    if (DBBC_CHECKED) raise_device_status(0u);
  });
  if (st != DBBC_OK) {
    free_graph_memory(g);
    (void)cudaStreamSynchronize(g->stream);
    delete g;
    return st;
  }
  *out = g;
  return DBBC_OK;
}

dbbc_status dbbc_graph_from_coo_multi(const int32_t* u, const int32_t* v, const int8_t* sign,
                                      const int64_t* edge_offsets, const int32_t* n_u, const int32_t* n_v,
                                      int32_t n_graphs, uint32_t flags, void* cuda_stream, dbbc_graph** out) {
  if (!out || n_graphs < 0 || (flags & ~3u) != 0) return DBBC_EINVAL;
  if (n_graphs > 0 && (!edge_offsets || !n_u || !n_v)) return DBBC_EINVAL;
  if (n_graphs > 0 && edge_offsets[n_graphs] > 0 && (!u || !v || !sign)) return DBBC_EINVAL;
  dbbc_graph* g = nullptr;
  try {
    g = new dbbc_graph();
  } catch (...) {
    return DBBC_ENOMEM;
  }
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  const int64_t zero = 0;
  const dbbc_status st = guarded([&] {
    DBBC_CUDA(cudaGetDevice(&g->device));
    build_graph_multi(g, u, v, sign, n_graphs > 0 ? edge_offsets : &zero, n_u, n_v, n_graphs,
                      (flags & DBBC_INPUT_DEVICE) != 0, (flags & DBBC_DUP_REJECT) != 0, g->stream);
    if (DBBC_CHECKED) raise_device_status(0u);
  });
  if (st != DBBC_OK) {
    free_graph_memory(g);
    (void)cudaStreamSynchronize(g->stream);
    delete g;
    return st;
  }
  *out = g;
  return DBBC_OK;
}

void dbbc_graph_free(dbbc_graph* g) {
  if (!g) return;
  free_graph_memory(g);
  delete g;
}

size_t dbbc_graph_device_bytes(const dbbc_graph* g) { return g ? g->device_bytes : 0; }

size_t dbbc_estimate_bytes(int64_t m, int32_t n_u, int32_t n_v) {
  if (m < 0 || n_u < 0 || n_v < 0) return 0;
  const size_t n = (size_t)n_u + (size_t)n_v, mm = (size_t)m;
  // handle: row_ptr 8(n+1), col 8m, lower/vertex 8n, work 8n, order 4n, items
  const size_t handle = 8 * (n + 1) + 8 * mm + 8 * n + 8 * n + 4 * n + 16 * (mm / 64 + 16);
  // build peak: inputs 9m, dedup 24m + flags/pos 8m, edges 9m, CSR keys 32m and their U positions 8m, vertex
  // keys 16n + 16n
  const size_t build = 9 * mm + 32 * mm + 9 * mm + 32 * mm + 8 * mm + 48 * n + (mm / 4096 + 1) * 1024;
  return handle + build;
}

dbbc_status dbbc_graph_get_info(const dbbc_graph* g, dbbc_graph_info* info) {
  if (!g || !info) return DBBC_EINVAL;
  dbbc_graph_info r;
  std::memset(&r, 0, sizeof(r));
  r.n_u = g->n_u;
  r.n_v = g->n_v;
  r.m_input = g->m_input;
  r.m = g->m;
  r.wedges = g->wedges;
  r.n_pivots = g->n_piv;
  r.n_light = g->n_light;
  r.n_medium = g->n_medium;
  r.n_hub = g->n_hub;
  r.wedges_light = g->wedges_light;
  r.wedges_medium = g->wedges_medium;
  r.wedges_hub = g->wedges_hub;
  r.lower_light = g->lower_light;
  r.lower_medium = g->lower_medium;
  r.lower_hub = g->lower_hub;
  r.hub_items = g->n_sweep_items;
  r.hub_cursor_inits = g->hub_cursor_inits;
  r.hub_cursor_steps = g->hub_cursor_steps;
  r.device_bytes = g->device_bytes;
  r.n_components = g->n_components;
  *info = r;
  return DBBC_OK;
}

dbbc_status dbbc_count_async(const dbbc_graph* g, void* cuda_stream, uint64_t* d_out) {
  if (!g || !d_out) return DBBC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return guarded([&] {
    Scratch sc(s);
    unsigned* d_status = sc.get<unsigned>(1);
    DBBC_CUDA(cudaMemsetAsync(d_status, 0, sizeof(unsigned), s));
    DBBC_CUDA(cudaMemsetAsync(d_out, 0, 2 * sizeof(uint64_t), s));
    enqueue_count(g, s, reinterpret_cast<unsigned long long*>(d_out), d_status, sc);
  });
}

dbbc_status dbbc_count(const dbbc_graph* g, void* cuda_stream, uint64_t* balanced, uint64_t* unbalanced) {
  if (!g) return DBBC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  uint64_t h[2] = {0, 0};
  const dbbc_status st = guarded([&] {
    Scratch sc(s);
    unsigned long long* d_out = sc.get<unsigned long long>(2);
    unsigned* d_status = sc.get<unsigned>(1);
    DBBC_CUDA(cudaMemsetAsync(d_status, 0, sizeof(unsigned), s));
    DBBC_CUDA(cudaMemsetAsync(d_out, 0, 2 * sizeof(uint64_t), s));
    enqueue_count(g, s, d_out, d_status, sc);
    DBBC_CUDA(cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, s));
    check_status_word(d_status, s);  // synchronizes
  });
  if (st != DBBC_OK) return st;
  if (balanced) *balanced = h[0];
  if (unbalanced) *unbalanced = h[1];
  return DBBC_OK;
}

dbbc_status dbbc_count_profiled(const dbbc_graph* g, void* cuda_stream, uint64_t* balanced, uint64_t* unbalanced,
                                dbbc_count_profile* prof) {
  if (!g) return DBBC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  uint64_t h[2] = {0, 0};
  dbbc_count_profile p;
  std::memset(&p, 0, sizeof(p));
  const dbbc_status st = guarded([&] {
    Scratch sc(s);
    CountProfiler cp;
    unsigned long long* d_out = sc.get<unsigned long long>(2);
    unsigned* d_status = sc.get<unsigned>(1);
    DBBC_CUDA(cudaMemsetAsync(d_status, 0, sizeof(unsigned), s));
    DBBC_CUDA(cudaMemsetAsync(d_out, 0, 2 * sizeof(uint64_t), s));
    enqueue_count(g, s, d_out, d_status, sc, &cp);
    DBBC_CUDA(cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, s));
    check_status_word(d_status, s);  // synchronizes
    cp.summarize(&p);
  });
  if (st != DBBC_OK) return st;
  if (balanced) *balanced = h[0];
  if (unbalanced) *unbalanced = h[1];
  if (prof) *prof = p;
  return DBBC_OK;
}

uint64_t dbbc_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

dbbc_status dbbc_graph_export(const dbbc_graph* g, void* cuda_stream, int64_t* row_ptr, uint32_t* col,
                              uint32_t* lower, int32_t* vertex, uint64_t* work) {
  if (!g) return DBBC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return guarded([&] {
    if (row_ptr) DBBC_CUDA(cudaMemcpyAsync(row_ptr, g->row_ptr, (size_t)(g->n + 1) * 8, cudaMemcpyDeviceToHost, s));
    if (col && g->nnz) DBBC_CUDA(cudaMemcpyAsync(col, g->col, (size_t)g->nnz * 4, cudaMemcpyDeviceToHost, s));
    if (lower && g->n) DBBC_CUDA(cudaMemcpyAsync(lower, g->lower, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
    if (vertex && g->n) DBBC_CUDA(cudaMemcpyAsync(vertex, g->vertex, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
    if (work && g->n) DBBC_CUDA(cudaMemcpyAsync(work, g->work, (size_t)g->n * 8, cudaMemcpyDeviceToHost, s));
    DBBC_CUDA(cudaStreamSynchronize(s));
  });
}

}  // extern "C"
