// Internal layout of a built graph and the launch entry points shared by the
// library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/dbbc.h"
#include "common.cuh"

namespace dbbc {

// Counting tiers by accepted wedges W(p) of a pivot (defaults; see Tuning).
constexpr uint64_t kLightMaxWork = 512;    // warp per pivot, per-warp shared hash (<= 1024 slots)
constexpr uint64_t kMediumMaxWork = 4096;  // CTA per pivot, shared hash (<= 8192 slots)
constexpr int kLightSlots = 1024;
constexpr int kMediumSlots = 8192;
// Hub window sweep: shared-memory windows of side ranks (224 KB of counters
// by default). Build-time overrides exist for tuning.
#ifndef DBBC_SWEEP_WINDOW16
#define DBBC_SWEEP_WINDOW16 57344
#endif
#ifndef DBBC_SWEEP_THREADS
#define DBBC_SWEEP_THREADS 1024
#endif
// entries per lane per chunk of the per-vertex / per-edge window walks (4
// measured 5% faster than 2 on GB300)
#ifndef DBBC_SWEEP_UNROLL
#define DBBC_SWEEP_UNROLL 4
#endif
constexpr uint32_t kSweepWindow16 = DBBC_SWEEP_WINDOW16;     // 32-bit counters packing two 16-bit halves
constexpr uint32_t kSweepWindow32 = DBBC_SWEEP_WINDOW16 / 2;  // 64-bit counters packing two 32-bit halves
constexpr uint64_t kSweepItemWork = 1u << 20;  // target accepted wedges per work item
// mean (neighbour, window) segment length at which 32 / 16 / 8 / 4 lanes walk a segment
#ifndef DBBC_GROUP_T32
#define DBBC_GROUP_T32 40
#endif
#ifndef DBBC_GROUP_T16
#define DBBC_GROUP_T16 16
#endif
#ifndef DBBC_GROUP_T8
#define DBBC_GROUP_T8 6
#endif
#ifndef DBBC_GROUP_T4
#define DBBC_GROUP_T4 2
#endif
// Hub items in list mode (see sweep_device.cuh) run in spans of at most
// kListMaxWindows windows, with at most kListCapEntries list slots (8 bytes
// each) per CTA. Longer spans re-queue fewer neighbours between spans: on the
// 300M-edge polarized graph 128 windows and 2^23 slots (up to 10 GB of list
// scratch over 152 CTAs) swept 2.0% faster than 64 and 2^22; 2^24 slots gained
// another 0.6% but held twice the scratch, which the memory pool then had to
// map again for the next build.
#ifndef DBBC_LIST_MAX_WINDOWS
#define DBBC_LIST_MAX_WINDOWS 128
#endif
#ifndef DBBC_LIST_CAP_LOG
#define DBBC_LIST_CAP_LOG 23
#endif
constexpr int kListMaxWindows = DBBC_LIST_MAX_WINDOWS;
constexpr int64_t kListCapEntries = int64_t{1} << DBBC_LIST_CAP_LOG;

// Hub items with at least this many estimated wedges per window finalise each
// window by a scan of its counters (kItemFinalize); sparser ones take the
// Lemma 1 contribution of every wedge from its atomic's old value.
constexpr uint64_t kFinalizeWindowWedges = 65536;

// Runtime tuning (dbbc_set_tuning), snapshotted into every graph at build.
struct Tuning {
  uint64_t light_max_work = kLightMaxWork;
  uint64_t medium_max_work = kMediumMaxWork;
  uint64_t hub_item_work = kSweepItemWork;
  double group_density[4] = {DBBC_GROUP_T32, DBBC_GROUP_T16, DBBC_GROUP_T8, DBBC_GROUP_T4};
  int32_t hash_mult_log = 1;
  double list_density = 8.0;  // hubs with a mean (neighbour, window) segment shorter than this use list mode
  int32_t list_group_log = 2; // lanes per neighbour segment in list mode (log2)
  uint64_t finalize_window_wedges = kFinalizeWindowWedges;  // see kItemFinalize
  double list_wide_density = 1e30;  // list-mode items with a mean segment at least this use >= 8 lanes
};
Tuning current_tuning();  // a copy, taken under the tuning lock

// Throws the error a kernel status word h (already read back) stands for; in
// a checked build it first adds the bounds-check flags of every kernel run
// since the last collection (synchronizing the device).
void raise_device_status(unsigned h);

// Counts below this fit the 16-bit halves of a narrow counter.
constexpr int32_t kNarrowCountLimit = 65536;

// One unit of hub work: endpoints with side ranks [lo, hi) of hub row `row`,
// swept in windows whose counters are as narrow as the counts allow: ranks
// below q_end in quarter windows (4-bit halves, 4 * kSweepWindow16 ranks),
// below t_end in tiny ones (8-bit halves, 2 * kSweepWindow16 ranks), below
// n_end in narrow ones (16-bit halves, kSweepWindow16 ranks), the rest in wide
// ones (32-bit halves, kSweepWindow32 ranks); q_end, t_end and n_end are the
// hub's boundaries (clamped to the item). Each lower neighbour's segment is
// walked by 2^group_log lanes. A count never exceeds the endpoint's degree nor
// the hub's lower-neighbour count.
struct SweepItem {
  int32_t row;
  uint32_t lo;
  uint32_t hi;
  uint32_t q_end;
  uint32_t t_end;
  uint32_t n_end;
  int16_t group_log;
  int16_t flags;  // kItemList | kItemFinalize
};
constexpr int16_t kItemList = 2;  // list mode: visit a neighbour only in windows holding its entries
// counters of a window are finalised when it is cleared (C(p,2) + C(q,2) and
// p*q per endpoint) instead of wedge by wedge
constexpr int16_t kItemFinalize = 4;
// the item starts at its hub's first accepted rank: no row lists a rank below
// it, so a neighbour's cursor starts at the row's first entry (no search)
constexpr int16_t kItemFirst = 8;
// Counts below this fit the 8-bit halves of a tiny counter, and below the
// next the 4-bit halves of a quarter counter.
constexpr int32_t kTinyCountLimit = 256;
constexpr int32_t kQuarterCountLimit = 16;

// Read-only view of the device CSR passed to kernels by value.
// Rows [0, n_u) are U vertices in ascending Def. 3 priority, rows [n_u, n)
// V vertices in ascending priority. A row lists its neighbours by ascending
// priority as (side_rank << 1) | negative; the first lower[r] of them have
// lower priority than the row's vertex.
struct CsrView {
  const int64_t* row_ptr;
  const uint32_t* col;
  const uint32_t* lower;
  int32_t n_u;
  int64_t n;
  int64_t nnz;  // row_ptr[n]
};

}  // namespace dbbc


struct dbbc_graph {
  int device = 0;
  cudaStream_t stream = nullptr;  // stream the handle was built on (frees are ordered on it)
  int32_t n_u = 0, n_v = 0;
  int64_t n = 0;        // rows = n_u + n_v
  int64_t m_input = 0;  // edges passed in
  int64_t m = 0;        // distinct edges
  int64_t nnz = 0;      // 2m
  int64_t* row_ptr = nullptr;  // [n + 1]
  uint32_t* col = nullptr;     // [nnz]
  uint32_t* lower = nullptr;   // [n]
  int32_t* vertex = nullptr;   // [n] unified id per row
  uint64_t* work = nullptr;    // [n] accepted wedges per pivot row
  int32_t* order = nullptr;    // [n_piv] pivot rows, descending work: hubs | medium | light
  int64_t n_piv = 0, n_hub = 0, n_medium = 0, n_light = 0;
  uint64_t wedges = 0, wedges_hub = 0, wedges_medium = 0, wedges_light = 0;
  int64_t lower_hub = 0, lower_medium = 0, lower_light = 0;
  int64_t hub_cursor_inits = 0, hub_cursor_steps = 0;
  // hub plan: window-span items in descending estimated work
  dbbc::SweepItem* sweep_items = nullptr;
  int64_t n_sweep_items = 0;
  std::vector<dbbc::SweepItem> sweep_items_host;  // same items on the host (batch planning)
  std::vector<uint64_t> sweep_est_host;           // their estimated accepted wedges
  int64_t sweep_max_lower = 0;  // largest lower-neighbour count of a hub (cursor scratch per CTA)
  int64_t sweep_list_cap = 0;   // largest windows x lower neighbours of a list-mode item (list slots per CTA)
  int64_t narrow_ranks_u = 0, narrow_ranks_v = 0;  // per side: vertices of degree < 2^16 (a rank prefix)
  int64_t tiny_ranks_u = 0, tiny_ranks_v = 0;      // per side: vertices of degree < 2^8 (a rank prefix)
  int64_t quarter_ranks_u = 0, quarter_ranks_v = 0;  // per side: vertices of degree < 2^4 (a rank prefix)
  int64_t zero_ranks_u = 0, zero_ranks_v = 0;      // per side: vertices of degree 0 (a rank prefix; no row lists them)
  // disjoint union of several graphs (dbbc_graph_from_coo_multi): component
  // of every row, 0 for a plain handle (n_components == 1)
  int32_t n_components = 1;
  dbbc::Tuning tune;  // tuning the handle was built with
  int32_t* component = nullptr;  // [n] or nullptr for a plain handle
  size_t device_bytes = 0;
  std::vector<void*> allocations;
};

namespace dbbc {

// prep.cu
// Components of a union being built: host and device copies of the per-side
// id offsets (n_graphs + 1 entries each) and the largest side of any component.
struct UnionSpec {
  int32_t n_graphs = 1;
  std::vector<int64_t> uoff, voff;
  const int64_t* d_uoff = nullptr;
  const int64_t* d_voff = nullptr;
  int64_t max_side = 0;
};
void build_graph(dbbc_graph* g, const int32_t* u, const int32_t* v, const int8_t* s, int64_t m, bool on_device,
                 bool reject_duplicates, cudaStream_t stream, const UnionSpec* un = nullptr);
void build_graph_multi(dbbc_graph* g, const int32_t* u, const int32_t* v, const int8_t* s,
                       const int64_t* edge_offsets, const int32_t* n_u, const int32_t* n_v, int32_t n_graphs,
                       bool on_device, bool reject_duplicates, cudaStream_t stream);
void free_graph_memory(dbbc_graph* g);
void* graph_alloc(dbbc_graph* g, size_t bytes);

// Event brackets around tiers of one count (profiled counts only).
struct CountProfiler {
  enum Tier { LIGHT = 0, MEDIUM = 1, HUB_AGG = 2, HUB_FIN = 3, TOTAL = 4, NTIERS = 5 };
  struct Mark {
    int tier;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  unsigned long long* d_visits = nullptr;  // device counter of list-mode (neighbour, window) visits
  uint64_t list_visits = 0;
  int64_t launches[NTIERS] = {0, 0, 0, 0, 0};
  cudaEvent_t begin(cudaStream_t s);
  void end(int tier, cudaEvent_t a, cudaStream_t s);
  // after the stream has been synchronized
  void summarize(dbbc_count_profile* out);
  ~CountProfiler();
};

// count.cu: enqueue the counting kernels of one graph, accumulating
// {balanced, unbalanced} into d_out[0..1] (device, must be zeroed by caller).
void enqueue_count(const dbbc_graph* g, cudaStream_t stream, unsigned long long* d_out, unsigned* d_status,
                   Scratch& scratch, CountProfiler* prof = nullptr);

// count.cu: the same kernels with caller-supplied scratch (see noalloc.cu).
void enqueue_count_prealloc(const dbbc_graph* g, cudaStream_t stream, unsigned long long* d_out, unsigned* d_status,
                            int* d_next, uint32_t* cursors, size_t cursor_bytes);

}  // namespace dbbc
