/*
 * dbbc.h -- balanced / unbalanced butterfly counting in signed bipartite graphs
 * on one NVIDIA GB300 GPU (sm_103a).
 *
 * Problem (Section III, "Problem Statement"; Def. 1 and Def. 2): a signed
 * bipartite graph G = (U, V, E = E+ u E-) has a butterfly for every
 * {u, u'} in U and {v, v'} in V whose four edges all exist. The butterfly is
 * balanced when the number of negative edges among the four is even and
 * unbalanced when it is odd. This library returns both totals as exact 64-bit
 * integers.
 *
 * Method (Section IV-A, Algorithm 1, Phase 5; Lemma 1): vertices are ordered by
 * the Def. 3 priority (degree, then id, over U u V with unified ids
 * id(u) = u, id(v) = |U| + v). Every wedge u-v-w with p(v) < p(u) and
 * p(w) < p(u) adds one to a symmetric counter of w when s(u,v) = s(v,w) and to
 * an asymmetric counter otherwise; each (u, w) then contributes
 * C(sym,2) + C(asym,2) balanced and sym * asym unbalanced butterflies.
 *
 * Conventions shared by every entry point:
 *   - Vertex ids are per side: 0 <= u < n_u and 0 <= v < n_v, int32.
 *   - Signs are int8, +1 (positive) or -1 (negative). The paper writes a
 *     negative edge as sign 0 (Def. 2); here -1 is used instead.
 *   - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Work is ordered on that stream.
 *   - The library copies its inputs; the caller keeps ownership of every
 *     array it passes. A graph handle is owned by the caller until
 *     dbbc_graph_free.
 *   - On error, output parameters are left untouched and a status other than
 *     DBBC_OK is returned. No C++ exception crosses this interface.
 *   - Device memory is taken from the allocator set with dbbc_set_allocator,
 *     else stream-ordered on the call's stream from the library's own memory
 *     pool (see dbbc_set_allocator).
 *   - A handle may be read by several counts at once (each count allocates its
 *     own scratch); it must not be freed while a count on it is in flight.
 *     The one exception is dbbc_count_noalloc, which allocates nothing and
 *     whose calls share one fixed device array: its calls must not overlap
 *     on the GPU.
 */
#ifndef DBBC_H
#define DBBC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__) || defined(__clang__)
#define DBBC_API __attribute__((visibility("default")))
#else
#define DBBC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dbbc_graph dbbc_graph; /* opaque: device CSR, buckets, hub plan */

typedef enum {
  DBBC_OK = 0,
  DBBC_EINVAL = 1,    /* bad argument or input (id out of range, sign not +-1, m < 0, duplicate under DUP_REJECT) */
  DBBC_ENOMEM = 2,    /* a device allocation failed */
  DBBC_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
  DBBC_ETIMEOUT = 4,  /* reserved: no kernel of this library waits on another, so no call returns it */
  DBBC_EOVERFLOW = 5, /* a count or an internal capacity exceeded its type */
  DBBC_EINTERNAL = 6  /* an internal consistency check failed (a bug: please report) */
} dbbc_status;

enum {
  DBBC_INPUT_HOST = 0,   /* u, v, sign are host pointers (pageable or pinned) */
  DBBC_INPUT_DEVICE = 1, /* u, v, sign are device pointers */
  DBBC_DUP_KEEP_LAST = 0, /* repeated (u, v) pairs keep the sign of the last occurrence (Section V) */
  DBBC_DUP_REJECT = 2     /* repeated (u, v) pairs make the call fail with DBBC_EINVAL */
};

/* Build a graph from COO arrays (Def. 1 input; duplicates per Section V,
 * dataset preprocessing: the latest occurrence of a pair wins).
 *   u, v, sign : m entries each, host or device memory per `flags`.
 *   m          : number of input edges, 0 <= m < 2^31.
 *   n_u, n_v   : side sizes, 0 <= n_u, n_v and n_u + n_v < 2^31.
 *   flags      : DBBC_INPUT_* | DBBC_DUP_*.
 *   out        : receives a new handle on success.
 * Synchronous with respect to `cuda_stream` (it reads sizes back to the host).
 * Errors: DBBC_EINVAL (any id out of range, any sign not +-1, bad sizes or
 * flags, duplicates under DBBC_DUP_REJECT), DBBC_ENOMEM, DBBC_ECUDA. */
DBBC_API dbbc_status dbbc_graph_from_coo(const int32_t* u, const int32_t* v, const int8_t* sign, int64_t m, int32_t n_u,
                                int32_t n_v, uint32_t flags, void* cuda_stream, dbbc_graph** out);

/* Build the disjoint union of n_graphs graphs as one handle. Graph i's edges
 * are u, v, sign [edge_offsets[i], edge_offsets[i+1]) with ids local to graph
 * i (0 <= u < n_u[i], 0 <= v < n_v[i]); edge_offsets (n_graphs + 1 entries,
 * starting at 0), n_u and n_v are HOST arrays; u, v, sign are host or device
 * per `flags` as in dbbc_graph_from_coo. Butterflies never span two
 * components, and shifting each component's ids by a constant per side keeps
 * its Def. 3 order, so dbbc_count_components returns exactly what counting
 * every graph alone would (Theorem 1); dbbc_count returns their sum. One build
 * pipeline serves all graphs. Errors as dbbc_graph_from_coo; the union must
 * have < 2^31 edges and < 2^31 vertices. */
DBBC_API dbbc_status dbbc_graph_from_coo_multi(const int32_t* u, const int32_t* v, const int8_t* sign,
                                               const int64_t* edge_offsets, const int32_t* n_u, const int32_t* n_v,
                                               int32_t n_graphs, uint32_t flags, void* cuda_stream,
                                               dbbc_graph** out);

/* Per-component counts of a handle: balanced[i] and unbalanced[i] (host
 * arrays of n_components entries, see dbbc_graph_info) for component i of a
 * dbbc_graph_from_coo_multi handle; one entry for a plain handle. Synchronous. */
DBBC_API dbbc_status dbbc_count_components(const dbbc_graph* g, void* cuda_stream, uint64_t* balanced,
                                           uint64_t* unbalanced);

/* Butterflies containing each vertex: balanced_v[x] and unbalanced_v[x]
 * (HOST arrays of n_u + n_v entries, indexed by unified id: U vertex u is u,
 * V vertex v is n_u + v; for a dbbc_graph_from_coo_multi handle the ids are
 * the union's, graph i's U vertex u at sum_{j<i} n_u[j] + u and its V vertex v
 * at N_U + sum_{j<i} n_v[j] + v, N_U the union's U side). Each butterfly of
 * Def. 4 counted by dbbc_count is credited to its four vertices, so each array
 * sums to four times the matching total. Computed by Algorithm 1 with a second
 * walk of every pivot's wedges once its endpoint counts (Lemma 1's B1, B2) are
 * final. Synchronous. Errors: DBBC_EINVAL (NULL graph, NULL array with
 * vertices), DBBC_ENOMEM, DBBC_ECUDA, DBBC_EINTERNAL (a device-side check
 * failed). */
DBBC_API dbbc_status dbbc_count_vertices(const dbbc_graph* g, void* cuda_stream, uint64_t* balanced_v,
                                         uint64_t* unbalanced_v);

/* Butterflies containing each queried edge: balanced_e[i] and
 * unbalanced_e[i] for the pair (qu[i], qv[i]) (U id, V id, as passed to the
 * build; a union handle takes the union's ids as in dbbc_count_vertices). A
 * pair that is not an edge of the graph is in no butterfly and gets zeros; a
 * pair passed to the build several times answers for the edge it became
 * (latest sign). Every butterfly counted by dbbc_count is credited to its four
 * edges, so over all distinct edges each array sums to four times the
 * matching total. Computed by Algorithm 1 with a second walk of every pivot's
 * wedges once Lemma 1's B1, B2 are final: a wedge u-v-w pairs with the other
 * wedges ending at w, which closes one butterfly through (u, v) and (v, w)
 * per pair.
 *   qu, qv, balanced_e, unbalanced_e : k entries each, all four HOST or all
 *       four DEVICE memory per `flags` (DBBC_INPUT_HOST / DBBC_INPUT_DEVICE).
 * Device scratch: 16 bytes per CSR entry (2m) plus 4 bytes per vertex.
 * Synchronous. Errors: DBBC_EINVAL (NULL graph or array, k < 0, unknown
 * flags, an id out of range), DBBC_ENOMEM, DBBC_ECUDA, DBBC_EINTERNAL. */
DBBC_API dbbc_status dbbc_count_edges(const dbbc_graph* g, void* cuda_stream, const int32_t* qu, const int32_t* qv,
                                      int64_t k, uint32_t flags, uint64_t* balanced_e, uint64_t* unbalanced_e);

/* Count balanced and unbalanced butterflies of one graph (Algorithm 1,
 * Phase 5, with the Lemma 1 unbalanced count). Host out-parameters; the call
 * returns after the counts are on the host. Either pointer may be NULL. */
DBBC_API dbbc_status dbbc_count(const dbbc_graph* g, void* cuda_stream, uint64_t* balanced, uint64_t* unbalanced);

/* Same as dbbc_count but asynchronous: writes {balanced, unbalanced} to the
 * DEVICE array d_out[2] in stream order and returns after enqueueing. */
DBBC_API dbbc_status dbbc_count_async(const dbbc_graph* g, void* cuda_stream, uint64_t* d_out);

/* Per-tier timings of one count, measured with CUDA events on the call's
 * stream around the tier's kernels (milliseconds), with launch counts and the
 * number of (lower neighbour, window) visits the hub sweep made in list mode
 * (the visits of the other hub items are dbbc_graph_info.hub_cursor_steps). */
typedef struct {
  float ms_light, ms_medium, ms_hub_aggregate, ms_hub_finalize, ms_total;
  int64_t launches_light, launches_medium, launches_hub_aggregate, launches_hub_finalize;
  uint64_t hub_list_visits;
} dbbc_count_profile;

/* dbbc_count plus per-tier timings in *prof (may be NULL). Synchronous. */
DBBC_API dbbc_status dbbc_count_profiled(const dbbc_graph* g, void* cuda_stream, uint64_t* balanced,
                                         uint64_t* unbalanced, dbbc_count_profile* prof);

/* Number of CUDA kernels this library has launched in this process so far
 * (graph builds and counts). */
DBBC_API uint64_t dbbc_kernel_launches(void);

/* Counting without allocating device memory, for callers that cannot call
 * cudaMalloc while they count (a fixed device-memory budget held by another
 * allocator, work that must not touch the device allocator, set-up-once
 * hosts). The paper has no counterpart; this is a deployment entry point.
 *   d_out : DEVICE array of two uint64 {balanced, unbalanced}, written in
 *           stream order; the call returns after enqueueing (like
 *           dbbc_count_async, device-side status bits are not reported).
 * Scratch comes from one fixed 32 MiB array inside the library, held on
 * every GPU that loads the library until the process exits. The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress),
 * so make the first call on each device before any stream capture. All calls
 * share the array and it keeps the previous call's contents (the parts that
 * must start at zero are cleared by each call); calls that overlap on the GPU,
 * on any streams, race on it, so serialize them. Graphs whose largest hub
 * needs more cursor scratch than the array holds (8 bytes per lower
 * neighbour of that hub for even one CTA) are rejected with DBBC_EOVERFLOW;
 * below that limit fewer CTAs run the hub tier when the array cannot hold
 * cursors for all of them. */
DBBC_API dbbc_status dbbc_count_noalloc(const dbbc_graph* g, void* cuda_stream, uint64_t* d_out);

/* Count several resident graphs in one launch sequence (a temporary batch
 * plan, see dbbc_batch_create). balanced[i] and unbalanced[i] (host arrays of
 * n_graphs entries) receive graph i's counts. Synchronous. */
DBBC_API dbbc_status dbbc_count_batch(const dbbc_graph* const* gs, int32_t n_graphs, void* cuda_stream, uint64_t* balanced,
                             uint64_t* unbalanced);

/* Asynchronous batch: d_out is a DEVICE array [n_graphs][2] of
 * {balanced, unbalanced}. Returns after enqueueing. */
DBBC_API dbbc_status dbbc_count_batch_async(const dbbc_graph* const* gs, int32_t n_graphs, void* cuda_stream,
                                   uint64_t* d_out);

/* Batch plan over resident graphs: their light and medium pivots and their
 * hub work items (in descending estimated work across all graphs) form one
 * work list, counted by one kernel per tier for all graphs. The first count
 * captures that sequence into a CUDA graph; later counts replay it. The graphs
 * must stay alive and unchanged while the plan exists. Counts of one plan
 * must not overlap on the GPU (they share the plan's scratch). */
typedef struct dbbc_batch dbbc_batch;
DBBC_API dbbc_status dbbc_batch_create(const dbbc_graph* const* gs, int32_t n_graphs, void* cuda_stream,
                                       dbbc_batch** out);
/* Replay the plan; d_out (DEVICE [n_graphs][2], may be NULL) receives the
 * counts in stream order. Returns after enqueueing. */
DBBC_API dbbc_status dbbc_batch_count_async(dbbc_batch* b, void* cuda_stream, uint64_t* d_out);
/* Replay the plan and copy the counts to host arrays of n_graphs entries. */
DBBC_API dbbc_status dbbc_batch_count(dbbc_batch* b, void* cuda_stream, uint64_t* balanced, uint64_t* unbalanced);
DBBC_API void dbbc_batch_free(dbbc_batch* b);

typedef struct {
  int32_t n_u, n_v;
  int64_t m_input;     /* edges passed in */
  int64_t m;           /* distinct edges kept */
  uint64_t wedges;     /* accepted wedges of Algorithm 1 (sum over all pivots) */
  int64_t n_pivots;    /* pivots with at least two lower neighbours and one accepted wedge */
  int64_t n_light, n_medium, n_hub; /* pivots per counting tier */
  uint64_t wedges_light, wedges_medium, wedges_hub;
  int64_t lower_light, lower_medium, lower_hub; /* lower neighbours summed over the tier's pivots */
  int64_t hub_items;         /* hub work items (a hub and a span of its endpoint windows) */
  int64_t hub_cursor_inits;  /* sum over hub items of the hub's lower neighbours */
  int64_t hub_cursor_steps;  /* sum over hub items swept by cursors of lower neighbours x windows (list-mode
                                items visit only the windows that hold a neighbour's entries; see
                                dbbc_count_profile.hub_list_visits) */
  size_t device_bytes; /* device memory held by the handle */
  int32_t n_components; /* graphs in a dbbc_graph_from_coo_multi handle, else 1 */
} dbbc_graph_info;

/* Sizes and the per-tier wedge split of a built graph. */
DBBC_API dbbc_status dbbc_graph_get_info(const dbbc_graph* g, dbbc_graph_info* info);

/* Device bytes held by a handle (for admission control). 0 for NULL. */
DBBC_API size_t dbbc_graph_device_bytes(const dbbc_graph* g);

/* Upper estimate of the peak device bytes dbbc_graph_from_coo needs for a
 * graph of this size (handle plus build scratch). A count needs scratch of its
 * own on top of the handle, mostly the hub sweep's neighbour lists: at most
 * 2^23 slots of 8 bytes per SM, in practice a few slots per lower neighbour of
 * the largest sparse hub per SM. */
DBBC_API size_t dbbc_estimate_bytes(int64_t m, int32_t n_u, int32_t n_v);

/* Release a handle (NULL is a no-op). Frees in stream order on the stream the
 * handle was built on. */
DBBC_API void dbbc_graph_free(dbbc_graph* g);

/* Export the device CSR for inspection (tests and tools). All arrays are HOST
 * buffers sized by the caller from dbbc_graph_get_info:
 *   row_ptr[n_u + n_v + 1] (int64), col[2m] (uint32 (side_rank << 1) | negative),
 *   lower[n_u + n_v] (uint32, lower-priority neighbours per row),
 *   vertex[n_u + n_v] (int32 unified id of each row), work[n_u + n_v]
 *   (uint64 accepted wedges with that row as pivot).
 * Rows 0..n_u-1 are U vertices in ascending Def. 3 priority, rows n_u..n-1
 * are V vertices in ascending priority; any pointer may be NULL. */
DBBC_API dbbc_status dbbc_graph_export(const dbbc_graph* g, void* cuda_stream, int64_t* row_ptr, uint32_t* col,
                              uint32_t* lower, int32_t* vertex, uint64_t* work);

/* Device allocator hook (e.g. a framework's caching allocator). alloc returns
 * NULL on failure. Passing NULL for both restores the default: stream-ordered
 * allocations (cudaMallocFromPoolAsync) from one memory pool per device owned
 * by the library, which keeps up to 8 GiB of freed memory mapped between
 * calls instead of returning it to the device at every synchronization.
 * Not thread-safe against concurrent library calls. */
DBBC_API void dbbc_set_allocator(void* (*alloc_fn)(size_t bytes, void* cuda_stream, void* ctx),
                        void (*free_fn)(void* ptr, void* cuda_stream, void* ctx), void* ctx);

/* Greedy bin packing of Phase 3 (Section IV-A, Example 2): items in
 * descending `work` order, each to the part with the smallest load so far
 * (lowest part index on ties). Host arrays: work[n_items] in, part_of[n_items]
 * and loads[n_parts] out. Pure host code (no GPU). */
DBBC_API dbbc_status dbbc_lpt_partition(const uint64_t* work, int64_t n_items, int32_t n_parts, int32_t* part_of,
                                        uint64_t* loads);

/* Counts of the pivots that dbbc_lpt_partition assigns to `part` of
 * `n_parts` by their accepted wedges (a hub's work items stay with it): with
 * the graph replicated on n_parts GPUs, GPU k counts part k and the 16-byte
 * results add up to dbbc_count's (Theorem 1). Host out-parameters;
 * synchronous. */
DBBC_API dbbc_status dbbc_count_partition(const dbbc_graph* g, void* cuda_stream, int32_t part, int32_t n_parts,
                                          uint64_t* balanced, uint64_t* unbalanced);

/* Tuning of the counting tiers, applied to graphs built after the call (a
 * handle keeps the values it was built with). Chosen per GPU by the
 * project's autotuner (paper_2609_21848_gb300/autotune.py); every setting only
 * changes speed, never a count.
 *   light_max_work  : pivots with at most this many accepted wedges use one
 *                     warp each (1..512);
 *   medium_max_work : ... and up to this many one CTA each (light..4096);
 *                     more go to the hub window sweep;
 *   hub_item_work   : target accepted wedges per hub work item (>= 1024);
 *   group_density   : mean (lower neighbour, window) segment lengths at which
 *                     32, 16, 8 and 4 lanes walk a segment (descending);
 *   hash_mult_log   : shared hash tables get at least 2^hash_mult_log slots
 *                     per accepted wedge of the pivot (1..3; capped by the
 *                     tier's table size, never below 2 per wedge);
 *   list_density    : hubs whose mean (lower neighbour, window) segment is
 *                     shorter than this (>= 0; 0 turns it off) sweep in list
 *                     mode, visiting a neighbour only in the windows that
 *                     hold its entries;
 *   list_group_log  : lanes per neighbour segment in list mode, log2 (0 or
 *                     2..5: one lane, or lane groups of 4 to 32);
 *   finalize_window_wedges : hub work items with at least this many accepted
 *                     wedges per window (estimated) finalise each window by
 *                     one scan of its counters (C(p,2) + C(q,2) and p*q per
 *                     endpoint, Lemma 1) when clearing it; sparser items add
 *                     every wedge's Lemma 1 contribution as it is counted
 *                     (0: every item scans; UINT64_MAX: none does);
 *   list_wide_density : list-mode items whose mean (lower neighbour, window)
 *                     segment is at least this (>= 0) walk each segment with
 *                     at least 8 lanes instead of 2^list_group_log.
 * Setting and reading the tuning is safe against builds on other threads. */
typedef struct {
  uint64_t light_max_work;
  uint64_t medium_max_work;
  uint64_t hub_item_work;
  double group_density[4];
  int32_t hash_mult_log;
  double list_density;
  int32_t list_group_log;
  uint64_t finalize_window_wedges;
  double list_wide_density;
} dbbc_tuning;
DBBC_API dbbc_status dbbc_set_tuning(const dbbc_tuning* t); /* NULL restores the defaults; DBBC_EINVAL if out of range */
DBBC_API void dbbc_get_tuning(dbbc_tuning* t);

/* Static description of a status code. */
DBBC_API const char* dbbc_status_string(dbbc_status s);

/* Library version as "major.minor.patch" ("+checked" appended in a checked build). */
DBBC_API const char* dbbc_version(void);

/* Checked builds. A library compiled with -DDBBC_CHECKED=1 is a debug build of
   the same kernels in which every index derived from graph data is tested
   before the access it guards: CSR row and entry positions, the shared-memory
   address of every window counter of the hub sweep (and that the entry lies at
   or past the window's first rank), cursor and neighbour-list slots against
   their capacity, and per-vertex / per-edge output positions. A failed test
   skips the access (the counts are then wrong) and records bit 2 in a flag
   word of the library; nothing traps. Synchronous calls (dbbc_count,
   dbbc_count_profiled, dbbc_graph_from_coo[_multi], dbbc_count_vertices,
   dbbc_count_edges, dbbc_batch_count, ...) collect the flags before they
   return and fail with DBBC_EINTERNAL when one is set.

   dbbc_is_checked: 1 in a checked build, 0 in a regular one.
   dbbc_checked_flags: synchronizes the current device, stores in *flags the OR
   of the bits recorded since the last collection (2: an index left its array)
   and clears them; in a regular build stores 0. DBBC_EINVAL if flags is NULL,
   DBBC_ECUDA if the device cannot be synchronized. The flag words are per
   device and per process: calls on several host threads share them. */
DBBC_API int dbbc_is_checked(void);
DBBC_API dbbc_status dbbc_checked_flags(uint32_t* flags);

#ifdef __cplusplus
}
#endif

#endif /* DBBC_H */
