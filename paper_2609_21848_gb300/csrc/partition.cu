// Pivot partitioning for counting one graph on several GPUs (Phase 3,
// Section IV-A, greedy bin packing as in Example 2): pivots in descending
// accepted-wedge order, each to the least-loaded part. Every part's pivots
// are counted by a one-graph batch plan; the parts' counts add up to the
// graph's (Theorem 1: each butterfly is counted at exactly one pivot).
#include <algorithm>
#include <queue>
#include <vector>

#include "internal.h"

namespace dbbc {
// batch.cu: counts of one graph restricted to the given pivots / hub items
void count_subset(const dbbc_graph* g, cudaStream_t s, const std::vector<int32_t>& medium_rows,
                  const std::vector<int32_t>& light_rows, const std::vector<SweepItem>& hub_items, uint64_t* balanced,
                  uint64_t* unbalanced);
}  // namespace dbbc

using namespace dbbc;

extern "C" {

dbbc_status dbbc_lpt_partition(const uint64_t* work, int64_t n_items, int32_t n_parts, int32_t* part_of,
                               uint64_t* loads) {
  if (n_items < 0 || n_parts <= 0 || (n_items > 0 && (!work || !part_of)) || !loads) return DBBC_EINVAL;
  try {
    std::vector<int64_t> order((size_t)n_items);
    for (int64_t i = 0; i < n_items; i++) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return work[a] > work[b]; });
    // min-heap on (load, part): the least-loaded part, lowest index on ties
    using Slot = std::pair<uint64_t, int32_t>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
    for (int32_t p = 0; p < n_parts; p++) heap.push({0, p});
    std::vector<uint64_t> ld((size_t)n_parts, 0);
    for (int64_t i : order) {
      Slot s = heap.top();
      heap.pop();
      part_of[i] = s.second;
      s.first += work[i];
      ld[(size_t)s.second] = s.first;
      heap.push(s);
    }
    std::copy(ld.begin(), ld.end(), loads);
  } catch (...) {
    return DBBC_ENOMEM;
  }
  return DBBC_OK;
}

dbbc_status dbbc_count_partition(const dbbc_graph* g, void* cuda_stream, int32_t part, int32_t n_parts,
                                 uint64_t* balanced, uint64_t* unbalanced) {
  if (!g || n_parts <= 0 || part < 0 || part >= n_parts) return DBBC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  try {
    // pivots in descending work with their work (the graph's tier order)
    std::vector<int32_t> rows((size_t)g->n_piv);
    std::vector<uint64_t> work((size_t)g->n_piv);
    if (g->n_piv > 0) {
      std::vector<uint64_t> all((size_t)g->n);
      DBBC_CUDA(cudaMemcpyAsync(rows.data(), g->order, rows.size() * 4, cudaMemcpyDeviceToHost, s));
      DBBC_CUDA(cudaMemcpyAsync(all.data(), g->work, all.size() * 8, cudaMemcpyDeviceToHost, s));
      DBBC_CUDA(cudaStreamSynchronize(s));
      for (size_t i = 0; i < rows.size(); i++) work[i] = all[(size_t)rows[i]];
    }
    std::vector<int32_t> part_of(rows.size());
    std::vector<uint64_t> loads((size_t)n_parts);
    const dbbc_status st = dbbc_lpt_partition(work.data(), (int64_t)rows.size(), n_parts, part_of.data(),
                                              loads.data());
    if (st != DBBC_OK) return st;
    std::vector<int32_t> med, light;
    std::vector<uint8_t> mine((size_t)g->n, 0);
    for (size_t i = 0; i < rows.size(); i++) {
      if (part_of[i] != part) continue;
      mine[(size_t)rows[i]] = 1;
      if ((int64_t)i >= g->n_hub + g->n_medium) light.push_back(rows[i]);
      else if ((int64_t)i >= g->n_hub) med.push_back(rows[i]);
    }
    std::vector<SweepItem> hubs;
    for (const SweepItem& it : g->sweep_items_host)
      if (mine[(size_t)it.row]) hubs.push_back(it);
    count_subset(g, s, med, light, hubs, balanced, unbalanced);
  } catch (const Error& e) {
    return e.status;
  } catch (...) {
    return DBBC_EINTERNAL;
  }
  return DBBC_OK;
}

}  // extern "C"
