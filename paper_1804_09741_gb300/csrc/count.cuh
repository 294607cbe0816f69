// Enumerate-and-classify launch (K2) and its planner.
#pragma once

#include "graph.cuh"

namespace mt {

const uint32_t* table_device(const mt_table* t);
int table_k(const mt_table* t);
uint32_t table_classes(const mt_table* t);
TableView table_view(const mt_table* t);
bool table_compact(const mt_table* t);

// Host-side shape of one counting launch over G graphs.
struct CountPlan {
  int K = 0;
  int G = 0;
  int nmax = 0;             // largest n among the graphs
  int dmax = 0;             // bound on every undirected degree
  int64_t fwd_bound = 0;    // bound on the number of forward entries, all graphs
  int64_t entry_stride = 0; // per-graph stride of the planner's entry arrays (>= max nu)
  int warps_per_block = 0;
  int blocks = 0;
  bool lab_smem = true;      // relation words in shared memory (else global slabs)
  bool gcache = true;        // the current graph's CSR copied into shared memory
  bool stack_global = false; // candidate stacks in global memory (hub graphs)
  int nu_cap = 0;            // capacity of that copy (undirected entries)
  size_t graph_bytes = 0, hist_bytes = 0, lab_bytes = 0, buf_bytes = 0, cell_bytes = 0;
  bool comb = false;         // count the last two positions by cells (Algorithm 1)
  bool compact = false;      // the table is the compact k = 6 form
  size_t map_bytes = 0;      // per-warp word relabelling (compact form)
  int cap = 0;              // stack entries per warp
  size_t smem_bytes = 0;
  uint64_t items_max = 0;
  double split_cost = 0.0;  // 0 = automatic
  double split_scale = 1.0; // multiplier of the automatic threshold
  double items_factor = 1.25;  // work items budget, in units of the automatic target
  uint32_t classes = 0;
  size_t ws_bytes = 0;
  // workspace offsets
  size_t off_hdr = 0, off_qhead = 0, off_est = 0, off_cnt = 0, off_items = 0, off_lab = 0;
  size_t off_stack = 0;
};

// Fill in the launch shape and the workspace size.  `fwd_bound` is a bound on
// the total number of forward entries (sum of undirected edges) of the G graphs.
mt_status count_configure(CountPlan* p, int K, int G, int nmax, int dmax, int64_t fwd_bound,
                          int64_t entry_stride, uint32_t classes, double split_cost,
                          int warps_per_block, bool compact = false);

// Same, with the tuning of include/motifs.h (nullptr = automatic).
// `compact`: the table is the compact k = 6 form (per-subgraph method only;
// MT_EUNSUPPORTED otherwise).
mt_status count_configure_tuned(CountPlan* p, int K, int G, int nmax, int dmax, int64_t fwd_bound,
                                int64_t entry_stride, uint32_t classes, const mt_tuning* tuning,
                                bool compact = false);

// Enqueue planner + enumerator.  `graphs` is a device array of G DevGraph whose
// hist pointers are already zeroed (the launch adds into them).  Roots in
// [root_begin, root_end) only.  No host synchronisation, no allocation.
// `copies` > 1 (k = 6, G = 1 only): block b adds into copy b mod copies of the
// graph's histogram, copy 0 being the graph's own and copy c >= 1 starting at
// copies_base + (c - 1) * copy_stride (zeroed by the caller, folded by the
// caller afterwards).
mt_status count_enqueue(const CountPlan& p, void* ws, const DevGraph* graphs,
                        const TableView& table, int32_t root_begin, int32_t root_end,
                        cudaStream_t s, unsigned long long* copies_base = nullptr,
                        int copies = 1, uint32_t copy_stride = 0);

// Read the launch's error word and item count from the workspace (device
// pointers into `ws`).  The header holding the error word is at offset 0 of
// every plan's workspace, so the error word's address does not depend on the
// plan.
uint32_t* count_err_ptr(const CountPlan& p, void* ws);
uint32_t* count_nitems_ptr(const CountPlan& p, void* ws);

}  // namespace mt
