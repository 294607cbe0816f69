// Host-side graph handle and the device graph builder (sorted CSR + labelled
// undirected CSR) shared by the loader, the randomiser and the batch path.
#pragma once

#include "common.cuh"

struct mt_graph {
  int32_t n = 0, m = 0;
  int32_t nu = 0, dmax = 0;    // filled after the build (host copy of the stats)
  int32_t* row_ptr = nullptr;  // device, n+1
  int32_t* col = nullptr;      // device, m (sorted rows)
  int32_t* urow = nullptr;     // device, n+1
  uint32_t* ucol = nullptr;    // device, 2m (nu used)
  int32_t* usrc = nullptr;     // device, 2m
  int32_t* ufwd = nullptr;     // device, n
  void* mem = nullptr;         // one allocation backing all of the above
  bool pooled = false;         // mem came from the stream-ordered pool (cudaMallocAsync)

  // Counting scratch, grown on demand by mt_count, or the caller's buffer
  // attached by mt_set_workspace (ws_owned false: never grown or freed here).
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = true;
  // Where the last count left its error word and item count inside `ws`.
  bool stats_valid = false;
  size_t off_err = 0, off_nitems = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace mt {

// Per-graph results of the builder.
struct BuildStats {
  int32_t nu;
  int32_t dmax;
  uint32_t err;
  int32_t pad;
};

// Pointers of G equally sized graphs laid out with fixed strides.
struct BuildArgs {
  int32_t n, m, G;
  const int32_t* row_ptr;   // stride row_stride (0: shared by all graphs)
  int64_t row_stride;
  const int32_t* col_in;    // unsorted destinations, stride m
  int32_t* col_out;         // sorted destinations, stride m (may alias nothing else)
  int32_t* in_ptr;          // scratch n+1 per graph
  int32_t* in_tmp;          // scratch m per graph
  int32_t* in_col;          // scratch m per graph
  int32_t* cursor;          // scratch n per graph
  int32_t* urow;            // n+1 per graph
  uint32_t* ucol;           // 2m per graph
  int32_t* usrc;            // 2m per graph
  int32_t* ufwd;            // n per graph
  BuildStats* stats;        // one per graph
};

// Enqueue the builder (one thread block per graph).
cudaError_t launch_build(const BuildArgs& a, cudaStream_t s);

// Bytes of builder scratch per graph.
inline size_t build_scratch_ints(int32_t n, int32_t m) {
  return (size_t)(n + 1) + (size_t)m * 2 + (size_t)n;
}

DevGraph dev_view(const mt_graph* g, unsigned long long* hist);

// Host-side checks of a CSR (MT_OK, MT_EINVAL or MT_EUNSUPPORTED).
mt_status validate_csr(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col);

// Load a graph with stream-ordered allocations on `s` (no device-wide sync);
// release it with graph_release on a stream.  Synchronises `s` only.
mt_status graph_load_on(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col,
                        cudaStream_t s, mt_graph** out);
void graph_release(mt_graph* g, cudaStream_t s);
size_t graph_device_bytes(int32_t n, int32_t m);

}  // namespace mt
