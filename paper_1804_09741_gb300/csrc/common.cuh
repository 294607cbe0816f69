// Shared definitions of the Motifs-k CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/motifs.h"

namespace mt {

constexpr int kMaxVertices = 65535;  // vertex ids are stored as uint16 on the device stacks
constexpr uint32_t kNoClass = 0xFFFFFFFFu;

// Number of weakly connected classes for k = 0..6 (index = k).
constexpr uint32_t kNumClasses[7] = {0, 1, 2, 13, 199, 9364, 1530843};

// Error bits written by kernels into a device status word.
constexpr uint32_t kErrStackOverflow = 1u;
constexpr uint32_t kErrDuplicateArc = 2u;
constexpr uint32_t kErrWaitLimit = 4u;  // a bounded device wait gave up

// Undirected neighbour entry: vertex id in bits 0..29, bit 30 set iff the arc
// row-vertex -> neighbour exists, bit 31 set iff neighbour -> row-vertex exists
// (the A/B/C relation of Sec. 2: both bits = A, bit 30 only = B, bit 31 only = C).
constexpr uint32_t kVertexMask = 0x3FFFFFFFu;

// Device view of one graph.
struct DevGraph {
  int32_t n;
  int32_t m;                // arcs
  int32_t nu;               // undirected adjacency entries (2 * undirected edges)
  int32_t root_begin;       // only k-sets whose smallest vertex is in
  int32_t root_end;         //   [root_begin, root_end) are counted
  int32_t pad;
  const int32_t* row_ptr;   // n+1, directed out-CSR (sorted rows)
  const int32_t* col;       // m
  const int32_t* urow;      // n+1
  const uint32_t* ucol;     // nu, packed entries (see kVertexMask)
  const int32_t* usrc;      // nu, row vertex of each undirected entry
  const int32_t* ufwd;      // n, index within the row of the first neighbour > v
  unsigned long long* hist; // histogram this graph's subgraphs are added to
};

// Work item of the enumerator: root `root` of graph `g`, first-level branches
// [j1a, j1b) of the root's forward neighbour list; when j1b == j1a + 1 the
// second-level choices may be limited to [a2, b2) (b2 == 0xFFFF: no limit).
struct Item {
  uint32_t g;
  uint32_t root;
  uint16_t j1a, j1b;
  uint16_t a2, b2;
};
static_assert(sizeof(Item) == 16, "Item is 16 bytes");

// What a counting launch reads of a table: the slots, and for the compact
// k = 6 form (xclass != nullptr) the class of each 4-vertex prefix key and its
// word relabelling (4096 x 256 bytes).
struct TableView {
  const uint32_t* slots = nullptr;
  const uint16_t* xclass = nullptr;
  const uint8_t* xmap = nullptr;
};

// Record one CUDA error text for mt_last_error().
void set_last_error(const std::string& s);

#define MT_CUDA_TRY(expr)                                                        \
  do {                                                                           \
    cudaError_t err__ = (expr);                                                  \
    if (err__ != cudaSuccess) {                                                  \
      ::mt::set_last_error(std::string(#expr) + ": " + cudaGetErrorString(err__)); \
      return err__ == cudaErrorMemoryAllocation ? MT_ENOMEM : MT_ECUDA;          \
    }                                                                            \
  } while (0)

#define MT_TRY(expr)                \
  do {                              \
    mt_status st__ = (expr);        \
    if (st__ != MT_OK) return st__; \
  } while (0)

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ int warp_incl_scan(int x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  return x;
}

// Exclusive prefix sum of data[0..count) in place, by one thread block (any
// blockDim multiple of 32, <= 1024); returns the total to every thread.  `tmp`
// is shared scratch of 33 ints.  All threads of the block must call it.
__device__ inline long long block_exclusive_scan(int32_t* data, int count, int* tmp) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nw = blockDim.x >> 5;
  long long carry = 0;
  for (int base = 0; base < count; base += blockDim.x) {
    int i = base + tid;
    int x = i < count ? data[i] : 0;
    int inc = warp_incl_scan(x);
    if (lane == 31) tmp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      int s = lane < nw ? tmp[lane] : 0;
      int si = warp_incl_scan(s);
      if (lane < nw) tmp[lane] = si - s;
      if (lane == nw - 1) tmp[32] = si;
    }
    __syncthreads();
    if (i < count) data[i] = (int32_t)(carry + tmp[wid] + inc - x);
    carry += tmp[32];
    __syncthreads();
  }
  return carry;
}

}  // namespace mt
