// K2: enumerate every weakly connected k-vertex set once, classify it by one
// table read, add it to the histogram (Problem 1 of Sec. 1; Sec. 3.1, 3.2).
//
// Enumeration (extension scheme of ESU, the "Fanmod" method of Table 1): a set
// is produced from its smallest vertex, the root v.  The root's candidate list
// is {u in delta(v) : u > v}; choosing a candidate w appends to the remaining
// candidates the exclusive neighbours of w -- neighbours larger than v that are
// neither in the current set nor adjacent to it.  With k-1 vertices chosen,
// every remaining candidate completes one k-set.
//
// GPU mapping (one warp = one depth-first walk, lanes cooperate):
//  * per warp a "relation word" lab[u] for every vertex: bits 2p, 2p+1 hold the
//    A/B/C relation (Sec. 2) of u to the vertex at position p of the current
//    set.  Pushing w at position p scans delta(w) above the root coalesced
//    (the row-scan strategy of Sec. 3.1), ORs its relation bits into lab[u]
//    and, with one ballot, appends to the candidate stack every u with no
//    relation to the earlier positions (exclusive neighbour).  Popping clears
//    the same bits.  Words are 8, 16 or 32 bits (see LabT): the bits above the
//    first k-2 positions are slots for the (k-1)-th choices;
//  * candidate lists of all levels live in one per-warp stack: level p+1's list
//    is the unused tail of level p's list followed by the newly appended
//    exclusive neighbours, so no list is ever copied;
//  * the current level's state (cursor, ends, key prefix) lives in warp-uniform
//    registers; suspended levels wait in a small per-warp stack in shared
//    memory;
//  * choosing the (k-1)-th vertex finishes its k-sets in place, for up to GS
//    choices at once: the choices' rows, concatenated over the lanes, mark
//    each choice's slot in its neighbours' words and classify the exclusive
//    neighbours (their word is the arc code to the choice); then one pass over
//    the remaining candidates classifies every choice's leaves from the words
//    (key prefix OR word) and clears the slots again -- no per-subgraph
//    adjacency test; one match_any groups the pass's lanes for every choice
//    at once (tag: the candidate's word, which fixes its key for each choice,
//    plus the number of choices it is a leaf of), and a group of equal keys
//    shares one table read; k = 6 launches with many blocks per graph match
//    three choices at a time instead (see kWideTailBlocksPerGraph); at k = 6,
//    short candidate lists let several choices share one pass, a (choice,
//    candidate) pair per lane;
//  * MT_METHOD_CELLS stops one level earlier and counts the last two vertices
//    per pair of cells (Algorithm 1 of Sec. 3; see pair_level below);
//  * histograms: per-block shared-memory 32-bit counters for k <= 5 (13 / 199
//    / 9,364 classes), the graph's 64-bit global counters for k = 6 (a
//    one-graph count spreads its blocks over kHistCopies copies of them and
//    folds the copies afterwards), both updated with reductions that return
//    nothing (PTX red).
//
// Work items are (graph, root, first-level branch range) or, for expensive
// branches, (graph, root, branch, second-level choice range); a planner sizes
// them from per-branch cost estimates.  Hub graphs whose candidate stacks
// ((k-2) x max degree + 32 entries per warp) would leave few warps in shared
// memory keep the stacks in per-warp slices of global memory.  Blocks work
// graph by graph, warps take the items of the block's current graph from that
// graph's queue, and a warp that runs out takes halves of its block-mates'
// remaining ranges (work donation).
#include <algorithm>
#include <type_traits>

#include "count.cuh"

namespace mt {

struct Hdr {
  uint32_t head;
  uint32_t err;
  uint32_t pad0, pad1;
  double total_est;
  double pad2;
};

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kTargetItemsPerWarp = 64;
// Adds one warp may make to a shared 32-bit histogram between two flushes of
// it by exchange (enumeration path, k <= 5; see `ladd` in k_count).
constexpr int kLeafBudget = 1 << 25;
// Items a block's warps can hand to each other at once (work donation).
constexpr int kDonSlots = 32;
// Bounds of the waits of work donation: lock attempts, idle polls, and the
// idle time (ns) after which a warp gives up and reports kErrWaitLimit.
constexpr int kLockTries = 1 << 24;
constexpr int kIdlePolls = 1 << 28;
constexpr unsigned long long kIdleNs = 60ull * 1000 * 1000 * 1000;  // default; mt_set_wait_limit

// Idle-wait limit (ns) given to the launches enqueued from now on.
static unsigned long long g_idle_ns = kIdleNs;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr int kMaxWarpsPerBlock = 32;
// k = 6 launches with at most this many blocks per histogram (copy) group a
// tail batch's lanes with one match for all of a group's choices; launches over
// fewer graphs match three choices at a time.  A block works on one graph at a time, so with
// few graphs many blocks add into the same global histogram; there the single
// match's finer groups (more leaders, each adding for every choice) sent 29%
// more reduction sectors to L2 and ran slower.  Measured on 152 blocks, k = 6
// batches of 2 .. 33 graphs run 22% .. 1.5% faster with three choices per
// match, 49 alike, 65 3% slower.
constexpr int kWideTailBlocksPerGraph = 3;
// A one-graph k = 6 count spreads its blocks over this many copies of the
// graph's histogram (block b adds into copy b mod kHistCopies), folded into the
// caller's histogram by k_fold_copies: ~19 blocks per copy on 152 SMs instead
// of all blocks on the same counters.  Measured on the k = 6 workload graph and
// three of its nulls (n = 800, m = 3,200): 16.0-16.4 ms per count without
// copies, 5.6-5.8 ms with 8, histograms identical.
constexpr int kHistCopies = 8;
// Per-warp stack of suspended DFS levels: (cursor, choice end, tail end, key, vertex).
constexpr int kLevelBytes = 128;

__device__ __forceinline__ float choose_f(int x, int r) {
  if (x < r) return 0.f;
  float c = 1.f;
  for (int i = 0; i < r; ++i) c = c * (float)(x - i) / (float)(i + 1);
  return c;
}

// Estimated work of a first-level branch whose second-level candidate list has
// x1 entries: about C(x1, k-2) sets of k-1 vertices, each touching its
// candidates once.
template <int K>
__device__ __forceinline__ float branch_cost(int x1) {
  return 1.f + (float)x1 + choose_f(x1, K - 2) * (K >= 4 ? 2.f : 1.f);
}

// Offset of position p's 2p bits in an extension-order key of k vertices:
// later positions sit lower, so the k-sets below one (k-2)-set differ only in
// the low bits of their keys and read nearby table slots.
__host__ __device__ constexpr int key_off(int k, int p) { return k * (k - 1) - p * (p + 1); }

// Histogram reductions without a returned value (PTX red): the issuing warp
// never waits for them.
__device__ __forceinline__ void red_add_global(unsigned long long* p, unsigned long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "l"(v)
               : "memory");
}
__device__ __forceinline__ void red_add_shared(int* p, int v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v)
               : "memory");
}

// Whether vertex x is in sorted packed entries [lo, hi).
__device__ __forceinline__ bool contains(const uint32_t* __restrict__ ucol, int lo, int hi, int x) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int y = (int)(__ldg(&ucol[mid]) & kVertexMask);
    if (y == x) return true;
    if (y < x) lo = mid + 1; else hi = mid;
  }
  return false;
}

// ------------------------------------------------------------------ planner

template <int K>
__global__ void __launch_bounds__(256) k_plan_est(const DevGraph* __restrict__ graphs,
                                                  int64_t stride, float* est, int32_t* x1s,
                                                  Hdr* hdr, int root_begin, int root_end) {
  __shared__ float red[8];
  const int g = blockIdx.y;
  const DevGraph G = graphs[g];
  float local = 0.f;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < G.nu; e += gridDim.x * blockDim.x) {
    const int v = G.usrc[e];
    const int u = (int)(G.ucol[e] & kVertexMask);
    float c = 0.f;
    int x1 = 0;
    if (u > v && v >= root_begin && v < root_end && v >= G.root_begin && v < G.root_end) {
      const int re = G.urow[v + 1];
      const int f = G.urow[v] + G.ufwd[v];
      const int j1 = e - f;
      int ex = 0;
      for (int i = G.urow[u]; i < G.urow[u + 1]; ++i) {
        const int x = (int)(G.ucol[i] & kVertexMask);
        if (x > v && !contains(G.ucol, f, re, x)) ++ex;
      }
      x1 = (re - f) - j1 - 1 + ex;
      c = branch_cost<K>(x1);
    }
    est[g * stride + e] = c;
    x1s[g * stride + e] = x1;
    local += c;
  }
  for (int d = 16; d; d >>= 1) local += __shfl_xor_sync(kFull, local, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    if (s > 0.f) atomicAdd(&hdr->total_est, (double)s);
  }
}

// Walk one root's forward branches and cut them into items (count or write).
// One warp per root: the lanes load 32 entries at a time, every lane walks them
// in order with the same (warp-uniform) packing state, and the many level-2
// ranges of a split branch are written by all lanes at once, so a hub root's
// thousands of items cost a few stores per lane instead of a serial loop.
template <int K, bool WRITE>
__global__ void __launch_bounds__(256) k_plan_items(const DevGraph* __restrict__ graphs,
                                                    int64_t stride, const float* est,
                                                    const int32_t* x1s, int nmax, int32_t* cnt,
                                                    Item* items, uint64_t items_max, Hdr* hdr,
                                                    double split_cost, double split_scale,
                                                    double target_items, double items_factor,
                                                    int root_begin, int root_end) {
  const int g = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int v = blockIdx.x * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
  if (!WRITE && g == 0 && v == 0 && lane == 0) cnt[(int64_t)gridDim.y * nmax] = 0;
  if (v >= nmax) return;
  const int64_t slot = (int64_t)g * nmax + v;
  const DevGraph G = graphs[g];
  if (v >= G.n || v < root_begin || v >= root_end || v < G.root_begin || v >= G.root_end) {
    if (!WRITE && lane == 0) cnt[slot] = 0;
    return;
  }
  // root-split threshold: explicit, or the automatic one scaled; never so small
  // that the items exceed their budget
  const double t_auto = hdr->total_est / target_items;
  double T = split_cost > 0.0 ? split_cost : t_auto * split_scale;
  const double t_min = hdr->total_est / (items_factor * target_items);
  if (T < t_min) T = t_min;
  if (T < 1.0) T = 1.0;
  const float Tf = (float)T;
  const int re = G.urow[v + 1];
  const int f = G.urow[v] + G.ufwd[v];
  const int dplus = re - f;
  int64_t pos = WRITE ? cnt[slot] : 0;
  int count = 0;
  auto put = [&](int64_t at, int j1a, int j1b, int a2, int b2) {
    if ((uint64_t)at < items_max) {
      Item it;
      it.g = (uint32_t)g;
      it.root = (uint32_t)v;
      it.j1a = (uint16_t)j1a;
      it.j1b = (uint16_t)j1b;
      it.a2 = (uint16_t)a2;
      it.b2 = (uint16_t)b2;
      items[at] = it;
    } else {
      atomicOr(&hdr->err, kErrStackOverflow);
    }
  };
  auto emit = [&](int j1a, int j1b) {  // one whole-range item, written by lane 0
    if (WRITE && lane == 0) put(pos, j1a, j1b, 0, 0xFFFF);
    ++pos;
    ++count;
  };
  float acc = 0.f;
  int start = 0;
  for (int base = 0; base < dplus; base += 32) {
    float c_l = 0.f;
    int x_l = 0;
    if (base + lane < dplus) {
      const int64_t e = (int64_t)g * stride + f + base + lane;
      c_l = est[e];
      x_l = x1s[e];
    }
    const int n = min(32, dplus - base);
    for (int i = 0; i < n; ++i) {
      const float c = __shfl_sync(kFull, c_l, i);
      const int x = __shfl_sync(kFull, x_l, i);
      const int j = base + i;
      if (K >= 4 && c > 2.f * Tf && x >= 2) {
        if (j > start) emit(start, j);
        int nch = (int)ceilf(c / Tf);
        if (nch > x) nch = x;
        const int r2 = (x + nch - 1) / nch;
        const int ns = (x + r2 - 1) / r2;
        if (WRITE)
          for (int t = lane; t < ns; t += 32) put(pos + t, j, j + 1, t * r2, min(t * r2 + r2, x));
        pos += ns;
        count += ns;
        start = j + 1;
        acc = 0.f;
      } else {
        acc += c;
        if (acc >= Tf) {
          emit(start, j + 1);
          start = j + 1;
          acc = 0.f;
        }
      }
    }
  }
  if (start < dplus) emit(start, dplus);
  if (!WRITE && lane == 0) cnt[slot] = count;
}

__global__ void __launch_bounds__(1024) k_scan_counts(int32_t* data, int count) {
  __shared__ int tmp[33];
  block_exclusive_scan(data, count, tmp);
}

// ------------------------------------------------------------------ enumerator

// Relation words: 2 bits per earlier position.  The first k-2 positions take
// 2(k-2) bits; the slots above them let several (k-1)-th choices be marked at
// once: 8 bits for k <= 4 (3 and 2 slots), 16 bits for k = 5 (5 slots), 32 bits
// for k = 6 (8 slots used).  The cell method needs only two flag bits above
// them: 8 bits up to k = 5, 16 bits for k = 6.
template <int K, bool CB>
using LabT = typename std::conditional<
    (K <= 4 || (CB && K <= 5)), uint8_t,
    typename std::conditional<(K == 5 || CB), uint16_t, uint32_t>::type>::type;

template <typename LT>
struct WarpCtx {
  const int32_t* urow;   // shared-memory copy of the graph or global memory
  const uint32_t* ucol;
  LT* lab;
  uint16_t* buf;
  int cap;
  int root;
  int lane;
  uint32_t* err;
};

// First index in sorted packed entries [lo, hi) whose vertex is > x.
__device__ __forceinline__ int first_above_p(const uint32_t* ucol, int lo, int hi, int x) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((int)(ucol[mid] & kVertexMask) > x) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Push x at position p: OR its relation bits into lab[] of its neighbours above
// the root and append the exclusive ones (no relation to positions 0..p-1, the
// bits in `low`; bits above it may be stale) at stack index e.  Returns the
// new end of the candidate list.
template <typename LT>
__device__ __forceinline__ int push_vertex(const WarpCtx<LT>& w, int x, int p, int e,
                                           uint32_t low) {
  const int rs = w.urow[x], re = w.urow[x + 1];
  const int start = (re - rs > 32) ? first_above_p(w.ucol, rs, re, w.root) : rs;
  const unsigned lt = (1u << w.lane) - 1u;
  int cnt = 0;
  for (int b = start; b < re; b += 32) {
    const int i = b + w.lane;
    bool ex = false;
    int u = 0;
    if (i < re) {
      const uint32_t ent = w.ucol[i];
      u = (int)(ent & kVertexMask);
      if (u > w.root) {
        const LT old = w.lab[u];
        w.lab[u] = (LT)(old | ((ent >> 30) << (2 * p)));
        ex = ((uint32_t)old & low) == 0;
      }
    }
    const unsigned bal = __ballot_sync(kFull, ex);
    if (ex) {
      const int pos = e + cnt + __popc(bal & lt);
      if (pos < w.cap) w.buf[pos] = (uint16_t)u;
      else atomicOr(w.err, kErrStackOverflow);
    }
    cnt += __popc(bal);
  }
  __syncwarp();
  const int ne = e + cnt;
  return ne < w.cap ? ne : w.cap;
}

// Pop the vertex x at position p: clear its relation bits again.
template <typename LT>
__device__ __forceinline__ void pop_vertex(const WarpCtx<LT>& w, int x, int p) {
  const int rs = w.urow[x], re = w.urow[x + 1];
  const int start = (re - rs > 32) ? first_above_p(w.ucol, rs, re, w.root) : rs;
  const LT clear = (LT)~(3u << (2 * p));
  for (int b = start; b < re; b += 32) {
    const int i = b + w.lane;
    if (i < re) {
      const int u = (int)(w.ucol[i] & kVertexMask);
      if (u > w.root) w.lab[u] &= clear;
    }
  }
  __syncwarp();
}

// hist[i] += the copies' counts of class i (a one-graph k = 6 count; see
// kHistCopies).  Counts are two's-complement 64-bit sums, so the cell method's
// negative corrections fold correctly.
__global__ void __launch_bounds__(256) k_fold_copies(unsigned long long* __restrict__ hist,
                                                     const unsigned long long* __restrict__ copies,
                                                     int ncopies, uint32_t C, uint32_t stride) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
    unsigned long long sum = 0;
    for (int c = 0; c < ncopies; ++c) sum += copies[(size_t)c * stride + i];
    if (sum) hist[i] += sum;
  }
}

struct CountArgs {
  const DevGraph* graphs;
  const Item* items;
  const int32_t* item_off;   // scanned item counts: graph g owns [item_off[g*nmax], item_off[(g+1)*nmax])
  uint32_t* qhead;           // per-graph queue heads
  Hdr* hdr;
  const uint32_t* table;
  const uint16_t* xclass;    // compact k = 6 table: prefix key -> class of the first 4 vertices
  const uint8_t* xmap;       //   and its word relabelling (256 bytes per prefix key)
  void* lab_global;
  void* stack_global;        // per-warp candidate stacks when they live in global memory
  unsigned long long* hist_copies;  // copies 1 .. copies-1 of a one-graph k = 6 histogram
  int copies;                // 1 = every block adds into the graph's own histogram
  uint32_t copy_stride;      // elements between two copies
  int G, nmax, nu_cap, cap;
  uint32_t classes;
  int graph_bytes, hist_bytes, lab_bytes, buf_bytes, cell_bytes, map_bytes;
  unsigned long long idle_ns;  // a warp waiting for donated work gives up after this
};

// Cells of the last two positions (combinatorial counting): a relation word to
// the k-2 chosen vertices has 2(k-2) bits.
template <int K>
constexpr int kCells = 1 << (2 * (K - 2));

// Persistent enumerator.  A thread block works on one graph at a time: its
// warps take that graph's items from the graph's queue.  A warp that finds the
// queue empty waits for work donated by the block's other warps: a busy warp
// that sees an idle one hands over half of its remaining first- or
// second-level choices as a new item.  When every warp is idle and nothing is
// left to take, the block flushes its shared histogram, picks the next graph
// that still has items and (GC) copies that graph's CSR into shared memory.
// SG: the candidate stacks live in per-warp slices of global memory (graphs
// with hubs so large that shared-memory stacks would leave few warps).
template <int K, bool GC, bool LS, bool COMB, bool SG = false>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32, 1) k_count(CountArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_cur_g;
  __shared__ int s_idle, s_ndon, s_lock;  // work donation (see above)
  __shared__ uint32_t s_don[kDonSlots * 4];  // donated items, 4 words each
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  const unsigned lanes_below = (1u << lane) - 1u;
  int since = 0;  // this warp's enumeration adds since its last flush
  bool bad_id = false;  // k = 6: a table read gave an id out of range
  unsigned char* sp = smem;
  int32_t* s_urow = (int32_t*)sp;
  uint32_t* s_ucol = (uint32_t*)(sp + (GC ? ((a.nmax + 1) * 4 + 15) / 16 * 16 : 0));
  sp += a.graph_bytes;
  int32_t* s_hist = (int32_t*)sp;
  sp += a.hist_bytes;
  const int sbuf = SG ? 0 : a.buf_bytes;  // stack bytes in this warp's shared slice
  unsigned char* mine =
      sp + (size_t)wid * ((LS ? a.lab_bytes : 0) + sbuf + (COMB ? a.cell_bytes : 0) +
                          kLevelBytes + a.map_bytes);
  int* lvs = (int*)(mine + (LS ? a.lab_bytes : 0) + sbuf + (COMB ? a.cell_bytes : 0));
  // compact k = 6 table: the current 4-vertex prefix's word relabelling
  uint8_t* xmw = (uint8_t*)lvs + kLevelBytes;
  const bool cpt = K == 6 && !COMB && a.xclass != nullptr;
  const bool wide_tail = K <= 5 || (int)gridDim.x <= kWideTailBlocksPerGraph * a.G * a.copies;
  using LT = LabT<K, COMB>;
  // each warp's relation words start on a 16-byte boundary (lab_bytes is a
  // multiple of 16), so 32-bit atomics on them are aligned
  LT* lab = LS ? (LT*)mine
               : (LT*)((char*)a.lab_global + ((size_t)blockIdx.x * nwarps + wid) * a.lab_bytes);
  uint16_t* buf =
      SG ? (uint16_t*)((char*)a.stack_global + ((size_t)blockIdx.x * nwarps + wid) * a.buf_bytes)
         : (uint16_t*)(mine + (LS ? a.lab_bytes : 0));
  // combinatorial mode: per-cell counts (choices in the low, tail in the high
  // 16 bits), the list of non-empty cells, and its length
  uint32_t* ct = (uint32_t*)(mine + (LS ? a.lab_bytes : 0) + sbuf);
  uint16_t* cl = (uint16_t*)(ct + kCells<K>);
  int* ncell = (int*)(mine + (LS ? a.lab_bytes : 0) + sbuf + a.cell_bytes - 16);
  uint32_t* xc = (uint32_t*)(mine + (LS ? a.lab_bytes : 0) + sbuf + a.cell_bytes - 16 - 384);
  const uint32_t C = a.classes;

  if (LS)
    for (int i = lane; i < a.nmax; i += 32) lab[i] = 0;
  if (COMB) {
    for (int i = lane; i < kCells<K>; i += 32) ct[i] = 0;
    for (int i = lane; i < 96; i += 32) xc[i] = 0;
    if (lane == 0) *ncell = 0;
  }
  if (K <= 5)
    for (int i = tid; i <= (int)C; i += blockDim.x) s_hist[i] = 0;  // C: catch slot
  if (tid == 0) {
    s_cur_g = (int)(((int64_t)blockIdx.x * a.G) / gridDim.x);
    s_idle = 0;
    s_ndon = 0;
    s_lock = 0;
  }
  __syncthreads();

  // Block-local lock of the donation slots (lane 0 of a warp only).
  auto block_lock = [&]() -> bool {
    for (int i = 0; i < kLockTries; ++i) {
      if (atomicCAS(&s_lock, 0, 1) == 0) {
        __threadfence_block();
        return true;
      }
      __nanosleep(32);
    }
    atomicOr(&a.hdr->err, kErrWaitLimit);
    return false;
  };
  auto block_unlock = [&]() {
    __threadfence_block();
    atomicExch(&s_lock, 0);
  };
  volatile int* v_idle = &s_idle;
  volatile int* v_ndon = &s_ndon;
  volatile uint32_t* v_don = s_don;

  WarpCtx<LT> w;
  w.lab = lab;
  w.buf = buf;
  w.cap = a.cap;
  w.lane = lane;
  w.err = &a.hdr->err;

  int g = s_cur_g;
  while (g >= 0) {
    const DevGraph* Gp = a.graphs + g;
    if (GC) {
      const int n = Gp->n, nu = Gp->nu;
      for (int i = tid; i <= n; i += blockDim.x) s_urow[i] = Gp->urow[i];
      for (int i = tid; i < nu; i += blockDim.x) s_ucol[i] = Gp->ucol[i];
      w.urow = s_urow;
      w.ucol = s_ucol;
    } else {
      w.urow = Gp->urow;
      w.ucol = Gp->ucol;
    }
    __syncthreads();
    unsigned long long* ghist = Gp->hist;
    if (K == 6 && a.copies > 1) {  // one graph: this block's copy of its histogram
      const int cp = (int)(blockIdx.x % (unsigned)a.copies);
      if (cp) ghist = a.hist_copies + (size_t)(cp - 1) * a.copy_stride;
    }
    const int32_t* ufwd = Gp->ufwd;
    const int ib = a.item_off[(int64_t)g * a.nmax];
    const int ie = a.item_off[(int64_t)(g + 1) * a.nmax];

    // Add `delta` (may be negative in the combinatorial corrections) to class
    // `id`.  Shared 32-bit counters spill +-2^29 to the graph's 64-bit counter
    // (two's complement), large deltas go there directly, so no counter wraps.
    auto hadd = [&](uint32_t id, long long delta) {
      if (id >= C) {
        atomicOr(w.err, kErrStackOverflow);
        return;
      }
      if (K <= 5 && delta < (1ll << 20) && delta > -(1ll << 20)) {
        const int d = (int)delta;
        const int old = atomicAdd(&s_hist[id], d);
        const long long now = (long long)old + d;
        if (old < (1 << 29) && now >= (1 << 29)) {
          atomicSub(&s_hist[id], 1 << 29);
          red_add_global(&ghist[id], 1ull << 29);
        } else if (old > -(1 << 29) && now <= -(1 << 29)) {
          atomicAdd(&s_hist[id], 1 << 29);
          red_add_global(&ghist[id], (unsigned long long)(-(1ll << 29)));
        }
      } else {
        red_add_global(&ghist[id], (unsigned long long)delta);
      }
    };

    // Positive adds of the enumeration path.  For k <= 5 the shared 32-bit
    // counters take them without returning the old value; each warp counts
    // what it added since it last flushed and, past kLeafBudget, moves the
    // whole shared histogram to the graph's 64-bit counters by exchange
    // (adds of other warps stay in the counters).  A counter then never holds
    // more than warps x (kLeafBudget + one choice's adds) < 2^31.
    // (An id out of range, which a valid table never holds, lands in the
    // shared catch slot C, checked at the flush; for k = 6 it adds nothing and
    // is recorded in `bad_id`, reported when the thread exits.  Neither form
    // branches on the table read, so the reads of several slots overlap.)
    auto ladd = [&](uint32_t id, int d) {
      if (K <= 5) {
        red_add_shared(&s_hist[min(id, C)], d);
      } else {
        const bool ok = id < C;
        bad_id |= !ok;
        red_add_global(&ghist[ok ? id : 0u], ok ? (unsigned long long)d : 0ull);
      }
    };
    auto leaf_budget = [&](int adds) {
      if (K <= 5) {
        if (since >= kLeafBudget) {
          for (int i = lane; i < (int)C; i += 32) {
            const int x = atomicExch(&s_hist[i], 0);
            if (x) atomicAdd(&ghist[i], (unsigned long long)(long long)x);
          }
          since = 0;
        }
        since += adds;
      }
    };

    // Combinatorial counting of the last two positions (Algorithm 1 of Sec. 3
    // on the enumerator's (k-2)-set X with candidate list E = buf[c, e) whose
    // choices are buf[c, ce)): the k-sets below X are the pairs {y, z}, y a
    // choice and z after it in E, plus {y, u} with u an exclusive neighbour of
    // y.  Without an arc between y and z the class depends only on the cells
    // (relation words to X) of y and z, so those pairs are counted per cell
    // pair; arcs inside E are corrected one by one; {y, u} depends only on y's
    // cell and the arc code between y and u.
    auto pair_level = [&](int c, int ce, int e, uint32_t P) {
      constexpr int NB = 2 * (K - 2);
      constexpr uint32_t LM = (1u << NB) - 1u;
      constexpr uint32_t INC = 1u << NB, INT = 2u << NB;
      constexpr int OFF2 = key_off(K, K - 2), OFF1 = key_off(K, K - 1);
      // 1. cells of the choices and of the tail; flag E's members
      for (int b = c; b < e; b += 32) {
        const int i = b + lane;
        const bool v = i < e;
        uint32_t lam = 0, tag = 0xFFFFFFFFu;
        bool inc = false;
        if (v) {
          const int u = buf[i];
          const uint32_t l0 = lab[u];
          lam = l0 & LM;
          inc = i < ce;
          lab[u] = (LT)(l0 | (inc ? INC : INT));
          tag = lam | (inc ? 0x10000u : 0u);
        }
        const unsigned peers = __match_any_sync(kFull, tag);
        if (v && lane == __ffs(peers) - 1) {
          const uint32_t old = atomicAdd(&ct[lam], (uint32_t)__popc(peers) << (inc ? 0 : 16));
          if (old == 0) cl[atomicAdd(ncell, 1)] = (uint16_t)lam;
        }
      }
      __syncwarp();
      const int r = *ncell;
      // 2. pairs without an arc, per cell pair
      for (int ia = 0; ia < r; ++ia) {
        const uint32_t la = cl[ia];
        const uint32_t pa = ct[la];
        const long long ca = pa & 0xFFFFu, ta = pa >> 16;
        for (int ib = ia + lane; ib < r; ib += 32) {
          const uint32_t lb = cl[ib];
          const uint32_t pb = ct[lb];
          const long long cb = pb & 0xFFFFu, tb = pb >> 16;
          const long long cnt = ia == ib ? ca * (ca - 1) / 2 + ca * ta : ca * cb + ca * tb + cb * ta;
          if (cnt) hadd(__ldg(&a.table[P | (la << OFF2) | (lb << OFF1)]), cnt);
        }
      }
      // 3. the choices' rows, 32 choices at a time with their rows (entries above
      //    the root) concatenated over the lanes: arcs inside E are corrected,
      //    exclusive neighbours are counted per (choice, arc code)
      for (int cb = c; cb < ce; cb += 32) {
        const int i = cb + lane;
        const bool vy = i < ce;
        int y = 0, rs = 0, len = 0;
        uint32_t ly = 0;
        if (vy) {
          y = buf[i];
          const int r0 = w.urow[y], r1 = w.urow[y + 1];
          rs = first_above_p(w.ucol, r0, r1, w.root);
          len = r1 - rs;
          ly = lab[y] & LM;
        }
        const int incl = warp_incl_scan(len);
        const int pre = incl - len;
        const int total = __shfl_sync(kFull, incl, 31);
        for (int q0 = 0; q0 < total; q0 += 32) {
          const int q = q0 + lane;
          // the lane's choice: the largest s with pre[s] <= q
          int sidx = 0;
          for (int step = 16; step; step >>= 1) {
            const int cand = sidx + step;
            const int pc = __shfl_sync(kFull, pre, cand & 31);
            if (cand <= 31 && pc <= q) sidx = cand;
          }
          const int ys = __shfl_sync(kFull, y, sidx);
          const int rss = __shfl_sync(kFull, rs, sidx);
          const int ps = __shfl_sync(kFull, pre, sidx);
          const uint32_t lys = __shfl_sync(kFull, ly, sidx);
          bool ex = false;
          uint32_t code = 0;
          if (q < total) {
            const uint32_t ent = w.ucol[rss + (q - ps)];
            const int u = (int)(ent & kVertexMask);
            code = ent >> 30;
            const uint32_t lu = lab[u];
            ex = lu == 0;
            if ((lu & INT) || ((lu & INC) && u > ys)) {
              const uint32_t bs = P | (lys << OFF2);
              const uint32_t cu = lu & LM;
              hadd(__ldg(&a.table[bs | ((cu | (code << NB)) << OFF1)]), 1);
              hadd(__ldg(&a.table[bs | (cu << OFF1)]), -1);
            }
          }
          const uint32_t tag = ex ? (uint32_t)(sidx * 4) + code : 0xFFFFFFFFu;
          const unsigned peers = __match_any_sync(kFull, tag);
          if (ex && lane == __ffs(peers) - 1) atomicAdd(&xc[sidx * 3 + code - 1], (uint32_t)__popc(peers));
        }
        __syncwarp();
        if (vy) {
          const uint32_t bs = P | (ly << OFF2);
          for (int cd = 1; cd <= 3; ++cd) {
            const uint32_t cnt = xc[lane * 3 + cd - 1];
            if (cnt) {
              hadd(__ldg(&a.table[bs | (((uint32_t)cd << NB) << OFF1)]), cnt);
              xc[lane * 3 + cd - 1] = 0;
            }
          }
        }
        __syncwarp();
      }
      // 4. clear flags and cells
      for (int b = c; b < e; b += 32) {
        const int i = b + lane;
        if (i < e) lab[buf[i]] &= (LT)~(INC | INT);
      }
      for (int ia = lane; ia < r; ia += 32) ct[cl[ia]] = 0;
      __syncwarp();
      if (lane == 0) *ncell = 0;
      __syncwarp();
    };

    // Lane 0: wait, idle, for a donated item (1) or for the whole block to be
    // idle with nothing left to take (0).
    auto take_donation = [&](uint4& raw) -> int {
      if (!block_lock()) return 0;
      *v_idle = *v_idle + 1;
      block_unlock();
      const unsigned long long t0 = global_ns();
      for (int poll = 0; poll < kIdlePolls; ++poll) {
        if (*v_ndon > 0 || *v_idle == nwarps) {
          if (!block_lock()) return 0;
          int r = -1;
          const int nd = *v_ndon;
          if (nd > 0) {
            raw.x = v_don[4 * (nd - 1)];
            raw.y = v_don[4 * (nd - 1) + 1];
            raw.z = v_don[4 * (nd - 1) + 2];
            raw.w = v_don[4 * (nd - 1) + 3];
            *v_ndon = nd - 1;
            *v_idle = *v_idle - 1;
            r = 1;
          } else if (*v_idle == nwarps) {
            r = 0;
          }
          block_unlock();
          if (r >= 0) return r;
        }
        if (global_ns() - t0 > a.idle_ns) break;
        __nanosleep(256);
      }
      atomicOr(&a.hdr->err, kErrWaitLimit);
      return 0;
    };
    // The warp's next item: the graph's queue, then donated items.
    auto next_item = [&](Item& out) -> bool {
      uint32_t idx = 0;
      if (lane == 0) idx = atomicAdd(&a.qhead[g], 1u);
      idx = __shfl_sync(kFull, idx, 0);
      const int64_t pos = (int64_t)ib + idx;
      if (pos < ie) {
        out = a.items[pos];
        return true;
      }
      uint4 raw = make_uint4(0, 0, 0, 0);
      int got = 0;
      if (lane == 0) got = take_donation(raw);
      got = __shfl_sync(kFull, got, 0);
      if (!got) return false;
      raw.x = __shfl_sync(kFull, raw.x, 0);
      raw.y = __shfl_sync(kFull, raw.y, 0);
      raw.z = __shfl_sync(kFull, raw.z, 0);
      raw.w = __shfl_sync(kFull, raw.w, 0);
      memcpy(&out, &raw, sizeof(Item));
      return true;
    };

    while (true) {
      Item it;
      if (!next_item(it)) break;
      const int v = (int)it.root;
      w.root = v;
      const int re = w.urow[v + 1];
      const int f = w.urow[v] + __ldg(&ufwd[v]);
      const int dplus = re - f;
      const int j1a = it.j1a, j1b = it.j1b;
      // push the root at position 0: every forward neighbour gets its relation
      // bits; candidates j1a.. go to the stack.
      for (int b = f; b < re; b += 32) {
        const int i = b + lane;
        if (i < re) {
          const uint32_t ent = w.ucol[i];
          const int u = (int)(ent & kVertexMask);
          lab[u] |= (LT)(ent >> 30);
          const int q = i - f - j1a;
          if (q >= 0) {
            if (q < w.cap) buf[q] = (uint16_t)u;
            else atomicOr(w.err, kErrStackOverflow);
          }
        }
      }
      __syncwarp();
      // the current level's state lives in (warp-uniform) registers; the
      // levels above it wait in the per-warp stack `lvs`
      int cur_e = min(dplus - j1a, w.cap);
      int cur_c = 0, cur_ce = min(j1b - j1a, cur_e);
      uint32_t cur_key = 0;
      const bool has2 = it.b2 != 0xFFFF;
      // The enumerator's slot codes (bits of positions k-2 and up) are not
      // cleared by row scans: the tail pass writes each candidate back
      // without them, and a candidate list is cleaned once when its level
      // (k-2 positions chosen) is entered; every other reader masks them.
      bool fresh = true;
      uint32_t xpre = 0;  // compact table: class of the current 4-vertex prefix, in place
      int L = 1;
      auto pop_level = [&]() {
        L -= 1;
        const int* sv = lvs + 5 * L;
        cur_c = sv[0];
        cur_ce = sv[1];
        cur_e = sv[2];
        cur_key = (uint32_t)sv[3];
        pop_vertex(w, sv[4], L);
      };
      while (true) {
        const int c = cur_c, ce = cur_ce, e = cur_e;
        const uint32_t key = cur_key;
        if (COMB && L == K - 2) {
          pair_level(c, ce, e, key);
          if (L == 1) break;
          pop_level();
          continue;
        }
        if (!COMB && L == K - 2) {
          // Choosing the (k-1)-th vertex finishes its k-sets in place, for up
          // to GS consecutive choices at once (as many as the relation word
          // has free 2-bit slots, at most 8: 3, 2, 5, 8 for k = 3..6): choice
          // g marks its row into slot g above the first k-2 positions' bits,
          // so one pass over the shared candidate tail classifies every
          // choice's leaves.
          if (c >= ce) {
            if (L == 1) break;
            pop_level();
            continue;
          }
          constexpr int NB = 2 * (K - 2);
          constexpr uint32_t LM = (1u << NB) - 1u;
          constexpr int OFF1 = key_off(K, K - 1);
          constexpr int OFF2 = key_off(K, K - 2);
          if (fresh) {
            // a new candidate list: clear slot codes left by earlier rows
            for (int b = c; b < e; b += 32) {
              const int i = b + lane;
              if (i < e) {
                const int u = buf[i];
                lab[u] = (LT)((uint32_t)lab[u] & LM);
              }
            }
            __syncwarp();
            fresh = false;
            if (cpt) {
              // class of the first four vertices and the relabelling of words
              // to their canonical order (positions 1..3 sit in key bits 18..29)
              const uint32_t xk = key >> 18;
              ((uint2*)xmw)[lane] = __ldg((const uint2*)(a.xmap + (size_t)xk * 256) + lane);
              uint32_t c4 = __ldg(&a.xclass[xk]);
              if (c4 >= 199u) {  // a disconnected prefix, which the enumeration never forms
                atomicOr(w.err, kErrStackOverflow);
                c4 = 0;
              }
              xpre = c4 << 18;
              __syncwarp();
            }
          }
          // slots left in the relation word above the first k-2 positions
          constexpr int GS = (8 * (int)sizeof(LT) - NB) / 2 < 8 ? (8 * (int)sizeof(LT) - NB) / 2 : 8;
          static_assert(COMB || GS >= 2, "at least two slots per relation word");
          const int ng = min(GS, ce - c);
          cur_c = c + ng;
          // lane g < ng: choice g's key prefix and its row above the root
          uint32_t Pg = 0;
          int rs_g = 0, len_g = 0;
          if (lane < ng) {
            const int y = buf[c + lane];
            Pg = cpt ? xpre | ((uint32_t)xmw[(uint32_t)lab[y] & LM] << OFF2)
                     : key | ((uint32_t)(lab[y] & LM) << OFF2);
            const int r0 = w.urow[y], r1 = w.urow[y + 1];
            rs_g = (r1 - r0 > 32) ? first_above_p(w.ucol, r0, r1, w.root) : r0;
            len_g = r1 - rs_g;
          }
          // qs[g] = where choice g's row starts in the concatenation
          int qs[GS + 1];
          qs[0] = 0;
#pragma unroll
          for (int gg = 0; gg < GS; ++gg) qs[gg + 1] = qs[gg] + __shfl_sync(kFull, len_g, gg);
          const int tot = qs[GS];
          leaf_budget(ng * (e - c - 1) + tot);
          // (a) the group's rows, concatenated over the lanes: choice g sets
          //     slot g of its neighbours (a 32-bit atomic OR on the word that
          //     holds the relation word, as two choices may share a
          //     neighbour); an exclusive neighbour u (no relation to the first
          //     k-2 vertices) completes a k-set keyed by the choice's prefix
          //     and the arc code between the choice and u, counted per
          //     (choice, code) group of the pass
          {
            constexpr int PER = 4 / (int)sizeof(LT);  // relation words per 32-bit word
            uint32_t* lab32 = (uint32_t*)lab;
            for (int b = 0; b < tot; b += 32) {
              const int q = b + lane;
              int gg = 0, off = 0;
#pragma unroll
              for (int t = 1; t < GS; ++t)
                if (q >= qs[t]) {
                  gg = t;
                  off = qs[t];
                }
              const int rs = __shfl_sync(kFull, rs_g, gg);
              const uint32_t pg = __shfl_sync(kFull, Pg, gg);
              bool ex = false;
              uint32_t code = 0;
              if (q < tot) {
                const uint32_t ent = w.ucol[rs + (q - off)];
                const int u = (int)(ent & kVertexMask);
                code = ent >> 30;
                if (u > w.root) {
                  const uint32_t old = (uint32_t)lab[u];
                  atomicOr(&lab32[u / PER],
                           (code << (NB + 2 * gg)) << (8 * (int)sizeof(LT) * (u % PER)));
                  ex = (old & LM) == 0;
                }
              }
              const unsigned peers = __match_any_sync(kFull, ex ? (uint32_t)(gg * 4) + code : 0xFFFFFFFFu);  // (choice, code)
              if (ex && !(peers & lanes_below))
                ladd(__ldg(&a.table[pg | ((code << NB) << OFF1)]), __popc(peers));
            }
            __syncwarp();
          }
          // (b) the candidates after the group's first choice; those after
          //     choice g are its leaves, keyed by their word to the first k-2
          //     vertices plus slot g; equal keys of a batch share a table read
          const int lc = e - c - 1;  // candidates after the group's first choice
          if (K == 6 && lc <= 16 && ng > 1) {
            // A short list (common at k = 6, where lists average 20
            // candidates; measured no better at k = 5): P choices per pass,
            // 32 / P lanes each, every lane one (choice, candidate) pair; the
            // match groups equal full keys, so pairs of different choices with
            // the same key share a read.
            const int P = lc <= 4 ? 8 : (lc <= 8 ? 4 : 2);
            const int lw = P == 8 ? 2 : (P == 4 ? 3 : 4);  // log2 of the lanes per choice
            const int h = lane >> lw, idx = lane & ((1 << lw) - 1);
            const bool v0 = idx < lc;
            const int u0 = v0 ? buf[c + 1 + idx] : 0;
            const uint32_t lt = v0 ? (uint32_t)lab[u0] : 0u;
            if (v0 && h == 0) lab[u0] = (LT)(lt & LM);
            const uint32_t lb = cpt ? (uint32_t)xmw[lt & LM] : (lt & LM);
            for (int p0 = 0; p0 < ng; p0 += P) {
              const int gg = p0 + h;
              const uint32_t pg = __shfl_sync(kFull, Pg, gg & 31);
              const bool vg = v0 && gg < ng && idx + 1 > gg;
              const uint32_t key = pg | ((lb | ((lt >> (2 * gg)) & (3u << NB))) << OFF1);
              const unsigned peers = __match_any_sync(kFull, vg ? key : 0xFFFFFFFFu);
              if (vg && !(peers & lanes_below)) ladd(__ldg(&a.table[key]), __popc(peers));
            }
            __syncwarp();
            continue;
          }
          uint32_t pgs[GS];
#pragma unroll
          for (int gg = 0; gg < GS; ++gg) pgs[gg] = __shfl_sync(kFull, Pg, gg);
          for (int b = c + 1; b < e; b += 32) {
            const int i0 = b + lane;
            const bool v0 = i0 < e;
            const int u0 = v0 ? buf[i0] : 0;
            const uint32_t lt = v0 ? (uint32_t)lab[u0] : 0u;
            if (v0) lab[u0] = (LT)(lt & LM);
            const int rel = v0 ? i0 - c : 0;  // candidate is after choice g iff rel > g
            const uint32_t lb = cpt ? (uint32_t)xmw[lt & LM] : (lt & LM);
            if (wide_tail) {
              // One match groups the batch's lanes for every choice of the
              // group (k <= 5, and k = 6 launches over many graphs).  A leaf's
              // key for choice g is a function of the candidate's relation word
              // (its bits to the first k-2 vertices and the group's slot
              // codes), and the candidate is a leaf of choices 0 .. vc-1,
              // vc = min(ng, rel); lanes with equal word and vc have equal keys
              // for every choice, and the leader of such a group classifies it
              // for each of its vc choices.
              constexpr int WB = NB + 2 * GS;  // relation-word bits in use (<= 24)
              const uint32_t vc = (uint32_t)min(ng, rel);
              const uint32_t tag = (lt & ((1u << WB) - 1u)) | (vc << WB);
              const unsigned peers = __match_any_sync(kFull, vc ? tag : 0xFFFFFFFFu);
              if (vc && !(peers & lanes_below)) {
                const int cnt = __popc(peers);
                uint32_t id[GS];
#pragma unroll
                for (int gg = 0; gg < GS; ++gg)
                  id[gg] = gg < (int)vc
                               ? __ldg(&a.table[pgs[gg] | ((lb | ((lt >> (2 * gg)) & (3u << NB))) << OFF1)])
                               : 0u;
#pragma unroll
                for (int gg = 0; gg < GS; ++gg)
                  if (gg < (int)vc) ladd(id[gg], cnt);
              }
            } else {
              // k = 6 over few graphs: one match groups the lanes for M = 3
              // choices at once, so a leader adds for at most three.  The tag
              // holds M fields of NB + 2 bits, the leaf's word for a choice it
              // is a leaf of and 0 otherwise (a candidate is adjacent to the
              // first k-2 vertices, so its word is never 0: at most 30 tag
              // bits, so no tag is all ones), and a group's leader classifies
              // it for each choice it is a leaf of.
              constexpr int FB = NB + 2;
              constexpr int M = (31 / FB) < GS ? (31 / FB) : GS;
#pragma unroll
              for (int g0 = 0; g0 < GS; g0 += M) {
                if (g0 < ng) {
                  uint32_t tag = 0, wdv[M];
                  bool vv[M];
                  bool any = false;
#pragma unroll
                  for (int t = 0; t < M; ++t) {
                    const int gg = g0 + t;
                    vv[t] = gg < ng && rel > gg;
                    wdv[t] = lb | ((lt >> (2 * gg)) & (3u << NB));
                    tag |= (vv[t] ? wdv[t] : 0u) << (FB * t);
                    any |= vv[t];
                  }
                  const unsigned peers = __match_any_sync(kFull, any ? tag : 0xFFFFFFFFu);
                  if (any && !(peers & lanes_below)) {
                    const int cnt = __popc(peers);
                    uint32_t id[M];
#pragma unroll
                    for (int t = 0; t < M; ++t)
                      id[t] = vv[t] ? __ldg(&a.table[pgs[(g0 + t) % GS] | (wdv[t] << OFF1)]) : 0u;
#pragma unroll
                    for (int t = 0; t < M; ++t)
                      if (vv[t]) ladd(id[t], cnt);
                  }
                }
              }
            }
          }
          __syncwarp();
          continue;
        }
        if (c < ce) {
          // work donation: with an idle warp in the block, hand the second
          // half of this level's remaining choices over as a new item (a
          // first-level range, or a second-level range under the current
          // first-level choice)
          int cee = ce;
          if (L <= 2 && L < K - 2 && ce - c >= 2) {
            int hungry = 0;
            if (lane == 0) hungry = *v_idle > 0 && *v_ndon < kDonSlots;
            hungry = __shfl_sync(kFull, hungry, 0);
            if (hungry) {
              const int mid = c + (ce - c + 1) / 2;
              int ok = 0;
              if (lane == 0) {
                Item d;
                d.g = (uint32_t)g;
                d.root = (uint32_t)v;
                if (L == 1) {
                  d.j1a = (uint16_t)(j1a + mid);
                  d.j1b = (uint16_t)(j1a + ce);
                  d.a2 = 0;
                  d.b2 = 0xFFFF;
                } else {
                  const int c1 = lvs[5] - 1;  // index of the first-level choice
                  d.j1a = (uint16_t)(j1a + c1);
                  d.j1b = (uint16_t)(j1a + c1 + 1);
                  d.a2 = (uint16_t)(mid - (c1 + 1));
                  d.b2 = (uint16_t)(ce - (c1 + 1));
                }
                if (block_lock()) {
                  const int nd = *v_ndon;
                  if (nd < kDonSlots) {
                    uint4 raw;
                    memcpy(&raw, &d, sizeof(Item));
                    v_don[4 * nd] = raw.x;
                    v_don[4 * nd + 1] = raw.y;
                    v_don[4 * nd + 2] = raw.z;
                    v_don[4 * nd + 3] = raw.w;
                    *v_ndon = nd + 1;
                    ok = 1;
                  }
                  block_unlock();
                }
              }
              ok = __shfl_sync(kFull, ok, 0);
              if (ok) cee = mid;
            }
          }
          const int x = buf[c];
          const uint32_t nkey = key | (((uint32_t)lab[x] & ((1u << (2 * L)) - 1u)) << key_off(K, L));
          const int ne = push_vertex(w, x, L, e, (1u << (2 * (K - 2))) - 1u);
          if (lane == 0) {
            int* sv = lvs + 5 * L;
            sv[0] = c + 1;
            sv[1] = cee;
            sv[2] = e;
            sv[3] = (int)key;
            sv[4] = x;
          }
          __syncwarp();
          cur_c = c + 1;
          cur_ce = ne;
          cur_e = ne;
          cur_key = nkey;
          if (L == 1 && has2) {
            cur_c = c + 1 + it.a2;
            cur_ce = min(c + 1 + (int)it.b2, ne);
          }
          L += 1;
          if (L == K - 2) fresh = true;
        } else {
          if (L == 1) break;
          pop_level();
        }
      }
      // pop the root
      for (int b = f; b < re; b += 32) {
        const int i = b + lane;
        if (i < re) lab[w.ucol[i] & kVertexMask] &= (LT)~3u;
      }
      __syncwarp();
    }
    // this graph's queue is empty: flush, then move to a graph with items left
    __syncthreads();
    since = 0;
    if (K <= 5) {
      for (int i = tid; i < (int)C; i += blockDim.x) {
        const int32_t x = s_hist[i];
        if (x) {
          atomicAdd(&ghist[i], (unsigned long long)(long long)x);
          s_hist[i] = 0;
        }
      }
      if (tid == 0 && s_hist[C] != 0) {
        atomicOr(w.err, kErrStackOverflow);
        s_hist[C] = 0;
      }
    }
    if (tid == 0) {
      s_idle = 0;
      s_ndon = 0;
      int next = -1;
      for (int t = 1; t <= a.G; ++t) {
        const int g2 = (g + t) % a.G;
        const int n2 = a.item_off[(int64_t)(g2 + 1) * a.nmax] - a.item_off[(int64_t)g2 * a.nmax];
        if ((int)*(volatile uint32_t*)&a.qhead[g2] < n2) {
          next = g2;
          break;
        }
      }
      s_cur_g = next;
    }
    __syncthreads();
    g = s_cur_g;
  }
  if (bad_id) atomicOr(&a.hdr->err, kErrStackOverflow);
}

// ------------------------------------------------------------------ host side

static size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }

template <int K, bool CB>
static const void* pick_kernel_kc(bool gc, bool ls, bool sg) {
  if (sg) return ls ? (const void*)k_count<K, false, true, CB, true>
                    : (const void*)k_count<K, false, false, CB, true>;
  if (gc) return ls ? (const void*)k_count<K, true, true, CB> : (const void*)k_count<K, true, false, CB>;
  return ls ? (const void*)k_count<K, false, true, CB> : (const void*)k_count<K, false, false, CB>;
}

template <int K>
static const void* pick_kernel_k(bool gc, bool ls, bool cb, bool sg) {
  return cb ? pick_kernel_kc<K, true>(gc, ls, sg) : pick_kernel_kc<K, false>(gc, ls, sg);
}

static const void* pick_kernel(int K, bool gc, bool ls, bool cb, bool sg) {
  switch (K) {
    case 3: return pick_kernel_k<3>(gc, ls, cb, sg);
    case 4: return pick_kernel_k<4>(gc, ls, cb, sg);
    case 5: return pick_kernel_k<5>(gc, ls, cb, sg);
    default: return pick_kernel_k<6>(gc, ls, cb, sg);
  }
}

mt_status count_configure(CountPlan* p, int K, int G, int nmax, int dmax, int64_t fwd_bound,
                          int64_t entry_stride, uint32_t classes, double split_cost,
                          int warps_per_block, bool compact) {
  mt_tuning t;
  t.split_cost = split_cost;
  t.split_scale = 0.0;
  t.warps_per_block = warps_per_block;
  t.stack_cap = 0;
  t.method = MT_METHOD_ENUMERATE;
  const bool plain = split_cost == 0.0;
  MT_TRY(count_configure_tuned(p, K, G, nmax, dmax, fwd_bound, entry_stride, classes,
                               plain && warps_per_block == 0 ? nullptr : &t, compact));
  return MT_OK;
}

mt_status count_configure_tuned(CountPlan* p, int K, int G, int nmax, int dmax, int64_t fwd_bound,
                                int64_t entry_stride, uint32_t classes, const mt_tuning* tuning,
                                bool compact) {
  if (K < 3 || K > 6 || G < 1 || nmax < 1) return MT_EINVAL;
  const double split_cost = tuning ? tuning->split_cost : 0.0;
  const int warps_per_block = tuning ? tuning->warps_per_block : 0;
  p->K = K;
  p->G = G;
  p->nmax = nmax;
  p->dmax = dmax;
  p->fwd_bound = fwd_bound;
  p->entry_stride = entry_stride > 0 ? entry_stride : 1;
  p->classes = classes;
  p->split_cost = split_cost;
  p->split_scale = (tuning && tuning->split_scale > 0.0) ? tuning->split_scale : 1.0;
  p->items_factor = tuning ? 5.0 : 1.25;
  // The stack holds the root's forward list and the exclusive neighbours of the
  // vertices at positions 1..k-3 (positions k-2 and k-1 are finished in place),
  // each at most one row: k-2 rows of at most dmax entries.
  p->cap = (tuning && tuning->stack_cap > 0) ? tuning->stack_cap
                                             : std::max(K - 2, 1) * std::max(dmax, 1) + 32;
  if (p->cap > 65535) return MT_EUNSUPPORTED;
  p->nu_cap = (int)p->entry_stride;
  p->comb = tuning && tuning->method == MT_METHOD_CELLS;
  p->compact = compact;
  if (compact && (K != 6 || p->comb)) return MT_EUNSUPPORTED;
  p->map_bytes = compact ? 256 : 0;
  const size_t lab_elem = (K <= 4 || (p->comb && K <= 5)) ? 1 : ((K == 5 || p->comb) ? 2 : 4);
  const size_t lab_bytes = round16((size_t)nmax * lab_elem);
  const size_t cells = (size_t)1 << (2 * (K - 2));
  const size_t cell_bytes =
      p->comb ? round16(cells * 4) + round16(std::min<size_t>(cells, p->cap) * 2) + 384 + 16 : 0;
  const size_t buf_bytes = round16((size_t)p->cap * 2) + cell_bytes + kLevelBytes + p->map_bytes;
  // k <= 5: one 32-bit counter per class plus a catch slot for invalid ids
  const size_t hist_bytes = K <= 5 ? round16(((size_t)classes + 1) * 4) : 0;
  const size_t graph_bytes = round16((size_t)(nmax + 1) * 4) + round16((size_t)p->nu_cap * 4);
  int dev = 0, sms = 0, max_smem = 0;
  MT_CUDA_TRY(cudaGetDevice(&dev));
  MT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  MT_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t budget = (size_t)max_smem - 1024;
  const int want = warps_per_block > 0 ? std::min(warps_per_block, kMaxWarpsPerBlock)
                                       : kMaxWarpsPerBlock;
  // Layout: the one that fits the most warps (>= 16 if any does), and on a tie
  // the first of: graph copy and relation words in shared memory, relation
  // words only, graph only, neither.  More warps beat the graph copy: rows
  // read through L1 cost less than the warps the copy displaces.
  struct Opt { bool gc, ls; };
  const Opt opts[4] = {{true, true}, {false, true}, {true, false}, {false, false}};
  bool found = false;
  for (int pass = 0; pass < 2 && !found; ++pass) {
    const int min_w = pass == 0 ? std::min(want, 16) : 1;
    int best_w = 0;
    for (const Opt& o : opts) {
      const size_t fixed = (o.gc ? graph_bytes : 0) + hist_bytes;
      const size_t per = (o.ls ? lab_bytes : 0) + buf_bytes;
      int w = want;
      while (w > min_w && fixed + (size_t)w * per > budget) --w;
      if (fixed + (size_t)w * per <= budget && w > best_w) {
        p->gcache = o.gc;
        p->lab_smem = o.ls;
        p->warps_per_block = w;
        p->smem_bytes = fixed + (size_t)w * per;
        found = true;
        best_w = w;
      }
    }
  }
  // Graphs with hubs so large that no shared-memory layout holds 16 warps'
  // candidate stacks: the stacks go to per-warp slices of global memory
  // (L1/L2-cached), with the relation words in shared memory when they fit.
  const size_t stack_bytes = round16((size_t)p->cap * 2);
  p->stack_global = false;
  if (!found || p->warps_per_block < std::min(want, 16)) {
    int best_w = found ? p->warps_per_block : 0;
    for (const bool ls : {true, false}) {
      const size_t per = (ls ? lab_bytes : 0) + buf_bytes - stack_bytes;
      int w = want;
      while (w > 1 && hist_bytes + (size_t)w * per > budget) --w;
      if (hist_bytes + (size_t)w * per <= budget && w > best_w) {
        p->gcache = false;
        p->lab_smem = ls;
        p->stack_global = true;
        p->warps_per_block = w;
        p->smem_bytes = hist_bytes + (size_t)w * per;
        found = true;
        best_w = w;
      }
    }
  }
  if (!found) return MT_EUNSUPPORTED;
  p->graph_bytes = p->gcache ? graph_bytes : 0;
  p->hist_bytes = hist_bytes;
  p->lab_bytes = lab_bytes;
  p->buf_bytes = buf_bytes - cell_bytes - kLevelBytes - p->map_bytes;
  p->cell_bytes = cell_bytes;
  const void* kern = pick_kernel(K, p->gcache, p->lab_smem, p->comb, p->stack_global);
  MT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)p->smem_bytes));
  int occ = 0;
  MT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, p->warps_per_block * 32,
                                                            p->smem_bytes));
  if (occ < 1) return MT_EUNSUPPORTED;
  p->blocks = sms * occ;
  const double target = (double)p->blocks * p->warps_per_block * kTargetItemsPerWarp;
  p->items_max = (uint64_t)(target * p->items_factor) + (uint64_t)G * nmax +
                 2 * (uint64_t)fwd_bound + 4096;
  size_t off = 0;
  p->off_hdr = off; off += 256;
  p->off_qhead = off; off += round16((size_t)G * 4);
  p->off_est = off; off += round16((size_t)G * p->entry_stride * 4) * 2;
  p->off_cnt = off; off += round16(((size_t)G * nmax + 1) * 4);
  p->off_items = off; off += round16(p->items_max * sizeof(Item));
  p->off_lab = off;
  if (!p->lab_smem) off += (size_t)p->blocks * p->warps_per_block * lab_bytes;
  p->off_stack = off;
  if (p->stack_global) off += (size_t)p->blocks * p->warps_per_block * p->buf_bytes;
  p->ws_bytes = off + 256;
  return MT_OK;
}

uint32_t* count_err_ptr(const CountPlan& p, void* ws) {
  return &((Hdr*)((char*)ws + p.off_hdr))->err;
}
uint32_t* count_nitems_ptr(const CountPlan& p, void* ws) {
  return (uint32_t*)((char*)ws + p.off_cnt) + (size_t)p.G * p.nmax;
}

template <int K, bool CB>
static void launch_count(const CountPlan& p, const CountArgs& a, unsigned threads, cudaStream_t s) {
  if (p.stack_global) {
    if (p.lab_smem) k_count<K, false, true, CB, true><<<p.blocks, threads, p.smem_bytes, s>>>(a);
    else k_count<K, false, false, CB, true><<<p.blocks, threads, p.smem_bytes, s>>>(a);
  } else if (p.gcache) {
    if (p.lab_smem) k_count<K, true, true, CB><<<p.blocks, threads, p.smem_bytes, s>>>(a);
    else k_count<K, true, false, CB><<<p.blocks, threads, p.smem_bytes, s>>>(a);
  } else {
    if (p.lab_smem) k_count<K, false, true, CB><<<p.blocks, threads, p.smem_bytes, s>>>(a);
    else k_count<K, false, false, CB><<<p.blocks, threads, p.smem_bytes, s>>>(a);
  }
}

template <int K>
static cudaError_t enqueue_k(const CountPlan& p, void* ws, const DevGraph* graphs,
                             const TableView& table, int32_t rb, int32_t re, cudaStream_t s,
                             unsigned long long* copies_base, int copies, uint32_t copy_stride) {
  char* base = (char*)ws;
  Hdr* hdr = (Hdr*)(base + p.off_hdr);
  uint32_t* qhead = (uint32_t*)(base + p.off_qhead);
  float* est = (float*)(base + p.off_est);
  int32_t* x1s = (int32_t*)(base + p.off_est + round16((size_t)p.G * p.entry_stride * 4));
  int32_t* cnt = (int32_t*)(base + p.off_cnt);
  Item* items = (Item*)(base + p.off_items);
  void* lab = base + p.off_lab;
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(Hdr), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(qhead, 0, (size_t)p.G * 4, s);
  if (e != cudaSuccess) return e;
  const int ex = (int)std::min<int64_t>((p.entry_stride + 255) / 256, 4096);
  k_plan_est<K><<<dim3(ex, p.G), 256, 0, s>>>(graphs, p.entry_stride, est, x1s, hdr, rb, re);
  const int rx = (p.nmax + 7) / 8;  // one warp per root, 8 per block
  const double target = (double)p.blocks * p.warps_per_block * kTargetItemsPerWarp;
  k_plan_items<K, false><<<dim3(rx, p.G), 256, 0, s>>>(graphs, p.entry_stride, est, x1s, p.nmax,
                                                       cnt, items, p.items_max, hdr, p.split_cost,
                                                       p.split_scale, target, p.items_factor, rb,
                                                       re);
  k_scan_counts<<<1, 1024, 0, s>>>(cnt, p.G * p.nmax + 1);
  k_plan_items<K, true><<<dim3(rx, p.G), 256, 0, s>>>(graphs, p.entry_stride, est, x1s, p.nmax,
                                                      cnt, items, p.items_max, hdr, p.split_cost,
                                                      p.split_scale, target, p.items_factor, rb,
                                                      re);
  if (!p.lab_smem) {
    e = cudaMemsetAsync(lab, 0, (size_t)p.blocks * p.warps_per_block * p.lab_bytes, s);
    if (e != cudaSuccess) return e;
  }
  CountArgs a;
  a.graphs = graphs;
  a.items = items;
  a.item_off = cnt;
  a.qhead = qhead;
  a.hdr = hdr;
  a.table = table.slots;
  a.xclass = p.compact ? table.xclass : nullptr;
  a.xmap = p.compact ? table.xmap : nullptr;
  a.map_bytes = (int)p.map_bytes;
  a.idle_ns = g_idle_ns;
  a.lab_global = lab;
  a.stack_global = base + p.off_stack;
  a.hist_copies = copies_base;
  a.copies = copies;
  a.copy_stride = copy_stride;
  a.G = p.G;
  a.nmax = p.nmax;
  a.nu_cap = p.nu_cap;
  a.cap = p.cap;
  a.classes = p.classes;
  a.graph_bytes = (int)p.graph_bytes;
  a.hist_bytes = (int)p.hist_bytes;
  a.lab_bytes = (int)p.lab_bytes;
  a.buf_bytes = (int)p.buf_bytes;
  a.cell_bytes = (int)p.cell_bytes;
  const unsigned threads = p.warps_per_block * 32;
  if (p.comb) launch_count<K, true>(p, a, threads, s);
  else launch_count<K, false>(p, a, threads, s);
  return cudaGetLastError();
}

mt_status count_enqueue(const CountPlan& p, void* ws, const DevGraph* graphs,
                        const TableView& table, int32_t root_begin, int32_t root_end,
                        cudaStream_t s, unsigned long long* copies_base, int copies,
                        uint32_t copy_stride) {
  if (copies > 1 && (p.K != 6 || p.G != 1 || !copies_base)) return MT_EINVAL;
  cudaError_t e;
  switch (p.K) {
    case 3: e = enqueue_k<3>(p, ws, graphs, table, root_begin, root_end, s, nullptr, 1, 0); break;
    case 4: e = enqueue_k<4>(p, ws, graphs, table, root_begin, root_end, s, nullptr, 1, 0); break;
    case 5: e = enqueue_k<5>(p, ws, graphs, table, root_begin, root_end, s, nullptr, 1, 0); break;
    default:
      e = enqueue_k<6>(p, ws, graphs, table, root_begin, root_end, s, copies_base, copies,
                       copy_stride);
      break;
  }
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MT_ENOMEM : MT_ECUDA;
  }
  return MT_OK;
}

// Histogram copies of a one-graph count (see kHistCopies).
static int count_hist_copies(const CountPlan& p) { return p.K == 6 && p.G == 1 ? kHistCopies : 1; }

// Scratch of a one-graph count: plan workspace + the DevGraph + a histogram +
// the histogram's extra copies.
static size_t count_scratch_bytes(const CountPlan& p, uint32_t C) {
  return p.ws_bytes + 256 + (size_t)count_hist_copies(p) * round16((size_t)C * 8);
}

// Plain one-graph count with the workspace cached in the graph handle.
static mt_status count_one(const mt_graph* gc, const mt_table* t, uint64_t* hist,
                           int32_t rb, int32_t re, const mt_tuning* tuning, cudaStream_t s) {
  mt_graph* g = const_cast<mt_graph*>(gc);
  const int K = table_k(t);
  const uint32_t C = table_classes(t);
  CountPlan p;
  MT_TRY(count_configure_tuned(&p, K, 1, g->n, g->dmax, g->nu / 2 + 1, std::max(g->nu, 1), C,
                               tuning, table_compact(t)));
  // workspace: plan scratch + the DevGraph + a device histogram
  const size_t need = count_scratch_bytes(p, C);
  if (!g->ws_owned && g->ws_bytes < need) {
    set_last_error("attached workspace holds " + std::to_string(g->ws_bytes) +
                   " bytes, this count needs " + std::to_string(need));
    return MT_EINVAL;
  }
  if (g->ws_bytes < need) {
    if (g->ws) {
      // an earlier count may still use the old scratch, on any stream
      MT_CUDA_TRY(cudaDeviceSynchronize());
      cudaFree(g->ws);
      g->ws = nullptr;
      g->ws_bytes = 0;
    }
    MT_CUDA_TRY(cudaMalloc(&g->ws, need));
    g->ws_bytes = need;
  }
  if (!g->ev0) {
    MT_CUDA_TRY(cudaEventCreate(&g->ev0));
    MT_CUDA_TRY(cudaEventCreate(&g->ev1));
  }
  char* base = (char*)g->ws;
  DevGraph* dg = (DevGraph*)(base + p.ws_bytes);
  cudaPointerAttributes attr;
  bool dev_hist = cudaPointerGetAttributes(&attr, hist) == cudaSuccess &&
                  (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (dev_hist && attr.type == cudaMemoryTypeDevice) {
    int dev = 0;
    MT_CUDA_TRY(cudaGetDevice(&dev));
    if (attr.device != dev) {  // this device's kernels would write another GPU's memory
      set_last_error("hist is memory of device " + std::to_string(attr.device) +
                     ", the current device is " + std::to_string(dev));
      return MT_EINVAL;
    }
  }
  unsigned long long* dh =
      dev_hist ? (unsigned long long*)hist : (unsigned long long*)(base + p.ws_bytes + 256);
  DevGraph hg = dev_view(g, dh);
  MT_CUDA_TRY(cudaMemcpyAsync(dg, &hg, sizeof(DevGraph), cudaMemcpyHostToDevice, s));
  MT_CUDA_TRY(cudaMemsetAsync(dh, 0, (size_t)C * 8, s));
  if (g->n >= K && rb < re) {
    const int copies = count_hist_copies(p);
    const uint32_t stride = (uint32_t)(round16((size_t)C * 8) / 8);
    unsigned long long* cbase = (unsigned long long*)(base + p.ws_bytes + 256) + stride;
    MT_CUDA_TRY(cudaEventRecord(g->ev0, s));
    if (copies > 1)
      MT_CUDA_TRY(cudaMemsetAsync(cbase, 0, (size_t)(copies - 1) * stride * 8, s));
    MT_TRY(count_enqueue(p, g->ws, dg, table_view(t), rb, re, s, cbase, copies, stride));
    if (copies > 1) {
      const unsigned fb = (unsigned)std::min<uint32_t>((C + 255) / 256, 152u * 8u);
      k_fold_copies<<<fb, 256, 0, s>>>(dh, cbase, copies - 1, C, stride);
      MT_CUDA_TRY(cudaGetLastError());
    }
    MT_CUDA_TRY(cudaEventRecord(g->ev1, s));
  } else {
    MT_CUDA_TRY(cudaEventRecord(g->ev0, s));
    MT_CUDA_TRY(cudaEventRecord(g->ev1, s));
  }
  if (!dev_hist) {
    MT_CUDA_TRY(cudaMemcpyAsync(hist, dh, (size_t)C * 8, cudaMemcpyDeviceToHost, s));
  }
  g->stats_valid = true;
  g->off_err = (size_t)((char*)count_err_ptr(p, g->ws) - base);
  g->off_nitems = (size_t)((char*)count_nitems_ptr(p, g->ws) - base);
  if (!dev_hist) {
    uint32_t err = 0;
    MT_CUDA_TRY(cudaMemcpyAsync(&err, base + g->off_err, 4, cudaMemcpyDeviceToHost, s));
    MT_CUDA_TRY(cudaStreamSynchronize(s));
    if (err) return (err & kErrWaitLimit) ? MT_ETIMEOUT : MT_EOVERFLOW;
  }
  return MT_OK;
}

}  // namespace mt

using namespace mt;

extern "C" {

mt_status mt_count_roots(const mt_graph* g, const mt_table* t, int32_t root_begin,
                         int32_t root_end, uint64_t* hist, void* stream) {
  if (!g || !t || !hist) return MT_EINVAL;
  if (root_begin < 0) root_begin = 0;
  if (root_end > g->n) root_end = g->n;
  return count_one(g, t, hist, root_begin, root_end, nullptr, (cudaStream_t)stream);
}

mt_status mt_count(const mt_graph* g, const mt_table* t, uint64_t* hist, void* stream) {
  if (!g || !t || !hist) return MT_EINVAL;
  return count_one(g, t, hist, 0, g->n, nullptr, (cudaStream_t)stream);
}

mt_status mt_count_tuned(const mt_graph* g, const mt_table* t, uint64_t* hist,
                         const mt_tuning* tuning, void* stream) {
  if (!g || !t || !hist) return MT_EINVAL;
  if (tuning && (tuning->split_cost < 0 || tuning->split_scale < 0 ||
                 tuning->warps_per_block < 0 || tuning->warps_per_block > 32 ||
                 tuning->stack_cap < 0 || tuning->stack_cap > 65535 ||
                 tuning->method < 0 || tuning->method > 1))
    return MT_EINVAL;
  return count_one(g, t, hist, 0, g->n, tuning, (cudaStream_t)stream);
}

mt_status mt_set_wait_limit(uint64_t ns) {
  g_idle_ns = ns ? (unsigned long long)ns : kIdleNs;
  return MT_OK;
}

mt_status mt_workspace_query(const mt_graph* g, int k, size_t* bytes) {
  if (!g || !bytes) return MT_EINVAL;
  if (k < 3 || k > 6) return MT_EUNSUPPORTED;
  CountPlan p;
  MT_TRY(count_configure_tuned(&p, k, 1, g->n, g->dmax, g->nu / 2 + 1, std::max(g->nu, 1),
                               kNumClasses[k], nullptr));
  *bytes = count_scratch_bytes(p, kNumClasses[k]);
  return MT_OK;
}

mt_status mt_count_launch_info(const mt_graph* g, int k, int32_t* warps_per_block,
                               int32_t* blocks, int32_t* stack_cap, uint32_t* layout) {
  if (!g) return MT_EINVAL;
  if (k < 3 || k > 6) return MT_EUNSUPPORTED;
  CountPlan p;
  MT_TRY(count_configure_tuned(&p, k, 1, g->n, g->dmax, g->nu / 2 + 1, std::max(g->nu, 1),
                               kNumClasses[k], nullptr));
  if (warps_per_block) *warps_per_block = p.warps_per_block;
  if (blocks) *blocks = p.blocks;
  if (stack_cap) *stack_cap = p.cap;
  if (layout)
    *layout = (p.gcache ? 1u : 0u) | (p.lab_smem ? 2u : 0u) | (p.stack_global ? 4u : 0u);
  return MT_OK;
}

mt_status mt_set_workspace(mt_graph* g, void* ws, size_t bytes) {
  if (!g) return MT_EINVAL;
  if (ws) {
    cudaPointerAttributes attr;
    const bool dev = cudaPointerGetAttributes(&attr, ws) == cudaSuccess &&
                     attr.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    if (!dev || ((uintptr_t)ws & 255u) || bytes == 0) {
      set_last_error("mt_set_workspace: ws must be device memory, 256-byte aligned, non-empty");
      return MT_EINVAL;
    }
  }
  // an earlier count may still use the current scratch, on any stream
  MT_CUDA_TRY(cudaDeviceSynchronize());
  if (g->ws && g->ws_owned) cudaFree(g->ws);
  g->ws = ws;
  g->ws_bytes = ws ? bytes : 0;
  g->ws_owned = ws == nullptr;
  g->stats_valid = false;
  return MT_OK;
}

mt_status mt_count_stats(const mt_graph* g, uint64_t* items, uint32_t* err, float* ms) {
  if (!g) return MT_EINVAL;
  uint32_t it = 0, er = 0;
  float t = 0.f;
  if (g->stats_valid) {
    MT_CUDA_TRY(cudaEventSynchronize(g->ev1));
    MT_CUDA_TRY(cudaMemcpy(&it, (char*)g->ws + g->off_nitems, 4, cudaMemcpyDeviceToHost));
    MT_CUDA_TRY(cudaMemcpy(&er, (char*)g->ws + g->off_err, 4, cudaMemcpyDeviceToHost));
    MT_CUDA_TRY(cudaEventElapsedTime(&t, g->ev0, g->ev1));
  }
  if (items) *items = it;
  if (err) *err = er;
  if (ms) *ms = t;
  return MT_OK;
}

}  // extern "C"
