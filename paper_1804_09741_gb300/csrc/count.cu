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
//  * per warp a 16-bit "relation word" lab[u] for every vertex: bits 2p, 2p+1
//    hold the A/B/C relation (Sec. 2) of u to the vertex at position p of the
//    current set.  Pushing w at position p scans delta(w) coalesced (the
//    row-scan strategy of Sec. 3.1, Algorithm 3), ORs its relation bits into
//    lab[u] and, with one ballot, appends to the candidate stack every u whose
//    word was zero (exclusive neighbour).  Popping clears the same bits.
//  * candidate lists of all levels live in one per-warp stack: level p+1's list
//    is the unused tail of level p's list followed by the newly appended
//    exclusive neighbours, so no list is ever copied;
//  * level state (cursor, ends, pushed vertex, key prefix) lives in registers of
//    lane p and is read with shuffles;
//  * the class key of a leaf u is the key prefix of the set OR lab[u] shifted to
//    the last position: no per-subgraph adjacency test at all;
//  * histograms: per-warp shared-memory counters for k <= 4 (13 / 199 classes),
//    warp-aggregated (match_any) 64-bit global atomics for k = 5, 6.
//
// Work items are (graph, root, first-level branch range) or, for expensive
// branches, (graph, root, branch, second-level choice range); a planner sizes
// them from per-branch cost estimates and warps take them from a global queue.
#include <algorithm>

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
constexpr int kTargetItemsPerWarp = 24;
constexpr int kMaxWarpsPerBlock = 16;

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

// First index in sorted packed entries [lo, hi) whose vertex is > x.
__device__ __forceinline__ int first_above(const uint32_t* __restrict__ ucol, int lo, int hi,
                                           int x) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((int)(__ldg(&ucol[mid]) & kVertexMask) > x) hi = mid; else lo = mid + 1;
  }
  return lo;
}

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
    if (u > v && v >= root_begin && v < root_end) {
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
template <int K, bool WRITE>
__global__ void __launch_bounds__(256) k_plan_items(const DevGraph* __restrict__ graphs,
                                                    int64_t stride, const float* est,
                                                    const int32_t* x1s, int nmax, int32_t* cnt,
                                                    Item* items, uint64_t items_max, Hdr* hdr,
                                                    double split_cost, double target_items,
                                                    int root_begin, int root_end) {
  const int g = blockIdx.y;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (!WRITE && g == 0 && v == 0) cnt[(int64_t)gridDim.y * nmax] = 0;
  if (v >= nmax) return;
  const int64_t slot = (int64_t)g * nmax + v;
  const DevGraph G = graphs[g];
  if (v >= G.n || v < root_begin || v >= root_end) {
    if (!WRITE) cnt[slot] = 0;
    return;
  }
  double T = hdr->total_est / target_items;
  if (split_cost > T) T = split_cost;
  if (T < 1.0) T = 1.0;
  const float Tf = (float)T;
  const int re = G.urow[v + 1];
  const int f = G.urow[v] + G.ufwd[v];
  const int dplus = re - f;
  int64_t pos = WRITE ? cnt[slot] : 0;
  int count = 0;
  auto emit = [&](int j1a, int j1b, int a2, int b2) {
    if (WRITE) {
      if ((uint64_t)pos < items_max) {
        Item it;
        it.g = (uint32_t)g;
        it.root = (uint32_t)v;
        it.j1a = (uint16_t)j1a;
        it.j1b = (uint16_t)j1b;
        it.a2 = (uint16_t)a2;
        it.b2 = (uint16_t)b2;
        items[pos] = it;
      } else {
        atomicOr(&hdr->err, kErrStackOverflow);
      }
      ++pos;
    }
    ++count;
  };
  float acc = 0.f;
  int start = 0;
  for (int j = 0; j < dplus; ++j) {
    const int64_t e = (int64_t)g * stride + f + j;
    const float c = est[e];
    const int x = x1s[e];
    if (K >= 4 && c > 2.f * Tf && x >= 2) {
      if (j > start) emit(start, j, 0, 0xFFFF);
      int nch = (int)ceilf(c / Tf);
      if (nch > x) nch = x;
      const int r2 = (x + nch - 1) / nch;
      for (int a = 0; a < x; a += r2) emit(j, j + 1, a, min(a + r2, x));
      start = j + 1;
      acc = 0.f;
    } else {
      acc += c;
      if (acc >= Tf) {
        emit(start, j + 1, 0, 0xFFFF);
        start = j + 1;
        acc = 0.f;
      }
    }
  }
  if (start < dplus) emit(start, dplus, 0, 0xFFFF);
  if (!WRITE) cnt[slot] = count;
}

__global__ void __launch_bounds__(1024) k_scan_counts(int32_t* data, int count) {
  __shared__ int tmp[33];
  block_exclusive_scan(data, count, tmp);
}

// ------------------------------------------------------------------ enumerator

struct WarpCtx {
  const int32_t* __restrict__ urow;
  const uint32_t* __restrict__ ucol;
  uint16_t* lab;
  uint16_t* buf;
  int cap;
  int root;
  int lane;
  uint32_t* err;
};

// Push w at position p: OR its relation bits into lab[] of its neighbours
// above the root and append the exclusive ones at stack index e.  Returns the
// new end of the candidate list.
__device__ __forceinline__ int push_vertex(const WarpCtx& w, int x, int p, int e) {
  const int rs = __ldg(&w.urow[x]), re = __ldg(&w.urow[x + 1]);
  const int start = (re - rs > 32) ? first_above(w.ucol, rs, re, w.root) : rs;
  const unsigned lt = (1u << w.lane) - 1u;
  int cnt = 0;
  for (int b = start; b < re; b += 32) {
    const int i = b + w.lane;
    bool ex = false;
    int u = 0;
    if (i < re) {
      const uint32_t ent = __ldg(&w.ucol[i]);
      u = (int)(ent & kVertexMask);
      if (u > w.root) {
        const uint16_t old = w.lab[u];
        w.lab[u] = (uint16_t)(old | ((ent >> 30) << (2 * p)));
        ex = (old == 0);
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
__device__ __forceinline__ void pop_vertex(const WarpCtx& w, int x, int p) {
  const int rs = __ldg(&w.urow[x]), re = __ldg(&w.urow[x + 1]);
  const int start = (re - rs > 32) ? first_above(w.ucol, rs, re, w.root) : rs;
  const uint16_t clear = (uint16_t)~(3u << (2 * p));
  for (int b = start; b < re; b += 32) {
    const int i = b + w.lane;
    if (i < re) {
      const int u = (int)(__ldg(&w.ucol[i]) & kVertexMask);
      if (u > w.root) w.lab[u] &= clear;
    }
  }
  __syncwarp();
}

template <int K, bool LAB_SMEM>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32)
    k_count(const DevGraph* __restrict__ graphs, const Item* __restrict__ items,
            const int32_t* n_items_p, uint64_t items_max, Hdr* hdr,
            const uint32_t* __restrict__ table, uint16_t* lab_global, int nmax, int cap,
            uint32_t classes, int lab_bytes, int buf_bytes, int hist_bytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int per_warp = (LAB_SMEM ? lab_bytes : 0) + buf_bytes + hist_bytes;
  unsigned char* mine = smem + (size_t)wid * per_warp;
  uint16_t* lab = LAB_SMEM ? (uint16_t*)mine
                           : lab_global + ((size_t)blockIdx.x * (blockDim.x >> 5) + wid) * nmax;
  uint16_t* buf = (uint16_t*)(mine + (LAB_SMEM ? lab_bytes : 0));
  uint32_t* whist = (uint32_t*)(mine + (LAB_SMEM ? lab_bytes : 0) + buf_bytes);
  if (LAB_SMEM)
    for (int i = lane; i < nmax; i += 32) lab[i] = 0;
  if (K <= 4)
    for (int i = lane; i < (int)classes; i += 32) whist[i] = 0;
  __syncwarp();

  const uint64_t nitems = min((uint64_t)(uint32_t)*n_items_p, items_max);
  int cur_g = -1;
  unsigned long long* cur_hist = nullptr;
  uint64_t pending = 0;

  WarpCtx w;
  w.lab = lab;
  w.buf = buf;
  w.cap = cap;
  w.lane = lane;
  w.err = &hdr->err;

  auto flush = [&]() {
    for (int i = lane; i < (int)classes; i += 32) {
      const uint32_t x = whist[i];
      if (x) {
        atomicAdd(&cur_hist[i], (unsigned long long)x);
        whist[i] = 0;
      }
    }
    __syncwarp();
    pending = 0;
  };

  while (true) {
    uint32_t idx = 0;
    if (lane == 0) idx = atomicAdd(&hdr->head, 1u);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx >= nitems) break;
    const Item it = items[idx];
    const DevGraph* Gp = graphs + it.g;
    if ((int)it.g != cur_g) {
      if (K <= 4 && cur_g >= 0) flush();
      cur_g = (int)it.g;
      cur_hist = Gp->hist;
      w.urow = Gp->urow;
      w.ucol = Gp->ucol;
    }
    const int v = (int)it.root;
    w.root = v;
    const int re = __ldg(&w.urow[v + 1]);
    const int f = __ldg(&w.urow[v]) + __ldg(&Gp->ufwd[v]);
    const int dplus = re - f;
    const int j1a = it.j1a, j1b = it.j1b;
    // push the root at position 0: every forward neighbour gets its relation
    // bits; candidates j1a.. are copied to the stack.
    for (int b = f; b < re; b += 32) {
      const int i = b + lane;
      if (i < re) {
        const uint32_t ent = __ldg(&w.ucol[i]);
        const int u = (int)(ent & kVertexMask);
        lab[u] |= (uint16_t)(ent >> 30);
        const int q = i - f - j1a;
        if (q >= 0) buf[q] = (uint16_t)u;
      }
    }
    __syncwarp();
    int s_c = 0, s_ce = 0, s_e = 0, s_vert = 0;
    uint32_t s_key = 0;
    if (lane == 1) {
      s_c = 0;
      s_ce = j1b - j1a;
      s_e = dplus - j1a;
    }
    if (lane == 0) s_vert = v;
    const bool has2 = it.b2 != 0xFFFF;
    int L = 1;
    while (true) {
      const int c = __shfl_sync(kFull, s_c, L);
      const int ce = __shfl_sync(kFull, s_ce, L);
      const int e = __shfl_sync(kFull, s_e, L);
      const uint32_t key = __shfl_sync(kFull, s_key, L);
      if (L == K - 1) {
        // leaves: every remaining candidate completes a k-set
        for (int b = c; b < e; b += 32) {
          const int i = b + lane;
          const bool valid = i < e;
          uint32_t id = kNoClass;
          if (valid) {
            const int u = buf[i];
            const uint32_t k2 = key | ((uint32_t)lab[u] << ((K - 1) * (K - 2)));
            id = __ldg(&table[k2]);
          }
          if (K <= 4) {
            if (valid) {
              if (id < classes) atomicAdd(&whist[id], 1u);
              else atomicOr(w.err, kErrStackOverflow);
            }
          } else {
            const unsigned act = __ballot_sync(kFull, valid);
            if (valid) {
              const unsigned peers = __match_any_sync(act, id);
              if (lane == __ffs(peers) - 1) {
                if (id < classes) atomicAdd(&cur_hist[id], (unsigned long long)__popc(peers));
                else atomicOr(w.err, kErrStackOverflow);
              }
            }
          }
        }
        if (K <= 4) pending += (uint64_t)(e > c ? e - c : 0);
        L -= 1;
        pop_vertex(w, __shfl_sync(kFull, s_vert, L), L);
        continue;
      }
      if (c < ce) {
        const int x = buf[c];
        if (lane == L) s_c = c + 1;
        const uint32_t nkey = key | ((uint32_t)lab[x] << (L * (L - 1)));
        const int ne = push_vertex(w, x, L, e);
        if (lane == L) s_vert = x;
        if (lane == L + 1) {
          s_c = c + 1;
          s_ce = ne;
          s_e = ne;
          s_key = nkey;
        }
        if (L == 1 && has2 && lane == 2) {
          s_c = c + 1 + it.a2;
          s_ce = min(c + 1 + (int)it.b2, ne);
        }
        L += 1;
      } else {
        if (L == 1) break;
        L -= 1;
        pop_vertex(w, __shfl_sync(kFull, s_vert, L), L);
      }
    }
    // pop the root
    for (int b = f; b < re; b += 32) {
      const int i = b + lane;
      if (i < re) lab[__ldg(&w.ucol[i]) & kVertexMask] &= (uint16_t)~3u;
    }
    __syncwarp();
    if (K <= 4 && pending > (1ull << 30)) flush();
  }
  if (K <= 4 && cur_g >= 0) flush();
}

// ------------------------------------------------------------------ host side

static size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }

template <int K, bool LS>
static const void* count_kernel() {
  return (const void*)k_count<K, LS>;
}

static const void* pick_kernel(int K, bool ls) {
  switch (K) {
    case 3: return ls ? count_kernel<3, true>() : count_kernel<3, false>();
    case 4: return ls ? count_kernel<4, true>() : count_kernel<4, false>();
    case 5: return ls ? count_kernel<5, true>() : count_kernel<5, false>();
    default: return ls ? count_kernel<6, true>() : count_kernel<6, false>();
  }
}

mt_status count_configure(CountPlan* p, int K, int G, int nmax, int dmax, int64_t fwd_bound,
                          int64_t entry_stride, uint32_t classes, double split_cost,
                          int warps_per_block) {
  if (K < 3 || K > 6 || G < 1 || nmax < 1) return MT_EINVAL;
  p->K = K;
  p->G = G;
  p->nmax = nmax;
  p->dmax = dmax;
  p->fwd_bound = fwd_bound;
  p->entry_stride = entry_stride > 0 ? entry_stride : 1;
  p->classes = classes;
  p->split_cost = split_cost;
  p->cap = (K - 1) * std::max(dmax, 1) + 32;
  if (p->cap > 65535) return MT_EUNSUPPORTED;
  const size_t lab_bytes = round16((size_t)nmax * 2);
  const size_t buf_bytes = round16((size_t)p->cap * 2);
  const size_t hist_bytes = K <= 4 ? round16((size_t)classes * 4) : 0;
  int dev = 0, sms = 0, max_smem = 0;
  MT_CUDA_TRY(cudaGetDevice(&dev));
  MT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  MT_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t budget = (size_t)max_smem - 1024;
  int wpb = warps_per_block > 0 ? std::min(warps_per_block, kMaxWarpsPerBlock) : kMaxWarpsPerBlock;
  bool ls = true;
  while (wpb > 1 && (size_t)wpb * (lab_bytes + buf_bytes + hist_bytes) > budget) wpb /= 2;
  if ((size_t)wpb * (lab_bytes + buf_bytes + hist_bytes) > budget || (warps_per_block == 0 && wpb < 8)) {
    ls = false;
    wpb = warps_per_block > 0 ? std::min(warps_per_block, kMaxWarpsPerBlock) : kMaxWarpsPerBlock;
    while (wpb > 1 && (size_t)wpb * (buf_bytes + hist_bytes) > budget) wpb /= 2;
    if ((size_t)wpb * (buf_bytes + hist_bytes) > budget) return MT_EUNSUPPORTED;
  }
  p->lab_smem = ls;
  p->warps_per_block = wpb;
  p->smem_bytes = (size_t)wpb * ((ls ? lab_bytes : 0) + buf_bytes + hist_bytes);
  const void* kern = pick_kernel(K, ls);
  MT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)p->smem_bytes));
  int occ = 0;
  MT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, wpb * 32, p->smem_bytes));
  if (occ < 1) return MT_EUNSUPPORTED;
  p->blocks = sms * occ;
  const double target = (double)p->blocks * wpb * kTargetItemsPerWarp;
  p->items_max = (uint64_t)(target * 1.25) + (uint64_t)G * nmax + 2 * (uint64_t)fwd_bound + 4096;
  // workspace layout
  size_t off = 0;
  p->off_hdr = off; off += 256;
  p->off_est = off; off += round16((size_t)G * p->entry_stride * 4) * 2;
  p->off_cnt = off; off += round16(((size_t)G * nmax + 1) * 4);
  p->off_items = off; off += round16(p->items_max * sizeof(Item));
  p->off_lab = off;
  if (!ls) off += round16((size_t)p->blocks * wpb * nmax * 2);
  p->ws_bytes = off + 256;
  return MT_OK;
}

uint32_t* count_err_ptr(const CountPlan& p, void* ws) {
  return &((Hdr*)((char*)ws + p.off_hdr))->err;
}
uint32_t* count_nitems_ptr(const CountPlan& p, void* ws) {
  return (uint32_t*)((char*)ws + p.off_cnt) + (size_t)p.G * p.nmax;
}

template <int K>
static cudaError_t enqueue_k(const CountPlan& p, void* ws, const DevGraph* graphs,
                             const uint32_t* table, int32_t rb, int32_t re, cudaStream_t s) {
  char* base = (char*)ws;
  Hdr* hdr = (Hdr*)(base + p.off_hdr);
  float* est = (float*)(base + p.off_est);
  int32_t* x1s = (int32_t*)(base + p.off_est + round16((size_t)p.G * p.entry_stride * 4));
  int32_t* cnt = (int32_t*)(base + p.off_cnt);
  Item* items = (Item*)(base + p.off_items);
  uint16_t* lab = (uint16_t*)(base + p.off_lab);
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(Hdr), s);
  if (e != cudaSuccess) return e;
  const int ex = (int)std::min<int64_t>((p.entry_stride + 255) / 256, 4096);
  k_plan_est<K><<<dim3(ex, p.G), 256, 0, s>>>(graphs, p.entry_stride, est, x1s, hdr, rb, re);
  const int rx = (p.nmax + 255) / 256;
  const double target = (double)p.blocks * p.warps_per_block * kTargetItemsPerWarp;
  k_plan_items<K, false><<<dim3(rx, p.G), 256, 0, s>>>(graphs, p.entry_stride, est, x1s, p.nmax,
                                                       cnt, items, p.items_max, hdr, p.split_cost,
                                                       target, rb, re);
  k_scan_counts<<<1, 1024, 0, s>>>(cnt, p.G * p.nmax + 1);
  k_plan_items<K, true><<<dim3(rx, p.G), 256, 0, s>>>(graphs, p.entry_stride, est, x1s, p.nmax,
                                                      cnt, items, p.items_max, hdr, p.split_cost,
                                                      target, rb, re);
  if (!p.lab_smem) {
    e = cudaMemsetAsync(lab, 0, (size_t)p.blocks * p.warps_per_block * p.nmax * 2, s);
    if (e != cudaSuccess) return e;
  }
  const int lab_bytes = (int)round16((size_t)p.nmax * 2);
  const int buf_bytes = (int)round16((size_t)p.cap * 2);
  const int hist_bytes = K <= 4 ? (int)round16((size_t)p.classes * 4) : 0;
  if (p.lab_smem)
    k_count<K, true><<<p.blocks, p.warps_per_block * 32, p.smem_bytes, s>>>(
        graphs, items, cnt + (size_t)p.G * p.nmax, p.items_max, hdr, table, lab, p.nmax, p.cap,
        p.classes, lab_bytes, buf_bytes, hist_bytes);
  else
    k_count<K, false><<<p.blocks, p.warps_per_block * 32, p.smem_bytes, s>>>(
        graphs, items, cnt + (size_t)p.G * p.nmax, p.items_max, hdr, table, lab, p.nmax, p.cap,
        p.classes, lab_bytes, buf_bytes, hist_bytes);
  return cudaGetLastError();
}

mt_status count_enqueue(const CountPlan& p, void* ws, const DevGraph* graphs,
                        const uint32_t* table, int32_t root_begin, int32_t root_end,
                        cudaStream_t s) {
  cudaError_t e;
  switch (p.K) {
    case 3: e = enqueue_k<3>(p, ws, graphs, table, root_begin, root_end, s); break;
    case 4: e = enqueue_k<4>(p, ws, graphs, table, root_begin, root_end, s); break;
    case 5: e = enqueue_k<5>(p, ws, graphs, table, root_begin, root_end, s); break;
    default: e = enqueue_k<6>(p, ws, graphs, table, root_begin, root_end, s); break;
  }
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MT_ENOMEM : MT_ECUDA;
  }
  return MT_OK;
}

// Plain one-graph count with the workspace cached in the graph handle.
static mt_status count_one(const mt_graph* gc, const mt_table* t, uint64_t* hist,
                           int32_t rb, int32_t re, double split_cost, int wpb, cudaStream_t s) {
  mt_graph* g = const_cast<mt_graph*>(gc);
  const int K = table_k(t);
  const uint32_t C = table_classes(t);
  CountPlan p;
  MT_TRY(count_configure(&p, K, 1, g->n, g->dmax, g->nu / 2 + 1, std::max(g->nu, 1), C,
                         split_cost, wpb));
  // workspace: plan scratch + the DevGraph + a device histogram
  const size_t extra = 256 + round16((size_t)C * 8);
  const size_t need = p.ws_bytes + extra;
  if (g->ws_bytes < need) {
    if (g->ws) {
      MT_CUDA_TRY(cudaStreamSynchronize(s));
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
  unsigned long long* dh =
      dev_hist ? (unsigned long long*)hist : (unsigned long long*)(base + p.ws_bytes + 256);
  DevGraph hg = dev_view(g, dh);
  MT_CUDA_TRY(cudaMemcpyAsync(dg, &hg, sizeof(DevGraph), cudaMemcpyHostToDevice, s));
  MT_CUDA_TRY(cudaMemsetAsync(dh, 0, (size_t)C * 8, s));
  if (g->n >= K && rb < re) {
    MT_CUDA_TRY(cudaEventRecord(g->ev0, s));
    MT_TRY(count_enqueue(p, g->ws, dg, table_device(t), rb, re, s));
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
    if (err) return MT_EOVERFLOW;
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
  return count_one(g, t, hist, root_begin, root_end, 0.0, 0, (cudaStream_t)stream);
}

mt_status mt_count(const mt_graph* g, const mt_table* t, uint64_t* hist, void* stream) {
  if (!g || !t || !hist) return MT_EINVAL;
  return count_one(g, t, hist, 0, g->n, 0.0, 0, (cudaStream_t)stream);
}

mt_status mt_count_tuned(const mt_graph* g, const mt_table* t, uint64_t* hist, double split_cost,
                         int warps_per_block, void* stream) {
  if (!g || !t || !hist || split_cost < 0 || warps_per_block < 0 || warps_per_block > 32)
    return MT_EINVAL;
  return count_one(g, t, hist, 0, g->n, split_cost, warps_per_block, (cudaStream_t)stream);
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
