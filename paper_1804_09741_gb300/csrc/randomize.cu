// K3: degree-preserving directed arc swaps (the null model of Sec. 1, step (c);
// the paper names no randomisation model, the reading is the switch of Milo et
// al.).  Attempts run in order, exactly as the sequential definition:
//   attempt t draws arc positions e1 = floor(r1 m / 2^64), e2 = floor(r2 m / 2^64)
//   with r1, r2 = SplitMix64 outputs 2t and 2t+1 of the graph's seed; arcs
//   (a->b) at e1 and (c->d) at e2 become (a->d), (c->b) unless e1 == e2, a == c,
//   b == d, a == d, c == b, or (a->d) or (c->b) is already an arc.
// A swap keeps the source of each position, so the out-CSR shape is unchanged:
// only the destinations move, and the builder re-sorts the rows afterwards.
//
// GPU mapping: one thread block per graph.  The arc array (src<<16 | dst) and an
// open-addressing hash set of the present arcs sit in shared memory; the block
// fills them in parallel; warp 0 draws the positions of 32 attempts at a time
// and one lane applies them in order.  Many graphs run side by side (the
// null-model batch).
//
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014, public-domain reference
// generator): state advances by the golden gamma 0x9E3779B97F4A7C15, output =
// mix(state) with the variant-13 mix; output i of seed s is mix(s + (i+1)*gamma).
#include "graph.cuh"
#include "trace.cuh"

namespace mt {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t hslot(uint32_t key, int bits) {
  return (key * 0x9E3779B1u) >> (32 - bits);
}

struct HashSet {
  uint32_t* t;
  int bits;
  uint32_t mask;
  __device__ int find(uint32_t key) const {
    uint32_t i = hslot(key, bits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      const uint32_t x = t[i];
      if (x == key) return (int)i;
      if (x == kEmpty) return -1;
      i = (i + 1) & mask;
    }
    return -1;
  }
  __device__ void insert(uint32_t key) const {
    uint32_t i = hslot(key, bits);
    while (t[i] != kEmpty) i = (i + 1) & mask;
    t[i] = key;
  }
  // Remove the entry at slot i, shifting later members of its probe run back
  // (deletion without tombstones for linear probing).
  __device__ void erase_slot(uint32_t i) const {
    uint32_t j = i;
    while (true) {
      j = (j + 1) & mask;
      const uint32_t x = t[j];
      if (x == kEmpty) break;
      const uint32_t home = hslot(x, bits);
      const bool stays = (i <= j) ? (i < home && home <= j) : (i < home || home <= j);
      if (!stays) {
        t[i] = x;
        i = j;
      }
    }
    t[i] = kEmpty;
  }
};

struct RandArgs {
  int32_t n, m, G, bits;
  const int32_t* row_ptr;  // shared out-CSR shape
  const int32_t* col0;     // destinations of the source graph (CSR order)
  const uint64_t* seeds;   // G seeds
  uint64_t swaps;
  int32_t* col_out;        // G x m destinations after the swaps (rows unsorted)
  uint32_t* gscratch;      // used when the arrays do not fit shared memory
  int use_smem;
  int64_t* accepted;       // G counters (may be null)
};

__global__ void __launch_bounds__(512) k_randomize(RandArgs a) {
  extern __shared__ __align__(16) uint32_t rsm[];
  const int g = blockIdx.x;
  const int m = a.m, n = a.n;
  const uint32_t tsize = 1u << a.bits;
  uint32_t* arcs = a.use_smem ? rsm : a.gscratch + (size_t)g * (m + tsize);
  HashSet hs{arcs + m, a.bits, tsize - 1u};
  for (uint32_t i = threadIdx.x; i < tsize; i += blockDim.x) hs.t[i] = kEmpty;
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
    }
    arcs[e] = ((uint32_t)lo << 16) | (uint32_t)a.col0[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    const uint32_t key = arcs[e];
    uint32_t i = hslot(key, a.bits);
    while (atomicCAS(&hs.t[i], kEmpty, key) != kEmpty) i = (i + 1) & hs.mask;
  }
  __syncthreads();
  // Warp 0: the 32 lanes draw the arc positions of the next 32 attempts (the
  // SplitMix64 outputs do not depend on the graph), then lane 0 applies those
  // attempts in order.
  __shared__ uint32_t s_e[64];
  if (threadIdx.x < 32 && m > 0) {
    const int lane = threadIdx.x;
    const uint64_t seed = a.seeds[g];
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    int64_t acc = 0;
    for (uint64_t t0 = 0; t0 < a.swaps; t0 += 32) {
      const uint64_t t = t0 + lane;
      s_e[lane] = (uint32_t)__umul64hi(sm64_mix(seed + (2 * t + 1) * gamma), (uint64_t)m);
      s_e[32 + lane] = (uint32_t)__umul64hi(sm64_mix(seed + (2 * t + 2) * gamma), (uint64_t)m);
      __syncwarp();
      if (lane == 0) {
        const int cnt = (int)((a.swaps - t0) < 32 ? (a.swaps - t0) : 32);
        for (int j = 0; j < cnt; ++j) {
          const uint32_t e1 = s_e[j], e2 = s_e[32 + j];
          if (e1 == e2) continue;
          const uint32_t A = arcs[e1], B = arcs[e2];
          const uint32_t sa = A >> 16, da = A & 0xFFFFu, sc = B >> 16, dc = B & 0xFFFFu;
          if (sa == sc || da == dc || sa == dc || sc == da) continue;
          const uint32_t n1 = (sa << 16) | dc, n2 = (sc << 16) | da;
          if (hs.find(n1) >= 0 || hs.find(n2) >= 0) continue;
          hs.erase_slot((uint32_t)hs.find(A));
          hs.erase_slot((uint32_t)hs.find(B));
          hs.insert(n1);
          hs.insert(n2);
          arcs[e1] = n1;
          arcs[e2] = n2;
          ++acc;
        }
      }
      __syncwarp();
    }
    if (lane == 0 && a.accepted) a.accepted[g] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m; e += blockDim.x)
    a.col_out[(size_t)g * m + e] = (int32_t)(arcs[e] & 0xFFFFu);
}

// Dyad-preserving variant (swap mutual pairs and one-way arcs separately; the
// reading of the null model that keeps reciprocity): the arcs are split, in CSR
// order, into singles (u->v without v->u) and mutual dyads {u,v} (listed once,
// from the smaller end).  Attempt t takes SplitMix64 outputs 3t, 3t+1, 3t+2:
// the first picks the list (singles if floor(r*(S+D)/2^64) < S), the other two
// pick two entries; (a,b), (c,d) become (a,d), (c,b) unless the entries
// coincide, a == c, b == d, a == d, c == b, or a new pair is already adjacent in
// either direction.  The set holds the unordered adjacent pairs (min<<16|max).
struct DyadArgs {
  int32_t n, m, G, bits;
  const int32_t* row_ptr;  // shared out-CSR shape (sorted rows)
  const int32_t* col0;
  const uint64_t* seeds;
  uint64_t attempts;
  int32_t* col_out;        // G x m destinations, rows unsorted
  int32_t* scratch;        // G x (2m + n + 2) ints
  int64_t* accepted;
};

__device__ __forceinline__ bool has_arc(const int32_t* row_ptr, const int32_t* col, int a, int b) {
  int lo = row_ptr[a], hi = row_ptr[a + 1];
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int x = col[mid];
    if (x == b) return true;
    if (x < b) lo = mid + 1; else hi = mid;
  }
  return false;
}

__global__ void __launch_bounds__(512) k_randomize_dyads(DyadArgs a) {
  extern __shared__ __align__(16) uint32_t dsm[];
  __shared__ int scan_tmp[33];
  const int g = blockIdx.x;
  const int m = a.m, n = a.n;
  const uint32_t tsize = 1u << a.bits;
  uint32_t* lists = dsm;  // singles [0, S), dyads [S, S + D)
  HashSet hs{dsm + m, a.bits, tsize - 1u};
  int32_t* fs = a.scratch + (size_t)g * (2 * (size_t)m + n + 2);
  int32_t* fd = fs + m + 1;
  int32_t* cur = fd + m + 1;
  for (uint32_t i = threadIdx.x; i < tsize; i += blockDim.x) hs.t[i] = kEmpty;
  for (int v = threadIdx.x; v < n; v += blockDim.x) cur[v] = 0;
  // kinds of the arcs, in CSR order
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const int v = lo, u = a.col0[e];
    const bool rev = has_arc(a.row_ptr, a.col0, u, v);
    fs[e] = rev ? 0 : 1;
    fd[e] = (rev && v < u) ? 1 : 0;
  }
  if (threadIdx.x == 0) {
    fs[m] = 0;
    fd[m] = 0;
  }
  __syncthreads();
  const int S = (int)block_exclusive_scan(fs, m + 1, scan_tmp);
  const int D = (int)block_exclusive_scan(fd, m + 1, scan_tmp);
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    const bool single = fs[e + 1] != fs[e];
    const bool dyad = fd[e + 1] != fd[e];
    if (single || dyad) {
      int lo = 0, hi = n - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
      }
      const uint32_t v = (uint32_t)lo, u = (uint32_t)a.col0[e];
      const uint32_t pk = v < u ? (v << 16) | u : (u << 16) | v;
      if (single) lists[fs[e]] = (v << 16) | u;
      else lists[S + fd[e]] = (v << 16) | u;
      uint32_t i = hslot(pk, a.bits);
      while (atomicCAS(&hs.t[i], kEmpty, pk) != kEmpty) i = (i + 1) & hs.mask;
    }
  }
  __syncthreads();
  __shared__ uint32_t s_r[96];
  if (threadIdx.x < 32 && S + D > 0) {
    const int lane = threadIdx.x;
    const uint64_t seed = a.seeds[g];
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    const uint64_t tot = (uint64_t)S + (uint64_t)D;
    int64_t acc = 0;
    for (uint64_t t0 = 0; t0 < a.attempts; t0 += 32) {
      const uint64_t t = t0 + lane;
      const uint64_t r0 = sm64_mix(seed + (3 * t + 1) * gamma);
      const uint64_t r1 = sm64_mix(seed + (3 * t + 2) * gamma);
      const uint64_t r2 = sm64_mix(seed + (3 * t + 3) * gamma);
      const bool single = __umul64hi(r0, tot) < (uint64_t)S;
      const uint64_t len = single ? (uint64_t)S : (uint64_t)D;
      s_r[lane] = single ? 1u : 0u;
      s_r[32 + lane] = (uint32_t)__umul64hi(r1, len);
      s_r[64 + lane] = (uint32_t)__umul64hi(r2, len);
      __syncwarp();
      if (lane == 0) {
        const int cnt = (int)((a.attempts - t0) < 32 ? (a.attempts - t0) : 32);
        for (int j = 0; j < cnt; ++j) {
          const uint32_t base = s_r[j] ? 0u : (uint32_t)S;
          const uint32_t e1 = base + s_r[32 + j], e2 = base + s_r[64 + j];
          if (e1 == e2) continue;
          const uint32_t A = lists[e1], B = lists[e2];
          const uint32_t pa = A >> 16, pb = A & 0xFFFFu, pc = B >> 16, pd = B & 0xFFFFu;
          if (pa == pc || pb == pd || pa == pd || pc == pb) continue;
          const uint32_t k1 = pa < pd ? (pa << 16) | pd : (pd << 16) | pa;
          const uint32_t k2 = pc < pb ? (pc << 16) | pb : (pb << 16) | pc;
          if (hs.find(k1) >= 0 || hs.find(k2) >= 0) continue;
          const uint32_t o1 = pa < pb ? (pa << 16) | pb : (pb << 16) | pa;
          const uint32_t o2 = pc < pd ? (pc << 16) | pd : (pd << 16) | pc;
          hs.erase_slot((uint32_t)hs.find(o1));
          hs.erase_slot((uint32_t)hs.find(o2));
          hs.insert(k1);
          hs.insert(k2);
          lists[e1] = (pa << 16) | pd;
          lists[e2] = (pc << 16) | pb;
          ++acc;
        }
      }
      __syncwarp();
    }
    if (lane == 0 && a.accepted) a.accepted[g] = acc;
  }
  __syncthreads();
  // arcs back into the rows of the fixed out-CSR shape (order inside a row is
  // arbitrary; the builder sorts)
  int32_t* out = a.col_out + (size_t)g * m;
  for (int i = threadIdx.x; i < S + D; i += blockDim.x) {
    const uint32_t x = lists[i];
    const int u = (int)(x >> 16), v = (int)(x & 0xFFFFu);
    out[a.row_ptr[u] + atomicAdd(&cur[u], 1)] = v;
    if (i >= S) out[a.row_ptr[v] + atomicAdd(&cur[v], 1)] = u;
  }
}

size_t dyad_scratch_ints(int32_t n, int32_t m) { return 2 * (size_t)m + (size_t)n + 2; }

int hash_bits_for(int32_t m);
size_t rand_smem_bytes(int32_t m);

cudaError_t launch_randomize_dyads(int32_t n, int32_t m, int G, const int32_t* row_ptr,
                                   const int32_t* col0, const uint64_t* seeds, uint64_t attempts,
                                   int32_t* col_out, int32_t* scratch, int64_t* accepted,
                                   cudaStream_t s) {
  DyadArgs a;
  a.n = n; a.m = m; a.G = G; a.bits = hash_bits_for(m);
  a.row_ptr = row_ptr; a.col0 = col0; a.seeds = seeds; a.attempts = attempts;
  a.col_out = col_out; a.scratch = scratch; a.accepted = accepted;
  const size_t bytes = rand_smem_bytes(m);
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (bytes > (size_t)max_smem - 2048) return cudaErrorInvalidValue;
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_randomize_dyads,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  k_randomize_dyads<<<G, 512, bytes, s>>>(a);
  return cudaGetLastError();
}

int hash_bits_for(int32_t m) {
  int bits = 4;
  while ((1ll << bits) < 2ll * (m > 0 ? m : 1)) ++bits;
  return bits;  // table of at least 2m slots: load factor <= 1/2
}

size_t rand_smem_bytes(int32_t m) {
  return ((size_t)m + ((size_t)1 << hash_bits_for(m))) * 4;
}

// Enqueue G randomisations of the graph (row_ptr, col0) into col_out.
cudaError_t launch_randomize(int32_t n, int32_t m, int G, const int32_t* row_ptr,
                             const int32_t* col0, const uint64_t* seeds, uint64_t swaps,
                             int32_t* col_out, uint32_t* gscratch, int64_t* accepted,
                             cudaStream_t s) {
  RandArgs a;
  a.n = n; a.m = m; a.G = G; a.bits = hash_bits_for(m);
  a.row_ptr = row_ptr; a.col0 = col0; a.seeds = seeds; a.swaps = swaps;
  a.col_out = col_out; a.gscratch = gscratch; a.accepted = accepted;
  const size_t bytes = rand_smem_bytes(m);
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  a.use_smem = bytes <= (size_t)max_smem - 1024 ? 1 : 0;
  if (!a.use_smem && !gscratch) return cudaErrorInvalidValue;
  const size_t smem = a.use_smem ? bytes : 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_randomize, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_randomize<<<G, 512, smem, s>>>(a);
  return cudaGetLastError();
}

// Scratch (uint32 words) needed by launch_randomize when shared memory is too small.
size_t rand_gscratch_words(int32_t m, int G) {
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (rand_smem_bytes(m) <= (size_t)max_smem - 1024) return 0;
  return (size_t)G * ((size_t)m + ((size_t)1 << hash_bits_for(m)));
}

mt_status graph_alloc(int32_t n, int32_t m, mt_graph** out);
mt_status graph_build_sync(mt_graph* g, const int32_t* col_in, cudaStream_t s);

}  // namespace mt

using namespace mt;

extern "C" {

mt_status mt_randomize(const mt_graph* src, uint64_t seed, uint64_t swaps, void* stream,
                       mt_graph** out) {
  if (!src || !out) return MT_EINVAL;
  TraceRange tr("mt_randomize");
  cudaStream_t s = (cudaStream_t)stream;
  mt_graph* g = nullptr;
  MT_TRY(graph_alloc(src->n, src->m, &g));
  const size_t m1 = (size_t)(src->m > 0 ? src->m : 1);
  const size_t gwords = rand_gscratch_words(src->m, 1);
  char* scratch = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&scratch, m1 * 4 + 16 + gwords * 4 + 16, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->row_ptr, src->row_ptr, (size_t)(src->n + 1) * 4,
                        cudaMemcpyDeviceToDevice, s);
  int32_t* col_tmp = (int32_t*)scratch;
  uint64_t* d_seed = (uint64_t*)(scratch + ((m1 * 4 + 15) & ~(size_t)15));
  uint32_t* gscr = gwords ? (uint32_t*)((char*)d_seed + 16) : nullptr;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_seed, &seed, 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_randomize(src->n, src->m, 1, src->row_ptr, src->col, d_seed, swaps, col_tmp, gscr,
                         nullptr, s);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    if (scratch) cudaFreeAsync(scratch, s);
    mt_graph_free(g);
    return MT_ECUDA;
  }
  mt_status st = graph_build_sync(g, col_tmp, s);
  cudaFreeAsync(scratch, s);
  if (st != MT_OK) {
    mt_graph_free(g);
    return st;
  }
  *out = g;
  return MT_OK;
}

mt_status mt_randomize_dyads(const mt_graph* src, uint64_t seed, uint64_t attempts, void* stream,
                             mt_graph** out) {
  if (!src || !out) return MT_EINVAL;
  TraceRange tr("mt_randomize_dyads");
  cudaStream_t s = (cudaStream_t)stream;
  if (rand_smem_bytes(src->m) > 200 * 1024) return MT_EUNSUPPORTED;
  mt_graph* g = nullptr;
  MT_TRY(graph_alloc(src->n, src->m, &g));
  const size_t m1 = (size_t)(src->m > 0 ? src->m : 1);
  const size_t sc = dyad_scratch_ints(src->n, src->m);
  char* scratch = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&scratch, (m1 + sc) * 4 + 64, s);
  int32_t* col_tmp = (int32_t*)scratch;
  int32_t* dsc = col_tmp + m1;
  uint64_t* d_seed = (uint64_t*)(((uintptr_t)(dsc + sc) + 15) & ~(uintptr_t)15);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->row_ptr, src->row_ptr, (size_t)(src->n + 1) * 4,
                        cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_seed, &seed, 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_randomize_dyads(src->n, src->m, 1, src->row_ptr, src->col, d_seed, attempts,
                               col_tmp, dsc, nullptr, s);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    if (scratch) cudaFreeAsync(scratch, s);
    mt_graph_free(g);
    return MT_ECUDA;
  }
  mt_status st = graph_build_sync(g, col_tmp, s);
  cudaFreeAsync(scratch, s);
  if (st != MT_OK) {
    mt_graph_free(g);
    return st;
  }
  *out = g;
  return MT_OK;
}

}  // extern "C"
