// K1: the isomorphism table ISO of Sec. 3.2, built on the device.
//
// Keys are "extension-order keys": position p >= 1 of the enumerated vertex
// sequence owns the 2p bits starting at k(k-1) - p(p+1) (the last position
// lowest); inside them bits 2q / 2q+1 (q < p) say whether the arcs q->p /
// p->q exist.  For every key the builder
//  1. expands it to an 8x8 bit matrix (row i in byte i, column j in bit j),
//  2. walks all k! orderings of the vertices by adjacent transpositions
//     (Steinhaus-Johnson-Trotter order; each step swaps two neighbouring rows
//     and the same two columns) and keeps the numerically smallest matrix --
//     the order of the 8x8 values is the order of the canonical-layout masks,
//     because both lay the off-diagonal entries out row-major,
//  3. marks the key's own canonical-layout mask in a bitmap when it is its
//     own minimum and weakly connected.
// A popcount prefix over the bitmap then ranks the connected canonical masks
// (dense id = rank), and a last pass replaces each slot by the id of its
// canonical mask, or 0xFFFFFFFF for disconnected patterns.
#include <algorithm>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "trace.cuh"

struct mt_table {
  int k = 0;
  uint32_t classes = 0;
  uint64_t nkeys = 0;
  uint32_t* table = nullptr;        // device, nkeys
  uint32_t* class_masks = nullptr;  // device, classes
  // compact k = 6 form (see build_compact6): `table` holds the slots of
  // (prefix class, relabelled words) instead of one slot per key
  bool compact = false;
  uint16_t* xclass = nullptr;       // device, 4096: prefix key -> class of the first 4 vertices
  uint8_t* xmap = nullptr;          // device, 4096 x 256: prefix key -> word relabelling
};

namespace mt {

__constant__ uint8_t c_sjt[720];  // transposition positions p (swap p, p+1)

// Positions of the adjacent transpositions that take the identity through all
// k! permutations (Steinhaus-Johnson-Trotter with directions).
static std::vector<uint8_t> sjt_sequence(int k) {
  std::vector<int> perm(k), dir(k, -1);
  std::iota(perm.begin(), perm.end(), 0);
  std::vector<uint8_t> out;
  while (true) {
    int best = -1, bi = -1;
    for (int i = 0; i < k; ++i) {
      int j = i + dir[perm[i]];
      if (j < 0 || j >= k) continue;
      if (perm[j] < perm[i] && perm[i] > best) {
        best = perm[i];
        bi = i;
      }
    }
    if (bi < 0) break;
    int j = bi + dir[perm[bi]];
    out.push_back((uint8_t)std::min(bi, j));
    std::swap(perm[bi], perm[j]);
    for (int x = best + 1; x < k; ++x) dir[x] = -dir[x];
  }
  return out;
}

__device__ __forceinline__ uint64_t key_to_matrix(uint32_t key, int k) {
  uint64_t x = 0;
  for (int p = 1; p < k; ++p) {
    const int off = k * (k - 1) - p * (p + 1);
    for (int q = 0; q < p; ++q) {
      if ((key >> (off + 2 * q)) & 1u) x |= 1ull << (8 * q + p);      // q -> p
      if ((key >> (off + 2 * q + 1)) & 1u) x |= 1ull << (8 * p + q);  // p -> q
    }
  }
  return x;
}

__device__ __forceinline__ uint32_t matrix_to_mask(uint64_t x, int k) {
  uint32_t m = 0;
  for (int i = 0; i < k; ++i) {
    const uint32_t row = (uint32_t)(x >> (8 * i)) & 0xFFu;
    const uint32_t r = (row & ((1u << i) - 1u)) | ((row >> (i + 1)) << i);
    m |= r << (i * (k - 1));
  }
  return m;
}

__device__ __forceinline__ bool matrix_connected(uint64_t x, int k) {
  // undirected adjacency rows: a[i] = row i | column i
  uint32_t a[8];
  for (int i = 0; i < k; ++i) {
    uint32_t r = (uint32_t)(x >> (8 * i)) & 0xFFu;
    uint32_t c = 0;
    for (int j = 0; j < k; ++j) c |= (uint32_t)((x >> (8 * j + i)) & 1ull) << j;
    a[i] = r | c;
  }
  uint32_t seen = 1u, frontier = 1u;
  while (frontier) {
    uint32_t nxt = 0;
    for (int i = 0; i < k; ++i)
      if ((frontier >> i) & 1u) nxt |= a[i];
    nxt &= ~seen;
    seen |= nxt;
    frontier = nxt;
  }
  return seen == (1u << k) - 1u;
}

__device__ __forceinline__ uint64_t swap_adjacent(uint64_t x, int p) {
  // rows p and p+1 (bytes)
  uint64_t t = ((x >> (8 * p)) ^ (x >> (8 * p + 8))) & 0xFFull;
  x ^= (t << (8 * p)) | (t << (8 * p + 8));
  // columns p and p+1 (bits p, p+1 of every byte)
  t = ((x >> 1) ^ x) & (0x0101010101010101ull << p);
  x ^= t | (t << 1);
  return x;
}

template <int K>
__global__ void __launch_bounds__(256) k_canon(uint32_t* table, uint32_t* bitmap, uint64_t nkeys,
                                               int nsteps) {
  for (uint64_t key = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; key < nkeys;
       key += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x0 = key_to_matrix((uint32_t)key, K);
    uint64_t x = x0, best = x0;
    for (int s = 0; s < nsteps; ++s) {
      x = swap_adjacent(x, c_sjt[s]);
      best = x < best ? x : best;
    }
    const uint32_t canon = matrix_to_mask(best, K);
    table[key] = canon;
    if (best == x0 && matrix_connected(x0, K))
      atomicOr(&bitmap[canon >> 5], 1u << (canon & 31u));
  }
}

// prefix[w] = number of set bits in bitmap[0..w); tile sums first.
constexpr int kScanThreads = 256, kScanPer = 16, kScanTile = kScanThreads * kScanPer;

__global__ void k_tile_popc(const uint32_t* bitmap, size_t nwords, int32_t* tile_sum) {
  __shared__ int red[kScanThreads / 32];
  const size_t base = (size_t)blockIdx.x * kScanTile;
  int s = 0;
  for (int i = 0; i < kScanPer; ++i) {
    size_t w = base + (size_t)i * kScanThreads + threadIdx.x;
    if (w < nwords) s += __popc(bitmap[w]);
  }
  for (int d = 16; d; d >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int i = 0; i < kScanThreads / 32; ++i) t += red[i];
    tile_sum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_scan_single(int32_t* data, int count) {
  __shared__ int tmp[33];
  block_exclusive_scan(data, count, tmp);
}

__global__ void k_tile_prefix(const uint32_t* bitmap, size_t nwords, const int32_t* tile_off,
                              int32_t* prefix) {
  __shared__ int wsum[kScanThreads / 32 + 1];
  const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanPer;
  int loc[kScanPer];
  int s = 0;
  for (int i = 0; i < kScanPer; ++i) {
    const size_t w = base + i;
    loc[i] = s;
    s += w < nwords ? __popc(bitmap[w]) : 0;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int inc = warp_incl_scan(s);
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int i = 0; i < kScanThreads / 32; ++i) {
      int t = wsum[i];
      wsum[i] = acc;
      acc += t;
    }
  }
  __syncthreads();
  const int off = tile_off[blockIdx.x] + wsum[wid] + inc - s;
  for (int i = 0; i < kScanPer; ++i) {
    const size_t w = base + i;
    if (w < nwords) prefix[w] = off + loc[i];
  }
}

__global__ void k_assign(uint32_t* table, uint64_t nkeys, const uint32_t* bitmap,
                         const int32_t* prefix) {
  for (uint64_t key = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; key < nkeys;
       key += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = table[key];
    const uint32_t w = bitmap[c >> 5];
    const uint32_t bit = 1u << (c & 31u);
    table[key] = (w & bit) ? (uint32_t)prefix[c >> 5] + __popc(w & (bit - 1u)) : kNoClass;
  }
}

__global__ void k_class_list(const uint32_t* bitmap, size_t nwords, const int32_t* prefix,
                             uint32_t* out, uint32_t classes) {
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < nwords;
       w += (size_t)gridDim.x * blockDim.x) {
    uint32_t bits = bitmap[w];
    int r = prefix[w];
    while (bits) {
      const int b = __ffs(bits) - 1;
      if ((uint32_t)r < classes) out[r] = (uint32_t)(w * 32 + b);
      ++r;
      bits &= bits - 1u;
    }
  }
}

static mt_status build_table(int k, cudaStream_t s, mt_table** out) {
  const uint64_t nkeys = 1ull << (k * (k - 1));
  const size_t nwords = (size_t)std::max<uint64_t>(nkeys / 32, 1);
  std::vector<uint8_t> seq = sjt_sequence(k);
  {  // the walk must visit every ordering exactly once
    std::vector<int> p(k);
    std::iota(p.begin(), p.end(), 0);
    std::vector<std::vector<int>> seen{p};
    for (uint8_t q : seq) {
      std::swap(p[q], p[q + 1]);
      seen.push_back(p);
    }
    std::sort(seen.begin(), seen.end());
    size_t fact = 1;
    for (int i = 2; i <= k; ++i) fact *= i;
    if (seq.size() + 1 != fact || std::unique(seen.begin(), seen.end()) != seen.end())
      return MT_ECUDA;
  }
  MT_CUDA_TRY(cudaMemcpyToSymbolAsync(c_sjt, seq.data(), seq.size(), 0, cudaMemcpyHostToDevice, s));

  mt_table* t = new mt_table();
  t->k = k;
  t->nkeys = nkeys;
  t->classes = kNumClasses[k];
  uint32_t* bitmap = nullptr;
  int32_t* prefix = nullptr;
  int32_t* tiles = nullptr;
  const size_t ntiles = (nwords + kScanTile - 1) / kScanTile;
  cudaError_t e = cudaMalloc(&t->table, nkeys * 4);
  if (e == cudaSuccess) e = cudaMalloc(&t->class_masks, (size_t)t->classes * 4);
  if (e == cudaSuccess) e = cudaMallocAsync(&bitmap, nwords * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&prefix, nwords * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&tiles, ntiles * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bitmap, 0, nwords * 4, s);
  if (e == cudaSuccess) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<uint64_t>((nkeys + 255) / 256, (uint64_t)sms * 16);
    const int nsteps = (int)seq.size();
    switch (k) {
      case 3: k_canon<3><<<grid, 256, 0, s>>>(t->table, bitmap, nkeys, nsteps); break;
      case 4: k_canon<4><<<grid, 256, 0, s>>>(t->table, bitmap, nkeys, nsteps); break;
      case 5: k_canon<5><<<grid, 256, 0, s>>>(t->table, bitmap, nkeys, nsteps); break;
      default: k_canon<6><<<grid, 256, 0, s>>>(t->table, bitmap, nkeys, nsteps); break;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      k_tile_popc<<<(unsigned)ntiles, kScanThreads, 0, s>>>(bitmap, nwords, tiles);
      k_scan_single<<<1, 1024, 0, s>>>(tiles, (int)ntiles);
      k_tile_prefix<<<(unsigned)ntiles, kScanThreads, 0, s>>>(bitmap, nwords, tiles, prefix);
      k_assign<<<grid, 256, 0, s>>>(t->table, nkeys, bitmap, prefix);
      const int g2 = (int)std::min<size_t>((nwords + 255) / 256, (size_t)sms * 8);
      k_class_list<<<g2, 256, 0, s>>>(bitmap, nwords, prefix, t->class_masks, t->classes);
      e = cudaGetLastError();
    }
  }
  // the number of connected canonical masks must equal the closed-form count
  int32_t last_prefix = 0;
  uint32_t last_word = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&last_prefix, prefix + nwords - 1, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&last_word, bitmap + nwords - 1, 4, cudaMemcpyDeviceToHost, s);
  if (bitmap) cudaFreeAsync(bitmap, s);
  if (prefix) cudaFreeAsync(prefix, s);
  if (tiles) cudaFreeAsync(tiles, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    if (t->table) cudaFree(t->table);
    if (t->class_masks) cudaFree(t->class_masks);
    delete t;
    return e == cudaErrorMemoryAllocation ? MT_ENOMEM : MT_ECUDA;
  }
  const uint32_t found = (uint32_t)last_prefix + (uint32_t)__builtin_popcount(last_word);
  if (found != t->classes) {
    set_last_error("table builder found " + std::to_string(found) + " classes");
    cudaFree(t->table);
    cudaFree(t->class_masks);
    delete t;
    return MT_ECUDA;
  }
  *out = t;
  return MT_OK;
}

// ---------------------------------------------------------- compact k = 6 form
//
// The k = 6 table has 2^30 slots (4 GiB), but a key is three parts: the first
// four vertices X (positions 0..3, 12 key bits), the fifth vertex's word y (8
// bits) and the sixth's z (10 bits).  Relabelling X into a canonical order of
// its own (one of the 199 weakly connected 4-vertex classes; X is connected in
// every enumerated set) and the words with it leaves the class of the whole
// unchanged, so a table indexed by (class of X, relabelled y, relabelled z)
// holds every class: 199 x 2^18 slots (208 MB).  Per prefix key it needs the
// class of X and the relabelling of an 8-bit word (4 two-bit fields, one per
// vertex of X); the sixth vertex's field for the fifth vertex is not moved.

constexpr int kXKeys = 1 << 12;          // prefix keys (positions 1..3 of a 6-vertex key)
constexpr int kXClasses = 199;           // weakly connected 4-vertex classes
constexpr int kXLow = 18;                // bits of y and z in a 6-vertex key

// The 4-vertex prefix of a 6-vertex key, as an 8x8 bit matrix.
__device__ __forceinline__ uint64_t xkey_matrix(uint32_t xk) { return key_to_matrix(xk << kXLow, 6); }

// For every prefix key: the smallest 4-vertex canonical-layout mask over the 24
// orderings sigma (new position i holds old vertex sigma(i)), the ordering that
// reaches it, and whether X is weakly connected.  Marks the connected minima.
__global__ void k_xprefix(uint16_t* xcanon, uint8_t* xsigma, uint32_t* xbits, int32_t* xrep) {
  const int xk = blockIdx.x * blockDim.x + threadIdx.x;
  if (xk >= kXKeys) return;
  const uint64_t x0 = xkey_matrix((uint32_t)xk);
  uint32_t best = 0xFFFFFFFFu, best_sigma = 0;
  for (int c = 0; c < 24; ++c) {
    // the c-th ordering of 4 vertices (factorial number system)
    int avail[4] = {0, 1, 2, 3}, sig[4];
    int r = c;
    for (int i = 0, f = 6; i < 4; ++i) {
      const int d = r / f;
      r %= f;
      sig[i] = avail[d];
      for (int j = d; j < 3 - i; ++j) avail[j] = avail[j + 1];
      f = i < 3 ? f / (3 - i) : 1;
    }
    uint64_t y = 0;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        if ((x0 >> (8 * sig[i] + sig[j])) & 1ull) y |= 1ull << (8 * i + j);
    const uint32_t mask = matrix_to_mask(y, 4);
    if (mask < best) {
      best = mask;
      best_sigma = (uint32_t)(sig[0] | (sig[1] << 2) | (sig[2] << 4) | (sig[3] << 6));
    }
  }
  xcanon[xk] = (uint16_t)best;
  xsigma[xk] = (uint8_t)best_sigma;
  const bool conn = matrix_connected(x0, 4);
  if (conn) atomicOr(&xbits[best >> 5], 1u << (best & 31u));
  // the prefix key whose own matrix is the canonical one represents the class
  if (conn && matrix_to_mask(x0, 4) == best) xrep[best] = xk;
}

// Class of each prefix key (rank of its canonical mask among the connected
// ones; 0xFFFF if X is disconnected) and the relabelling of all 256 words.
__global__ void k_xtables(const uint16_t* xcanon, const uint8_t* xsigma, const uint32_t* xbits,
                          uint16_t* xclass, uint8_t* xmap) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kXKeys * 256) return;
  const int xk = t >> 8, w = t & 255;
  const uint32_t sg = xsigma[xk];
  uint32_t out = 0;
  for (int i = 0; i < 4; ++i) out |= ((w >> (2 * ((sg >> (2 * i)) & 3u))) & 3u) << (2 * i);
  xmap[t] = (uint8_t)out;
  if (w == 0) {
    const uint32_t c = xcanon[xk];
    const bool conn = matrix_connected(xkey_matrix((uint32_t)xk), 4);
    uint32_t rank = 0;
    for (uint32_t q = 0; q < (c >> 5); ++q) rank += __popc(xbits[q]);
    rank += __popc(xbits[c >> 5] & ((1u << (c & 31u)) - 1u));
    xclass[xk] = conn ? (uint16_t)rank : (uint16_t)0xFFFFu;
  }
}

// Representative prefix key of each class, in class order.
__global__ void k_xreps(const uint32_t* xbits, const int32_t* xrep, int32_t* reps) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int r = 0;
  for (uint32_t c = 0; c < kXKeys && r < kXClasses; ++c)
    if ((xbits[c >> 5] >> (c & 31u)) & 1u) reps[r++] = xrep[c];
}

// compact[c << 18 | low] = full[rep(c) << 18 | low]
__global__ void k_xgather(const uint32_t* full, const int32_t* reps, uint32_t* compact) {
  const uint64_t n = (uint64_t)kXClasses << kXLow;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = (uint32_t)(i >> kXLow), low = (uint32_t)(i & ((1u << kXLow) - 1u));
    compact[i] = full[((uint64_t)reps[c] << kXLow) | low];
  }
}

static mt_status build_compact6(cudaStream_t s, mt_table** out) {
  mt_table* full = nullptr;
  MT_TRY(build_table(6, s, &full));
  mt_table* t = new mt_table();
  t->k = 6;
  t->classes = full->classes;
  t->class_masks = full->class_masks;
  full->class_masks = nullptr;
  t->compact = true;
  t->nkeys = (uint64_t)kXClasses << kXLow;
  uint16_t* xcanon = nullptr;
  uint8_t* xsigma = nullptr;
  uint32_t* xbits = nullptr;
  int32_t *xrep = nullptr, *reps = nullptr;
  cudaError_t e = cudaMalloc(&t->table, t->nkeys * 4);
  if (e == cudaSuccess) e = cudaMalloc(&t->xclass, kXKeys * 2);
  if (e == cudaSuccess) e = cudaMalloc(&t->xmap, kXKeys * 256);
  if (e == cudaSuccess) e = cudaMallocAsync(&xcanon, kXKeys * 2, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&xsigma, kXKeys, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&xbits, kXKeys / 8, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&xrep, kXKeys * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&reps, kXClasses * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(xbits, 0, kXKeys / 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(reps, 0, kXClasses * 4, s);
  int32_t nreps = 0;
  if (e == cudaSuccess) {
    k_xprefix<<<kXKeys / 256, 256, 0, s>>>(xcanon, xsigma, xbits, xrep);
    k_xtables<<<kXKeys, 256, 0, s>>>(xcanon, xsigma, xbits, t->xclass, t->xmap);
    k_xreps<<<1, 32, 0, s>>>(xbits, xrep, reps);
    k_xgather<<<1024, 256, 0, s>>>(full->table, reps, t->table);
    e = cudaGetLastError();
  }
  // the number of connected 4-vertex classes must be 199
  std::vector<uint32_t> hb(kXKeys / 32);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hb.data(), xbits, kXKeys / 8, cudaMemcpyDeviceToHost, s);
  if (xcanon) cudaFreeAsync(xcanon, s);
  if (xsigma) cudaFreeAsync(xsigma, s);
  if (xbits) cudaFreeAsync(xbits, s);
  if (xrep) cudaFreeAsync(xrep, s);
  if (reps) cudaFreeAsync(reps, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (uint32_t w : hb) nreps += __builtin_popcount(w);
  cudaFree(full->table);
  delete full;
  if (e != cudaSuccess || nreps != kXClasses) {
    if (e != cudaSuccess) set_last_error(cudaGetErrorString(e));
    else set_last_error("compact table: " + std::to_string(nreps) + " prefix classes");
    cudaFree(t->table);
    cudaFree(t->class_masks);
    cudaFree(t->xclass);
    cudaFree(t->xmap);
    delete t;
    return e == cudaErrorMemoryAllocation ? MT_ENOMEM : MT_ECUDA;
  }
  *out = t;
  return MT_OK;
}

TableView table_view(const mt_table* t) {
  TableView v;
  v.slots = t->table;
  v.xclass = t->compact ? t->xclass : nullptr;
  v.xmap = t->compact ? t->xmap : nullptr;
  return v;
}
bool table_compact(const mt_table* t) { return t->compact; }

const uint32_t* table_device(const mt_table* t) { return t->table; }
int table_k(const mt_table* t) { return t->k; }
uint32_t table_classes(const mt_table* t) { return t->classes; }

}  // namespace mt

using namespace mt;

extern "C" {

mt_status mt_table_build(int k, void* stream, mt_table** out) {
  if (!out) return MT_EINVAL;
  if (k < 3 || k > 6) return MT_EUNSUPPORTED;
  TraceRange tr("mt_table_build");
  return build_table(k, (cudaStream_t)stream, out);
}

mt_status mt_table_build_compact(int k, void* stream, mt_table** out) {
  if (!out) return MT_EINVAL;
  if (k != 6) return MT_EUNSUPPORTED;
  TraceRange tr("mt_table_build_compact");
  return build_compact6((cudaStream_t)stream, out);
}

mt_status mt_table_is_compact(const mt_table* t, int* compact) {
  if (!t || !compact) return MT_EINVAL;
  *compact = t->compact ? 1 : 0;
  return MT_OK;
}

mt_status mt_table_free(mt_table* t) {
  if (!t) return MT_OK;
  cudaDeviceSynchronize();
  cudaFree(t->table);
  cudaFree(t->class_masks);
  if (t->xclass) cudaFree(t->xclass);
  if (t->xmap) cudaFree(t->xmap);
  delete t;
  return MT_OK;
}

mt_status mt_table_k(const mt_table* t, int* k) {
  if (!t || !k) return MT_EINVAL;
  *k = t->k;
  return MT_OK;
}

mt_status mt_table_num_classes(const mt_table* t, uint32_t* out) {
  if (!t || !out) return MT_EINVAL;
  *out = t->classes;
  return MT_OK;
}

mt_status mt_table_class_masks(const mt_table* t, uint32_t* masks) {
  if (!t || !masks) return MT_EINVAL;
  MT_CUDA_TRY(cudaMemcpy(masks, t->class_masks, (size_t)t->classes * 4, cudaMemcpyDeviceToHost));
  return MT_OK;
}

mt_status mt_table_entries(const mt_table* t, uint64_t first, uint64_t count, uint32_t* ids) {
  if (!t || (!ids && count)) return MT_EINVAL;
  if (first > t->nkeys || count > t->nkeys - first) return MT_EINVAL;
  if (count == 0) return MT_OK;
  MT_CUDA_TRY(cudaMemcpy(ids, t->table + first, count * 4, cudaMemcpyDeviceToHost));
  return MT_OK;
}

}  // extern "C"
