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
// GPU mapping: one thread block per graph.  The arc array (src<<16 | dst) and a
// bucketed hash set of the present arcs sit in shared memory (global memory
// for graphs too large for it); the block fills them in parallel.  Then warp
// 0 runs the attempts 32 at a time, lane j taking attempt t0 + j:
//  * speculation: every lane evaluates its attempt against the state at the
//    start of the batch (the two arcs at its positions, the checks, whether
//    the two new arcs are present, where the two old ones and free slots for
//    the new ones are);
//  * resolution: an attempt's speculative outcome is its sequential outcome
//    unless an earlier attempt of the batch that the speculation accepted
//    wrote one of its two positions, inserted or erased one of the two arcs it
//    looks up, or would fill the same free slot (a new key takes the first free
//    slot of its bucket at or after one picked by the key's low bits, so
//    attempts sharing a bucket rarely pick the same).  Every lane checks this
//    against all earlier lanes at once; the attempts before the first unsafe
//    one are applied together (their writes are disjoint), the unsafe one is
//    evaluated on the current state by the whole warp, which looks up its four
//    arcs in one round of shared-memory loads (eight lanes per arc read its
//    32-slot bucket, a ballot finds the key or a free slot), and the next
//    batch starts after it.  The outcome is that of the attempts run one after
//    another.
//
// Bucketed set: 2^bb buckets of 32 slots (at least 2 slots per stored key,
// so a bucket holds 16 on average); a key lives in the first bucket of its
// probe sequence (home bucket, then the next ones) that had a free slot when it
// was inserted, and a bucket that was ever found full keeps a sticky
// "overflowed" flag, so a lookup moves on to the next bucket only past flagged
// ones.  Erasing empties the slot; flags stay.  Only membership matters to the
// attempts, not where a key is stored, so the results are those of the
// sequential definition.
//
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014, public-domain reference
// generator): state advances by the golden gamma 0x9E3779B97F4A7C15, output =
// mix(state) with the variant-13 mix; output i of seed s is mix(s + (i+1)*gamma).
#include "graph.cuh"
#include "trace.cuh"

namespace mt {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr unsigned kWarp = 0xFFFFFFFFu;

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Layout of one graph's randomiser state (in 32-bit words): the entry array
// (arcs, or the dyad lists) padded to 4 words, the buckets, the overflow flags.
struct RandLayout {
  int bb;          // log2 of the number of buckets (>= 1)
  size_t t_off;    // first slot
  size_t f_off;    // first flag word
  size_t words;    // total
};

__host__ __device__ inline RandLayout rand_layout(int32_t m) {
  RandLayout L;
  int bb = 1;
  while ((32ll << bb) < 2ll * (m > 0 ? m : 1)) ++bb;  // >= 2 slots per stored key
  L.bb = bb;
  L.t_off = ((size_t)(m > 0 ? m : 1) + 3) & ~(size_t)3;
  L.f_off = L.t_off + ((size_t)32 << bb);
  const size_t nflag = ((size_t)1 << bb) > 32 ? ((size_t)1 << bb) / 32 : 1;
  L.words = (L.f_off + nflag + 3) & ~(size_t)3;
  return L;
}

// The free slot of `free_mask` at or after slot r (cyclically), or -1.
__device__ __forceinline__ int free_slot_from(unsigned free_mask, int r) {
  if (!free_mask) return -1;
  const unsigned rot = r ? (free_mask >> r) | (free_mask << (32 - r)) : free_mask;
  return (__ffs(rot) - 1 + r) & 31;
}

struct BucketSet {
  uint32_t* t;     // (1 << bb) x 32 slots
  uint32_t* flag;  // overflow bits, one per bucket
  int bb;
  uint32_t bmask;
  __device__ uint32_t home(uint32_t key) const { return (key * 0x9E3779B1u) >> (32 - bb); }
  __device__ bool overflowed(uint32_t b) const { return (flag[b >> 5] >> (b & 31)) & 1u; }
  __device__ void mark(uint32_t b) const { atomicOr(&flag[b >> 5], 1u << (b & 31)); }

  // Thread-level insert (the parallel fill): a free slot of the key's bucket,
  // else the next bucket, flagging the full one.
  __device__ void insert_thread(uint32_t key) const {
    uint32_t b = home(key);
    for (uint32_t i = 0; i <= bmask; ++i) {
      for (int s = 0; s < 32; ++s) {
        const int slot = (s + (int)(key & 31u)) & 31;
        if (atomicCAS(&t[b * 32 + slot], kEmpty, key) == kEmpty) return;
      }
      mark(b);
      b = (b + 1) & bmask;
    }
  }

  // Warp-level lookup of one key (all lanes, same key): bucket index and slot,
  // or bucket -1 when absent.
  __device__ int2 find_warp(uint32_t key, int lane) const {
    uint32_t b = home(key);
    for (uint32_t i = 0; i <= bmask; ++i) {
      const unsigned hit = __ballot_sync(kWarp, t[b * 32 + lane] == key);
      if (hit) return make_int2((int)b, __ffs(hit) - 1);
      if (!overflowed(b)) break;
      b = (b + 1) & bmask;
    }
    return make_int2(-1, -1);
  }

  // Warp-level insert of a key known to be absent; returns its bucket.
  __device__ uint32_t insert_warp(uint32_t key, int lane) const {
    uint32_t b = home(key);
    for (uint32_t i = 0; i <= bmask; ++i) {
      const unsigned emp = __ballot_sync(kWarp, t[b * 32 + lane] == kEmpty);
      if (emp) {
        if (lane == 0) t[b * 32 + __ffs(emp) - 1] = key;
        __syncwarp();
        return b;
      }
      if (lane == 0) mark(b);
      __syncwarp();
      b = (b + 1) & bmask;
    }
    return b;
  }

  // Thread-level scan of one bucket (the lanes of a warp scan different
  // buckets, each starting at another quarter-row to spread the banks): the
  // slot holding `key` (-1 if none) and the mask of free slots.
  __device__ void scan(uint32_t b, uint32_t key, int lane, int& at, unsigned& free_mask) const {
    at = -1;
    free_mask = 0;
    const uint4* row = (const uint4*)(t + (size_t)b * 32);
#pragma unroll 4
    for (int c = 0; c < 8; ++c) {
      const int q = (c + lane) & 7;
      const uint4 v = row[q];
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (w[i] == key) at = 4 * q + i;
        if (w[i] == kEmpty) free_mask |= 1u << (4 * q + i);
      }
    }
  }
};

// One attempt's four set operations, by the whole warp: keys q[0], q[1] (the
// new arcs or pairs: looked up, must be absent) and q[2], q[3] (the old ones:
// present, erased on acceptance).  Lanes 8g..8g+7 read key g's home bucket as
// four slots each.  Returns whether the attempt is accepted (neither new key
// present) and, if so, has replaced the old keys by the new ones.
__device__ __forceinline__ bool swap_keys(const BucketSet& S, uint32_t n1, uint32_t n2,
                                          uint32_t o1, uint32_t o2, int lane, uint32_t& ib1,
                                          uint32_t& ib2) {
  const int grp = lane >> 3, sub = lane & 7;
  const uint32_t key = grp == 0 ? n1 : grp == 1 ? n2 : grp == 2 ? o1 : o2;
  const uint32_t b = S.home(key);
  const uint4 v = ((const uint4*)(S.t + (size_t)b * 32))[sub];
  const unsigned hit4 = (v.x == key ? 1u : 0u) | (v.y == key ? 2u : 0u) | (v.z == key ? 4u : 0u) |
                        (v.w == key ? 8u : 0u);
  const unsigned emp4 = (v.x == kEmpty ? 1u : 0u) | (v.y == kEmpty ? 2u : 0u) |
                        (v.z == kEmpty ? 4u : 0u) | (v.w == kEmpty ? 8u : 0u);
  const unsigned hm = __ballot_sync(kWarp, hit4 != 0);
  const unsigned em = __ballot_sync(kWarp, emp4 != 0);
  const bool miss = ((hm >> (8 * grp)) & 0xFFu) == 0;
  // a key not in its home bucket may sit in a later one only past a flagged bucket
  const unsigned deeper = __ballot_sync(kWarp, sub == 0 && miss && S.overflowed(b));
  bool present1, present2;
  if (deeper & 0x0101u) {  // a new key needs the slow lookup
    present1 = S.find_warp(n1, lane).x >= 0;
    present2 = S.find_warp(n2, lane).x >= 0;
  } else {
    present1 = (hm & 0xFFu) != 0;
    present2 = (hm & 0xFF00u) != 0;
  }
  if (present1 || present2) return false;
  // locations: slot = 4 * (first lane of the group with a match) + its first bit
  const int hl1 = __ffs((hm >> 16) & 0xFFu) - 1, hl2 = __ffs((hm >> 24) & 0xFFu) - 1;
  const unsigned h1 = __shfl_sync(kWarp, hit4, 16 + (hl1 < 0 ? 0 : hl1));
  const unsigned h2 = __shfl_sync(kWarp, hit4, 24 + (hl2 < 0 ? 0 : hl2));
  const int el1 = __ffs(em & 0xFFu) - 1, el2 = __ffs((em >> 8) & 0xFFu) - 1;
  const unsigned f1 = __shfl_sync(kWarp, emp4, el1 < 0 ? 0 : el1);
  const unsigned f2 = __shfl_sync(kWarp, emp4, 8 + (el2 < 0 ? 0 : el2));
  const uint32_t b1 = __shfl_sync(kWarp, b, 0), b2 = __shfl_sync(kWarp, b, 8);
  const uint32_t b3 = __shfl_sync(kWarp, b, 16), b4 = __shfl_sync(kWarp, b, 24);
  // erase the old keys (at home, else by the slow lookup)
  int2 p3 = make_int2((int)b3, hl1 < 0 ? -1 : 4 * hl1 + __ffs(h1) - 1);
  int2 p4 = make_int2((int)b4, hl2 < 0 ? -1 : 4 * hl2 + __ffs(h2) - 1);
  if (p3.y < 0) p3 = S.find_warp(o1, lane);
  if (p4.y < 0) p4 = S.find_warp(o2, lane);
  // insert the new keys into free slots of their home buckets; the slow insert
  // for a full home bucket, or for the second key when both share one
  const bool fast1 = el1 >= 0;
  const bool fast2 = el2 >= 0 && b2 != b1;
  if (lane == 0) {
    if (p3.x >= 0) S.t[(size_t)p3.x * 32 + p3.y] = kEmpty;
    if (p4.x >= 0) S.t[(size_t)p4.x * 32 + p4.y] = kEmpty;
    if (fast1) S.t[(size_t)b1 * 32 + 4 * el1 + __ffs(f1) - 1] = n1;
    if (fast2) S.t[(size_t)b2 * 32 + 4 * el2 + __ffs(f2) - 1] = n2;
  }
  __syncwarp();
  ib1 = fast1 ? b1 : S.insert_warp(n1, lane);
  ib2 = fast2 ? b2 : S.insert_warp(n2, lane);
  return true;
}

// The attempts of one graph: `ent` is the entry array (arcs, or the dyad
// lists), `Pol` draws an attempt's two positions and derives from the two
// entries there its validity, the two new keys (to be absent), the two old
// keys (to be erased) and the two new entries.  See the file comment for the
// speculation and resolution of a batch of 32 attempts.
template <class Pol>
__device__ void run_attempts(const Pol& pol, uint32_t* ent, const BucketSet& S, uint64_t attempts,
                             int lane, int64_t* accepted_out) {
  int64_t acc = 0;
  for (uint64_t t0 = 0; t0 < attempts;) {
    const int cnt = (int)((attempts - t0) < 32 ? (attempts - t0) : 32);
    // speculation; mode: 0 never valid (same position twice or past the
    // end), 1 rejected (a new key present), 2 accepted with the recorded
    // locations, 3 to be evaluated on the current state, 4 invalid entries
    uint32_t e1 = 0, e2 = 0;
    const bool drawn = pol.draw(t0 + lane, e1, e2) && lane < cnt;
    int mode = 0;
    uint32_t k1 = 0, k2 = 0, o1 = 0, o2 = 0, w1 = 0, w2 = 0, hb1 = 0xFFFFFFFFu, hb2 = 0xFFFFFFFFu;
    int l1 = -1, l2 = -1, f1 = -1, f2 = -1;
    if (drawn) {
      mode = 4;
      if (pol.make(ent[e1], ent[e2], k1, k2, o1, o2, w1, w2)) {
        hb1 = S.home(k1);
        hb2 = S.home(k2);
        int at1, at2;
        unsigned fm1, fm2, dummy;
        S.scan(hb1, k1, lane, at1, fm1);
        S.scan(hb2, k2, lane, at2, fm2);
        S.scan(S.home(o1), o1, lane, l1, dummy);
        S.scan(S.home(o2), o2, lane, l2, dummy);
        if (l1 >= 0) l1 += (int)S.home(o1) * 32;
        if (l2 >= 0) l2 += (int)S.home(o2) * 32;
        if (at1 >= 0 || at2 >= 0) {
          mode = 1;
        } else if (S.overflowed(hb1) || S.overflowed(hb2) || l1 < 0 || l2 < 0) {
          mode = 3;  // a key may lie past its home bucket
        } else {
          f1 = free_slot_from(fm1, (int)(k1 & 31u));
          if (hb1 == hb2 && f1 >= 0) fm2 = fm1 & ~(1u << f1);
          f2 = free_slot_from(fm2, (int)(k2 & 31u));
          mode = (f1 >= 0 && f2 >= 0) ? 2 : 3;
        }
      }
    }
    // the slots this attempt would fill (bucket * 32 + slot)
    const uint32_t s1 = mode == 2 ? hb1 * 32 + (uint32_t)f1 : 0xFFFFFFFFu;
    const uint32_t s2 = mode == 2 ? hb2 * 32 + (uint32_t)f2 : 0xFFFFFFFFu;
    // An attempt is unsafe when an earlier attempt of the batch that the
    // speculation accepted wrote one of its positions, inserted or erased a
    // key it looks up, or fills a slot it would fill.  Before the first unsafe
    // attempt every speculative outcome is the sequential one, and the
    // accepted attempts there touch disjoint entries and slots.
    bool unsafe = mode == 3;
#pragma unroll 4
    for (int i = 0; i < 31; ++i) {
      const int im = __shfl_sync(kWarp, mode, i);
      const uint32_t ie1 = __shfl_sync(kWarp, e1, i), ie2 = __shfl_sync(kWarp, e2, i);
      const uint32_t ik1 = __shfl_sync(kWarp, k1, i), ik2 = __shfl_sync(kWarp, k2, i);
      const uint32_t io1 = __shfl_sync(kWarp, o1, i), io2 = __shfl_sync(kWarp, o2, i);
      const uint32_t is1 = __shfl_sync(kWarp, s1, i), is2 = __shfl_sync(kWarp, s2, i);
      const bool pos = e1 == ie1 || e1 == ie2 || e2 == ie1 || e2 == ie2;
      const bool key = k1 == ik1 || k1 == ik2 || k2 == ik1 || k2 == ik2 || k1 == io1 ||
                       k1 == io2 || k2 == io1 || k2 == io2;
      const bool slot = s1 == is1 || s1 == is2 || s2 == is1 || s2 == is2;
      unsafe |= im == 2 && lane > i &&
                (pos || (key && (mode == 1 || mode == 2)) || (slot && mode == 2));
    }
    const unsigned bad = __ballot_sync(kWarp, unsafe && mode != 0 && lane < cnt);
    const int p = bad ? __ffs(bad) - 1 : cnt;
    if (lane < p && mode == 2) {
      S.t[l1] = kEmpty;
      S.t[l2] = kEmpty;
      S.t[s1] = k1;
      S.t[s2] = k2;
      ent[e1] = w1;
      ent[e2] = w2;
    }
    acc += __popc(__ballot_sync(kWarp, lane < p && mode == 2));
    __syncwarp();
    if (p < cnt) {
      // the first unsafe attempt, on the current state, by the whole warp
      const uint32_t je1 = __shfl_sync(kWarp, e1, p), je2 = __shfl_sync(kWarp, e2, p);
      uint32_t nk1, nk2, no1, no2, nw1, nw2, nb1, nb2;
      if (pol.make(ent[je1], ent[je2], nk1, nk2, no1, no2, nw1, nw2) &&
          swap_keys(S, nk1, nk2, no1, no2, lane, nb1, nb2)) {
        if (lane == 0) {
          ent[je1] = nw1;
          ent[je2] = nw2;
        }
        ++acc;
      }
      __syncwarp();
      t0 += (uint64_t)p + 1;
    } else {
      t0 += (uint64_t)cnt;
    }
  }
  if (lane == 0 && accepted_out) *accepted_out = acc;
}

// Degree-preserving arc swaps: attempt t's positions are SplitMix64 outputs
// 2t and 2t+1 scaled to [0, m); entries and keys are arcs (src << 16 | dst).
struct ArcSwap {
  uint64_t seed, m;
  __device__ bool draw(uint64_t t, uint32_t& e1, uint32_t& e2) const {
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    e1 = (uint32_t)__umul64hi(sm64_mix(seed + (2 * t + 1) * gamma), m);
    e2 = (uint32_t)__umul64hi(sm64_mix(seed + (2 * t + 2) * gamma), m);
    return e1 != e2;
  }
  __device__ bool make(uint32_t A, uint32_t B, uint32_t& k1, uint32_t& k2, uint32_t& o1,
                       uint32_t& o2, uint32_t& w1, uint32_t& w2) const {
    const uint32_t sa = A >> 16, da = A & 0xFFFFu, sc = B >> 16, dc = B & 0xFFFFu;
    if (sa == sc || da == dc || sa == dc || sc == da) return false;
    k1 = w1 = (sa << 16) | dc;
    k2 = w2 = (sc << 16) | da;
    o1 = A;
    o2 = B;
    return true;
  }
};

struct RandArgs {
  int32_t n, m, G;
  const int32_t* row_ptr;  // shared out-CSR shape
  const int32_t* col0;     // destinations of the source graph (CSR order)
  const uint64_t* seeds;   // G seeds
  uint64_t swaps;
  int32_t* col_out;        // G x m destinations after the swaps (rows unsorted)
  uint32_t* gscratch;      // per-graph state when it does not fit shared memory
  int use_smem;
  int64_t* accepted;       // G counters (may be null)
};

__device__ __forceinline__ int row_of(const int32_t* row_ptr, int n, int e) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(512, 2) k_randomize(RandArgs a) {
  extern __shared__ __align__(16) uint32_t rsm[];
  const int g = blockIdx.x;
  const int m = a.m, n = a.n;
  const RandLayout L = rand_layout(m);
  uint32_t* base = a.use_smem ? rsm : a.gscratch + (size_t)g * L.words;
  uint32_t* arcs = base;
  BucketSet S{base + L.t_off, base + L.f_off, L.bb, (1u << L.bb) - 1u};
  for (size_t i = threadIdx.x; i < ((size_t)32 << L.bb); i += blockDim.x) S.t[i] = kEmpty;
  for (size_t i = threadIdx.x; i < L.words - L.f_off; i += blockDim.x) S.flag[i] = 0;
  for (int e = threadIdx.x; e < m; e += blockDim.x)
    arcs[e] = ((uint32_t)row_of(a.row_ptr, n, e) << 16) | (uint32_t)a.col0[e];
  __syncthreads();
  for (int e = threadIdx.x; e < m; e += blockDim.x) S.insert_thread(arcs[e]);
  __syncthreads();
  // Warp 0: the lanes draw the arc positions of 32 attempts at a time (the
  // SplitMix64 outputs do not depend on the graph), then the warp applies the
  // attempts one after another.
  if (threadIdx.x < 32 && m > 0) {
    const ArcSwap pol{a.seeds[g], (uint64_t)m};
    run_attempts(pol, arcs, S, a.swaps, threadIdx.x, a.accepted ? a.accepted + g : nullptr);
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
  int32_t n, m, G;
  const int32_t* row_ptr;  // shared out-CSR shape (sorted rows)
  const int32_t* col0;
  const uint64_t* seeds;
  uint64_t attempts;
  int32_t* col_out;        // G x m destinations, rows unsorted
  int32_t* scratch;        // G x (2m + n + 2) ints
  uint32_t* gscratch;      // per-graph state when it does not fit shared memory
  int use_smem;
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

__device__ __forceinline__ uint32_t pair_key(uint32_t u, uint32_t v) {
  return u < v ? (u << 16) | v : (v << 16) | u;
}

// Dyad-preserving swaps: attempt t takes SplitMix64 outputs 3t, 3t+1, 3t+2 (the
// list, then two entries of it); entries are (u << 16 | v) of the singles
// [0, S) and the mutual dyads [S, S + D), keys the unordered adjacent pairs.
struct DyadSwap {
  uint64_t seed, S, D;
  __device__ bool draw(uint64_t t, uint32_t& e1, uint32_t& e2) const {
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    const uint64_t r0 = sm64_mix(seed + (3 * t + 1) * gamma);
    const uint64_t r1 = sm64_mix(seed + (3 * t + 2) * gamma);
    const uint64_t r2 = sm64_mix(seed + (3 * t + 3) * gamma);
    const bool single = __umul64hi(r0, S + D) < S;
    const uint64_t len = single ? S : D;
    const uint32_t base_l = single ? 0u : (uint32_t)S;
    e1 = base_l + (uint32_t)__umul64hi(r1, len);
    e2 = base_l + (uint32_t)__umul64hi(r2, len);
    return e1 != e2;
  }
  __device__ bool make(uint32_t A, uint32_t B, uint32_t& k1, uint32_t& k2, uint32_t& o1,
                       uint32_t& o2, uint32_t& w1, uint32_t& w2) const {
    const uint32_t pa = A >> 16, pb = A & 0xFFFFu, pc = B >> 16, pd = B & 0xFFFFu;
    if (pa == pc || pb == pd || pa == pd || pc == pb) return false;
    k1 = pair_key(pa, pd);
    k2 = pair_key(pc, pb);
    o1 = pair_key(pa, pb);
    o2 = pair_key(pc, pd);
    w1 = (pa << 16) | pd;
    w2 = (pc << 16) | pb;
    return true;
  }
};

__global__ void __launch_bounds__(512, 2) k_randomize_dyads(DyadArgs a) {
  extern __shared__ __align__(16) uint32_t dsm[];
  __shared__ int scan_tmp[33];
  const int g = blockIdx.x;
  const int m = a.m, n = a.n;
  const RandLayout L = rand_layout(m);
  uint32_t* base = a.use_smem ? dsm : a.gscratch + (size_t)g * L.words;
  uint32_t* lists = base;  // singles [0, S), dyads [S, S + D)
  BucketSet Sset{base + L.t_off, base + L.f_off, L.bb, (1u << L.bb) - 1u};
  int32_t* fs = a.scratch + (size_t)g * (2 * (size_t)m + n + 2);
  int32_t* fd = fs + m + 1;
  int32_t* cur = fd + m + 1;
  for (size_t i = threadIdx.x; i < ((size_t)32 << L.bb); i += blockDim.x) Sset.t[i] = kEmpty;
  for (size_t i = threadIdx.x; i < L.words - L.f_off; i += blockDim.x) Sset.flag[i] = 0;
  for (int v = threadIdx.x; v < n; v += blockDim.x) cur[v] = 0;
  // kinds of the arcs, in CSR order
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    const int v = row_of(a.row_ptr, n, e), u = a.col0[e];
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
      const uint32_t v = (uint32_t)row_of(a.row_ptr, n, e), u = (uint32_t)a.col0[e];
      if (single) lists[fs[e]] = (v << 16) | u;
      else lists[S + fd[e]] = (v << 16) | u;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < S + D; i += blockDim.x)
    Sset.insert_thread(pair_key(lists[i] >> 16, lists[i] & 0xFFFFu));
  __syncthreads();
  if (threadIdx.x < 32 && S + D > 0) {
    const DyadSwap pol{a.seeds[g], (uint64_t)S, (uint64_t)D};
    run_attempts(pol, lists, Sset, a.attempts, threadIdx.x,
                 a.accepted ? a.accepted + g : nullptr);
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

// Shared memory of one graph's randomiser state, and whether it fits a block.
size_t rand_smem_bytes(int32_t m) { return rand_layout(m).words * 4; }

static bool rand_fits_smem(int32_t m) {
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return rand_smem_bytes(m) <= (size_t)max_smem - 2048;
}

// Scratch (uint32 words) that G randomisations need when their state does not
// fit shared memory (0 when it does).
size_t rand_gscratch_words(int32_t m, int G) {
  return rand_fits_smem(m) ? 0 : (size_t)G * rand_layout(m).words;
}

template <typename Kern, typename Args>
static cudaError_t launch_rand(Kern kern, Args& a, int32_t m, int G, uint32_t* gscratch,
                               cudaStream_t s) {
  a.use_smem = rand_fits_smem(m) ? 1 : 0;
  a.gscratch = gscratch;
  if (!a.use_smem && !gscratch) return cudaErrorInvalidValue;
  const size_t smem = a.use_smem ? rand_smem_bytes(m) : 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<G, 512, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_randomize_dyads(int32_t n, int32_t m, int G, const int32_t* row_ptr,
                                   const int32_t* col0, const uint64_t* seeds, uint64_t attempts,
                                   int32_t* col_out, int32_t* scratch, uint32_t* gscratch,
                                   int64_t* accepted, cudaStream_t s) {
  DyadArgs a;
  a.n = n; a.m = m; a.G = G;
  a.row_ptr = row_ptr; a.col0 = col0; a.seeds = seeds; a.attempts = attempts;
  a.col_out = col_out; a.scratch = scratch; a.accepted = accepted;
  return launch_rand(k_randomize_dyads, a, m, G, gscratch, s);
}

// Enqueue G randomisations of the graph (row_ptr, col0) into col_out.
cudaError_t launch_randomize(int32_t n, int32_t m, int G, const int32_t* row_ptr,
                             const int32_t* col0, const uint64_t* seeds, uint64_t swaps,
                             int32_t* col_out, uint32_t* gscratch, int64_t* accepted,
                             cudaStream_t s) {
  RandArgs a;
  a.n = n; a.m = m; a.G = G;
  a.row_ptr = row_ptr; a.col0 = col0; a.seeds = seeds; a.swaps = swaps;
  a.col_out = col_out; a.accepted = accepted;
  return launch_rand(k_randomize, a, m, G, gscratch, s);
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
  mt_graph* g = nullptr;
  MT_TRY(graph_alloc(src->n, src->m, &g));
  const size_t m1 = (size_t)(src->m > 0 ? src->m : 1);
  const size_t sc = dyad_scratch_ints(src->n, src->m);
  const size_t gwords = rand_gscratch_words(src->m, 1);
  char* scratch = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&scratch, (m1 + sc) * 4 + 64 + gwords * 4 + 16, s);
  int32_t* col_tmp = (int32_t*)scratch;
  int32_t* dsc = col_tmp + m1;
  uint64_t* d_seed = (uint64_t*)(((uintptr_t)(dsc + sc) + 15) & ~(uintptr_t)15);
  uint32_t* gscr = gwords ? (uint32_t*)((char*)d_seed + 16) : nullptr;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->row_ptr, src->row_ptr, (size_t)(src->n + 1) * 4,
                        cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_seed, &seed, 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_randomize_dyads(src->n, src->m, 1, src->row_ptr, src->col, d_seed, attempts,
                               col_tmp, dsc, gscr, nullptr, s);
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
