// Oracle for the Motifs-k hot path: a plain, slow CPU implementation.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
// CPU-baseline leg may load this library.  It shares no code with the CUDA path.
//
// What it computes (Problem 1 "Motifs-k" of Sec. 1 with the definitions of Sec. 2):
//   H_k(G)[c] = #{ S subset of V : |S| = k, G[S] weakly connected,
//                  canon(mask(G[S])) = c }
// * weak connectivity: delta(v) = A(v) u B(v) u C(v) is the undirected
//   neighbourhood (Sec. 2, definition of delta and adj(X));
// * "induced": every arc of G between two members of S is kept (Sec. 1);
// * mask bit layout: for positions i != j in [0,k) the bit index is
//   b(i,j) = i*(k-1) + (j - [j>i]), set iff the arc S[i] -> S[j] exists
//   (row-major adjacency matrix without its diagonal; Sec. 3.2 keys the
//   isomorphism table by the k x k adjacency matrix, 2^(k(k-1)) keys);
// * canon: the numerically smallest mask over all k! relabellings, computed by
//   brute force for every subgraph -- no table (Sec. 3.2 only fixes that each
//   isomorphism class gets one ID);
// * each connected vertex set counts once.
//
// Enumeration: ESU (Wernicke's extension scheme, the "Fanmod" method of Table 1)
// on the undirected graph, root = smallest vertex of the set; a second,
// independent enumerator tries every k-subset (brute force) for n <= 64.
//
// The randomiser is the sequential degree-preserving arc swap (null model of
// Sec. 1, step (c); the paper names no model, so the reading is Milo et al.'s
// switch): attempt t draws arc positions e1, e2 from SplitMix64 outputs 2t and
// 2t+1 of the graph's seed, index = floor(r * m / 2^64); arcs (a->b), (c->d)
// become (a->d), (c->b) unless e1 == e2, a == c, b == d, a == d, c == b, or a new
// arc already exists; the arc array starts in CSR order and the CSR is rebuilt by
// sorting at the end.
//
// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014, in the form of its public-domain reference code):
// state advances by the golden gamma 0x9E3779B97F4A7C15 and each output is
// the mix of the new state; output i of seed s is mix(s + (i+1)*gamma).

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

inline int bit_index(int k, int i, int j) { return i * (k - 1) + (j - (j > i ? 1 : 0)); }

// All k! permutations of 0..k-1 in lexicographic order.
std::vector<std::vector<int>> all_perms(int k) {
  std::vector<int> p(k);
  for (int i = 0; i < k; ++i) p[i] = i;
  std::vector<std::vector<int>> out;
  do {
    out.push_back(p);
  } while (std::next_permutation(p.begin(), p.end()));
  return out;
}

// Brute-force canonical form: minimum over every relabelling pi of the mask in
// which the bit of (i,j) moves to (pi(i), pi(j)).
uint32_t canon_brute(int k, uint32_t mask, const std::vector<std::vector<int>>& perms) {
  int ai[36], aj[36], na = 0;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j)
      if (i != j && ((mask >> bit_index(k, i, j)) & 1u)) {
        ai[na] = i;
        aj[na] = j;
        ++na;
      }
  uint32_t best = 0xFFFFFFFFu;
  for (const auto& pi : perms) {
    uint32_t m2 = 0;
    for (int t = 0; t < na; ++t) m2 |= 1u << bit_index(k, pi[ai[t]], pi[aj[t]]);
    if (m2 < best) best = m2;
  }
  return best;
}

bool mask_connected(int k, uint32_t mask) {
  // Breadth-first search over the underlying undirected graph of the mask.
  bool seen[8] = {false};
  int queue[8], qh = 0, qt = 0;
  queue[qt++] = 0;
  seen[0] = true;
  while (qh < qt) {
    int x = queue[qh++];
    for (int y = 0; y < k; ++y) {
      if (y == x || seen[y]) continue;
      bool xy = (mask >> bit_index(k, x, y)) & 1u;
      bool yx = (mask >> bit_index(k, y, x)) & 1u;
      if (xy || yx) {
        seen[y] = true;
        queue[qt++] = y;
      }
    }
  }
  return qt == k;
}

struct Digraph {
  int n = 0;
  std::vector<std::vector<int>> out;  // sorted out-neighbours
  std::vector<std::vector<int>> und;  // sorted undirected neighbours (delta)

  Digraph(int32_t n_, const int32_t* row_ptr, const int32_t* col) : n(n_), out(n_), und(n_) {
    for (int v = 0; v < n; ++v)
      for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        int u = col[e];
        out[v].push_back(u);
        und[v].push_back(u);
        und[u].push_back(v);
      }
    for (int v = 0; v < n; ++v) {
      std::sort(out[v].begin(), out[v].end());
      std::sort(und[v].begin(), und[v].end());
      und[v].erase(std::unique(und[v].begin(), und[v].end()), und[v].end());
    }
  }
  bool arc(int a, int b) const { return std::binary_search(out[a].begin(), out[a].end(), b); }
  bool adjacent(int a, int b) const {
    return std::binary_search(und[a].begin(), und[a].end(), b);
  }
  uint32_t mask_of(int k, const int* s) const {
    uint32_t mask = 0;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j)
        if (i != j && arc(s[i], s[j])) mask |= 1u << bit_index(k, i, j);
    return mask;
  }
};

using Hist = std::unordered_map<uint32_t, uint64_t>;

// ESU: Vext' = (Vext minus w) plus the exclusive neighbours of w that are larger than the root.
struct Esu {
  const Digraph& g;
  int k;
  const std::vector<std::vector<int>>* perms;  // null: count sets only
  Hist* hist;
  uint64_t sets = 0;

  void extend(std::vector<int>& sub, std::vector<int> ext, int root) {
    if ((int)sub.size() == k) {
      ++sets;
      if (perms) (*hist)[canon_brute(k, g.mask_of(k, sub.data()), *perms)] += 1;
      return;
    }
    while (!ext.empty()) {
      int w = ext.back();
      ext.pop_back();
      branch(sub, ext, root, w);
    }
  }

  // One step of the extension: add w to sub, whose remaining extension set is
  // ext (w already taken out of it), plus w's exclusive neighbours.
  void branch(std::vector<int>& sub, const std::vector<int>& ext, int root, int w) {
    std::vector<int> ext2 = ext;
    for (int u : g.und[w]) {
      if (u <= root) continue;
      bool in_sub = std::find(sub.begin(), sub.end(), u) != sub.end();
      bool near_sub = false;
      for (int x : sub)
        if (g.adjacent(x, u)) near_sub = true;
      if (!in_sub && !near_sub) ext2.push_back(u);
    }
    sub.push_back(w);
    extend(sub, ext2, root);
    sub.pop_back();
  }
};

void esu_roots(const Digraph& g, int k, bool classify, int tid, int nthreads, Hist* hist,
               uint64_t* sets) {
  std::vector<std::vector<int>> perms = all_perms(k);
  Esu esu{g, k, classify ? &perms : nullptr, hist, 0};
  for (int v = tid; v < g.n; v += nthreads) {
    std::vector<int> sub{v};
    std::vector<int> ext;
    for (int u : g.und[v])
      if (u > v) ext.push_back(u);
    esu.extend(sub, ext, v);
  }
  *sets = esu.sets;
}

int64_t write_hist(const Hist& h, uint32_t* masks, uint64_t* counts, int64_t cap) {
  std::map<uint32_t, uint64_t> sorted(h.begin(), h.end());
  int64_t i = 0;
  for (const auto& kv : sorted) {
    if (i < cap) {
      masks[i] = kv.first;
      counts[i] = kv.second;
    }
    ++i;
  }
  return i;
}

inline uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

inline uint64_t splitmix64_output(uint64_t seed, uint64_t i) {
  return splitmix64_mix(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
}

}  // namespace

extern "C" {

uint64_t oracle_splitmix64(uint64_t seed, uint64_t i) { return splitmix64_output(seed, i); }

int oracle_bit_index(int k, int i, int j) { return bit_index(k, i, j); }

uint32_t oracle_canon(int k, uint32_t mask) {
  if (k < 2 || k > 6) return 0xFFFFFFFFu;
  return canon_brute(k, mask, all_perms(k));
}

// Canonical forms of a batch of masks, split over threads.
void oracle_canon_many(int k, const uint32_t* masks, uint32_t* out, int64_t count, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([=] {
      auto perms = all_perms(k);
      for (int64_t i = t; i < count; i += nthreads) out[i] = canon_brute(k, masks[i], perms);
    });
  for (auto& x : th) x.join();
}

int oracle_connected(int k, uint32_t mask) { return mask_connected(k, mask) ? 1 : 0; }

// Every canonical mask (optionally only connected ones) for k <= 5, ascending.
int64_t oracle_class_masks(int k, int connected_only, uint32_t* out, int64_t cap, int nthreads) {
  if (k < 2 || k > 5) return -1;
  const uint64_t total = 1ull << (k * (k - 1));
  if (nthreads < 1) nthreads = 1;
  std::vector<std::vector<uint32_t>> part(nthreads);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t] {
      auto perms = all_perms(k);
      for (uint64_t m = t; m < total; m += nthreads) {
        uint32_t mm = (uint32_t)m;
        if (canon_brute(k, mm, perms) != mm) continue;
        if (connected_only && !mask_connected(k, mm)) continue;
        part[t].push_back(mm);
      }
    });
  for (auto& x : th) x.join();
  std::vector<uint32_t> all;
  for (auto& p : part) all.insert(all.end(), p.begin(), p.end());
  std::sort(all.begin(), all.end());
  for (int64_t i = 0; i < (int64_t)all.size() && i < cap; ++i) out[i] = all[i];
  return (int64_t)all.size();
}

// H_k(G) by ESU + brute-force canonicalisation.  Returns the number of classes
// seen (entries written up to cap, ascending by canonical mask); *sets_out gets
// the number of connected k-sets.
int64_t oracle_count(int32_t n, const int32_t* row_ptr, const int32_t* col, int k, int nthreads,
                     uint32_t* masks_out, uint64_t* counts_out, int64_t cap, uint64_t* sets_out) {
  if (k < 2 || k > 6 || n < 0) return -1;
  Digraph g(n, row_ptr, col);
  if (nthreads < 1) nthreads = 1;
  std::vector<Hist> hists(nthreads);
  std::vector<uint64_t> sets(nthreads, 0);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back(esu_roots, std::cref(g), k, true, t, nthreads, &hists[t], &sets[t]);
  for (auto& x : th) x.join();
  Hist total;
  uint64_t s = 0;
  for (int t = 0; t < nthreads; ++t) {
    for (const auto& kv : hists[t]) total[kv.first] += kv.second;
    s += sets[t];
  }
  if (sets_out) *sets_out = s;
  return write_hist(total, masks_out, counts_out, cap);
}

// H_k(G) restricted to the sets whose smallest vertex lies in roots[0..nroots):
// the same ESU, used to time a bounded sample of a large graph.
int64_t oracle_count_roots(int32_t n, const int32_t* row_ptr, const int32_t* col, int k,
                           const int32_t* roots, int64_t nroots, int nthreads,
                           uint32_t* masks_out, uint64_t* counts_out, int64_t cap,
                           uint64_t* sets_out) {
  if (k < 2 || k > 6 || n < 0) return -1;
  Digraph g(n, row_ptr, col);
  if (nthreads < 1) nthreads = 1;
  std::vector<Hist> hists(nthreads);
  std::vector<uint64_t> sets(nthreads, 0);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t] {
      auto perms = all_perms(k);
      Esu esu{g, k, &perms, &hists[t], 0};
      for (int64_t r = t; r < nroots; r += nthreads) {
        int v = roots[r];
        std::vector<int> sub{v};
        std::vector<int> ext;
        for (int u : g.und[v])
          if (u > v) ext.push_back(u);
        esu.extend(sub, ext, v);
      }
      sets[t] = esu.sets;
    });
  for (auto& x : th) x.join();
  Hist total;
  uint64_t s = 0;
  for (int t = 0; t < nthreads; ++t) {
    for (const auto& kv : hists[t]) total[kv.first] += kv.second;
    s += sets[t];
  }
  if (sets_out) *sets_out = s;
  return write_hist(total, masks_out, counts_out, cap);
}

// The same as oracle_count_roots, with the work of one root spread over the
// threads: the root's first-level extension steps (the i-th vertex taken from
// its extension set, with the set's remaining prefix) are independent of one
// another, so each (root, step) pair is a unit handed to the next free thread.
// Used for roots of very high degree, whose sets one thread would take minutes
// to enumerate.
int64_t oracle_count_roots_split(int32_t n, const int32_t* row_ptr, const int32_t* col, int k,
                                 const int32_t* roots, int64_t nroots, int nthreads,
                                 uint32_t* masks_out, uint64_t* counts_out, int64_t cap,
                                 uint64_t* sets_out) {
  if (k < 2 || k > 6 || n < 0) return -1;
  Digraph g(n, row_ptr, col);
  if (nthreads < 1) nthreads = 1;
  // units: (index into roots, step i); step i takes ext0[size - 1 - i]
  std::vector<std::pair<int64_t, int>> units;
  for (int64_t r = 0; r < nroots; ++r) {
    int v = roots[r];
    int size = 0;
    for (int u : g.und[v])
      if (u > v) ++size;
    for (int i = 0; i < size; ++i) units.push_back({r, i});
  }
  std::atomic<int64_t> next{0};
  std::vector<Hist> hists(nthreads);
  std::vector<uint64_t> sets(nthreads, 0);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t] {
      auto perms = all_perms(k);
      Esu esu{g, k, &perms, &hists[t], 0};
      for (int64_t j = next++; j < (int64_t)units.size(); j = next++) {
        int v = roots[units[j].first];
        std::vector<int> ext0;
        for (int u : g.und[v])
          if (u > v) ext0.push_back(u);
        const int i = units[j].second;
        const int w = ext0[ext0.size() - 1 - i];
        std::vector<int> ext(ext0.begin(), ext0.end() - 1 - i);
        std::vector<int> sub{v};
        esu.branch(sub, ext, v, w);
      }
      sets[t] = esu.sets;
    });
  for (auto& x : th) x.join();
  Hist total;
  uint64_t s = 0;
  for (int t = 0; t < nthreads; ++t) {
    for (const auto& kv : hists[t]) total[kv.first] += kv.second;
    s += sets[t];
  }
  if (sets_out) *sets_out = s;
  return write_hist(total, masks_out, counts_out, cap);
}

// Number of weakly connected k-sets only (ESU without classification).
uint64_t oracle_count_connected_sets(int32_t n, const int32_t* row_ptr, const int32_t* col, int k,
                                     int nthreads) {
  Digraph g(n, row_ptr, col);
  if (nthreads < 1) nthreads = 1;
  std::vector<Hist> hists(nthreads);
  std::vector<uint64_t> sets(nthreads, 0);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back(esu_roots, std::cref(g), k, false, t, nthreads, &hists[t], &sets[t]);
  for (auto& x : th) x.join();
  uint64_t s = 0;
  for (auto x : sets) s += x;
  return s;
}

// Independent enumerator: every k-subset of V (lexicographic combinations), kept
// if a breadth-first search over its undirected induced graph reaches all k
// members.  n <= 64.
int64_t oracle_count_bruteforce(int32_t n, const int32_t* row_ptr, const int32_t* col, int k,
                                uint32_t* masks_out, uint64_t* counts_out, int64_t cap,
                                uint64_t* sets_out) {
  if (n > 64 || k < 2 || k > 6) return -1;
  Digraph g(n, row_ptr, col);
  auto perms = all_perms(k);
  Hist h;
  uint64_t sets = 0;
  if (n >= k) {
    std::vector<int> s(k);
    for (int i = 0; i < k; ++i) s[i] = i;
    while (true) {
      // connectivity of G[s] by BFS over the pairs of s
      bool seen[8] = {false};
      int q[8], qh = 0, qt = 0;
      q[qt++] = 0;
      seen[0] = true;
      while (qh < qt) {
        int x = q[qh++];
        for (int y = 0; y < k; ++y)
          if (!seen[y] && g.adjacent(s[x], s[y])) {
            seen[y] = true;
            q[qt++] = y;
          }
      }
      if (qt == k) {
        ++sets;
        h[canon_brute(k, g.mask_of(k, s.data()), perms)] += 1;
      }
      // next combination
      int i = k - 1;
      while (i >= 0 && s[i] == n - k + i) --i;
      if (i < 0) break;
      ++s[i];
      for (int j = i + 1; j < k; ++j) s[j] = s[j - 1] + 1;
    }
  }
  if (sets_out) *sets_out = sets;
  return write_hist(h, masks_out, counts_out, cap);
}

// Sequential degree-preserving arc swaps; writes the new sorted CSR (same row_ptr
// shape: out-degrees are preserved).  Returns the number of accepted swaps.
int64_t oracle_randomize(int32_t n, const int32_t* row_ptr, const int32_t* col, uint64_t seed,
                         uint64_t swaps, int32_t* row_ptr_out, int32_t* col_out) {
  const int64_t m = row_ptr[n];
  std::vector<std::pair<int, int>> arcs;
  arcs.reserve(m);
  for (int v = 0; v < n; ++v)
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) arcs.emplace_back(v, col[e]);
  std::set<std::pair<int, int>> present(arcs.begin(), arcs.end());
  int64_t accepted = 0;
  for (uint64_t t = 0; t < swaps && m > 0; ++t) {
    uint64_t r1 = splitmix64_output(seed, 2 * t);
    uint64_t r2 = splitmix64_output(seed, 2 * t + 1);
    int64_t e1 = (int64_t)(((unsigned __int128)r1 * (unsigned __int128)m) >> 64);
    int64_t e2 = (int64_t)(((unsigned __int128)r2 * (unsigned __int128)m) >> 64);
    int a = arcs[e1].first, b = arcs[e1].second;
    int c = arcs[e2].first, d = arcs[e2].second;
    if (e1 == e2 || a == c || b == d || a == d || c == b) continue;
    if (present.count({a, d}) || present.count({c, b})) continue;
    present.erase({a, b});
    present.erase({c, d});
    present.insert({a, d});
    present.insert({c, b});
    arcs[e1] = {a, d};
    arcs[e2] = {c, b};
    ++accepted;
  }
  std::sort(arcs.begin(), arcs.end());
  std::vector<int64_t> cnt(n + 1, 0);
  for (auto& a : arcs) cnt[a.first + 1]++;
  row_ptr_out[0] = 0;
  for (int v = 0; v < n; ++v) row_ptr_out[v + 1] = (int32_t)(row_ptr_out[v] + cnt[v + 1]);
  for (int64_t i = 0; i < m; ++i) col_out[i] = arcs[i].second;
  return accepted;
}

// Dyad-preserving randomiser (reading of the "swap mutual pairs and one-way
// arcs separately" null model): the single arcs (u->v without v->u) and the
// mutual dyads {u,v} are two lists in CSR order (a dyad listed once, from its
// smaller end).  Attempt t takes SplitMix64 outputs 3t, 3t+1, 3t+2 of the seed:
// the first picks the kind (single if floor(r*(S+D)/2^64) < S, else dyad), the
// other two pick two entries of that list (index = floor(r*len/2^64)).
//  * singles (a->b), (c->d) become (a->d), (c->b);
//  * dyads {a,b}, {c,d} become {a,d}, {c,b};
// rejected (and counted as used) if the two entries coincide, a == c, b == d,
// a == d, c == b, or a new pair is already adjacent in either direction.
// In- and out-degrees, the number of mutual dyads per vertex and the dyad
// census are preserved.  The CSR is rebuilt by sorting at the end.
int64_t oracle_randomize_dyads(int32_t n, const int32_t* row_ptr, const int32_t* col,
                               uint64_t seed, uint64_t attempts, int32_t* row_ptr_out,
                               int32_t* col_out) {
  std::set<std::pair<int, int>> arcs_in;
  for (int v = 0; v < n; ++v)
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) arcs_in.insert({v, col[e]});
  std::vector<std::pair<int, int>> singles, dyads;
  for (int v = 0; v < n; ++v)
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      const int u = col[e];
      if (arcs_in.count({u, v})) {
        if (v < u) dyads.emplace_back(v, u);
      } else {
        singles.emplace_back(v, u);
      }
    }
  // adjacency of unordered pairs
  std::set<std::pair<int, int>> adj;
  for (auto& a : arcs_in) adj.insert({std::min(a.first, a.second), std::max(a.first, a.second)});
  auto key = [](int x, int y) { return std::make_pair(std::min(x, y), std::max(x, y)); };
  const uint64_t S = singles.size(), D = dyads.size();
  int64_t accepted = 0;
  for (uint64_t t = 0; t < attempts && S + D > 0; ++t) {
    const uint64_t r0 = splitmix64_output(seed, 3 * t);
    const uint64_t r1 = splitmix64_output(seed, 3 * t + 1);
    const uint64_t r2 = splitmix64_output(seed, 3 * t + 2);
    const uint64_t pick = (uint64_t)(((unsigned __int128)r0 * (unsigned __int128)(S + D)) >> 64);
    const bool single = pick < S;
    std::vector<std::pair<int, int>>& L = single ? singles : dyads;
    const uint64_t len = L.size();
    const uint64_t e1 = (uint64_t)(((unsigned __int128)r1 * (unsigned __int128)len) >> 64);
    const uint64_t e2 = (uint64_t)(((unsigned __int128)r2 * (unsigned __int128)len) >> 64);
    if (e1 == e2) continue;
    const int a = L[e1].first, b = L[e1].second, c = L[e2].first, d = L[e2].second;
    if (a == c || b == d || a == d || c == b) continue;
    if (adj.count(key(a, d)) || adj.count(key(c, b))) continue;
    adj.erase(key(a, b));
    adj.erase(key(c, d));
    adj.insert(key(a, d));
    adj.insert(key(c, b));
    L[e1] = {a, d};
    L[e2] = {c, b};
    ++accepted;
  }
  std::vector<std::pair<int, int>> arcs(singles.begin(), singles.end());
  for (auto& p : dyads) {
    arcs.emplace_back(p.first, p.second);
    arcs.emplace_back(p.second, p.first);
  }
  std::sort(arcs.begin(), arcs.end());
  std::vector<int64_t> cnt(n + 1, 0);
  for (auto& a : arcs) cnt[a.first + 1]++;
  row_ptr_out[0] = 0;
  for (int v = 0; v < n; ++v) row_ptr_out[v + 1] = (int32_t)(row_ptr_out[v] + cnt[v + 1]);
  for (size_t i = 0; i < arcs.size(); ++i) col_out[i] = arcs[i].second;
  return accepted;
}

}  // extern "C"
