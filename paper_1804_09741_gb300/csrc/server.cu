// Serving: continuous batching of count requests of mixed k and size.
//
// The paper has no serving layer (its parallelism is threads over graphs,
// Sec. 4); this runtime keeps the per-k isomorphism tables resident and runs
// count requests as they arrive.  Work advances in rounds:
//  * admission: pending requests (FIFO) are admitted while a slot is free and
//    the memory budget (graph + histogram + planner share) allows; their graphs
//    are loaded on a separate stream with stream-ordered allocations;
//  * a round gives every active request a chunk of its roots (a root range
//    whose estimated cost fits the request's share of the round budget; a
//    connected k-set belongs to its smallest vertex, so chunks never overlap)
//    and launches one planner + enumerator per k over all chunks of that k.
//    Shares are water-filled: a request that needs less than an equal share
//    finishes, and what it leaves goes to the others.  The k's launches of a
//    round run on their own streams, so one k's kernel tail overlaps the
//    next k's kernel;
//  * a request whose last chunk ran is complete when its round's event fires:
//    its histogram was copied to a pinned buffer behind the kernels, its device
//    memory goes back to the pool and its slot frees up for the next admission.
//    Each k's launch also copies its device status word out; a request any of
//    whose chunks ran in a launch that reported an error (an expired bounded
//    wait, a stack or queue bound) fails with that error instead of returning
//    a histogram that may be incomplete;
//  * the budget covers the requests' memory and the per-k round scratch
//    (planner, work queue, graph descriptors): a request is admitted only if
//    the scratch its k would need with it active still fits.
// Rounds are double-buffered: the host admits and plans round r+1 while the GPU
// runs round r, so requests that arrive mid-round join the next round instead
// of waiting for whole requests ahead of them to finish.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <vector>

#include "count.cuh"
#include "trace.cuh"

namespace mt {

struct SrvRequest {
  uint64_t id = 0;
  int k = 0;
  int32_t n = 0, m = 0;
  std::vector<int32_t> rp, col;  // host copy until admitted
  std::vector<double> cum;       // cumulative per-root cost estimate (n+1)
  int32_t dmax_b = 0;            // bounds for planning before the device build:
  int32_t nu_b = 0;              //   largest in+out degree, 2m undirected entries
  uint32_t taint = 0;            // device error bits of launches its chunks ran in
  mt_graph* g = nullptr;
  unsigned long long* d_hist = nullptr;
  uint64_t* h_result = nullptr;  // pinned
  size_t bytes = 0;              // memory budget charge
  int next_root = 0;
  int state = 0;                 // 0 pending, 1 active, 2 done, 3 failed
  mt_status status = MT_OK;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

struct RoundBuf {
  cudaEvent_t ev = nullptr;
  std::vector<SrvRequest*> finishing;
  std::vector<SrvRequest*> chunked[4];  // requests with a chunk in this round, per k
  uint32_t* h_err = nullptr;            // pinned: each k's launch status word
  DevGraph* h_graphs = nullptr;  // pinned staging of the round's graph descriptors
  size_t h_cap = 0;
  bool pending = false;
};

}  // namespace mt

struct mt_server {
  const mt_table* tables[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t budget = 0, used = 0;
  int max_slots = 0;
  double round_cost = 0;
  cudaStream_t stream = nullptr, load_stream = nullptr;
  cudaEvent_t load_ev = nullptr;
  cudaStream_t kstream[4] = {nullptr, nullptr, nullptr, nullptr};  // a round's launch per k
  cudaEvent_t fork_ev = nullptr, kdone_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  std::deque<mt::SrvRequest*> pending;
  std::vector<mt::SrvRequest*> active;
  std::map<uint64_t, mt::SrvRequest*> all;
  uint64_t next_id = 1;
  int64_t round = 0;
  mt::RoundBuf rb[2];
  void* ws[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t ws_bytes[4] = {0, 0, 0, 0};
  mt::DevGraph* d_graphs[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t d_graphs_cap[4] = {0, 0, 0, 0};
  size_t reserved[4] = {0, 0, 0, 0};  // round scratch charged to the budget, per k
  std::vector<uint64_t*> pinned_free[4];  // result buffers by k
  std::chrono::steady_clock::time_point t0;
  int method = MT_METHOD_ENUMERATE;
};

namespace mt {

static double now_ms(const mt_server* s) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - s->t0)
      .count();
}

static double choose_d(double x, int r) {
  if (x < r) return 0.0;
  double c = 1.0;
  for (int i = 0; i < r; ++i) c = c * (x - i) / (i + 1);
  return c;
}

// Per-root cost estimate from degrees: every arc (a,b) adds C(d_a + d_b, k-2)
// to its smaller end, the root that owns the sets grown through it.
static void root_costs(SrvRequest* r) {
  const int n = r->n;
  std::vector<int32_t> deg(n, 0);
  for (int v = 0; v < n; ++v) deg[v] += r->rp[v + 1] - r->rp[v];
  for (int32_t e = 0; e < r->m; ++e) deg[r->col[e]] += 1;
  r->dmax_b = 1;
  for (int v = 0; v < n; ++v) r->dmax_b = std::max(r->dmax_b, deg[v]);
  r->nu_b = std::max(2 * r->m, 1);
  std::vector<double> cost(n, 1.0);
  for (int v = 0; v < n; ++v)
    for (int32_t e = r->rp[v]; e < r->rp[v + 1]; ++e) {
      const int u = r->col[e];
      const int lo = std::min(v, u), hi = std::max(v, u);
      cost[lo] += 1.0 + choose_d((double)deg[lo] + deg[hi], r->k - 2);
    }
  r->cum.assign(n + 1, 0.0);
  for (int v = 0; v < n; ++v) r->cum[v + 1] = r->cum[v] + cost[v];
}

static size_t request_bytes(const SrvRequest* r, uint32_t C) {
  // graph arrays + histogram + a planner/work-item share per arc
  return graph_device_bytes(r->n, r->m) + (size_t)C * 8 + (size_t)64 * (r->m + r->n) + 4096;
}

// Launch plan of one k's round over the active requests of that k (plus
// `extra`, when given): the round's chunks are a subset of them, and a
// request's degree bound and 2m bound its device graph's, so the scratch of
// any round is at most this plan's.
static mt_status plan_for(const mt_server* s, int ki, const SrvRequest* extra, CountPlan* p,
                          int* G) {
  int nmax = 1, dmax = 1, numax = 1, g = 0;
  int64_t fwd = 0;
  auto add = [&](const SrvRequest* r) {
    nmax = std::max(nmax, r->n);
    dmax = std::max(dmax, r->dmax_b);
    numax = std::max(numax, r->nu_b);
    fwd += r->nu_b / 2 + 1;
    ++g;
  };
  for (const SrvRequest* r : s->active)
    if (r->k == ki + 3) add(r);
  if (extra) add(extra);
  *G = g;
  if (g == 0) return MT_OK;
  mt_tuning tun;
  tun.split_cost = 0.0;
  tun.split_scale = 0.0;
  tun.warps_per_block = 0;
  tun.stack_cap = 0;
  tun.method = s->method;
  return count_configure_tuned(p, ki + 3, g, nmax, dmax, fwd, numax,
                               table_classes(s->tables[ki]),
                               s->method == MT_METHOD_ENUMERATE ? nullptr : &tun,
                               table_compact(s->tables[ki]));
}

// Round scratch of k's launch (planner and work queue, graph descriptors) for
// the active requests of k plus `extra`; 0 when there are none or when the
// launch cannot be configured (such requests fail in the round, unscheduled).
static size_t scratch_need(const mt_server* s, int ki, const SrvRequest* extra) {
  CountPlan p;
  int G = 0;
  if (plan_for(s, ki, extra, &p, &G) != MT_OK || G == 0) return 0;
  return p.ws_bytes + (size_t)G * sizeof(DevGraph);
}

static size_t reserved_total(const mt_server* s) {
  size_t t = 0;
  for (size_t x : s->reserved) t += x;
  return t;
}

static mt_status acquire_pinned(mt_server* s, int k, uint32_t C, uint64_t** out) {
  auto& pool = s->pinned_free[k - 3];
  if (!pool.empty()) {
    *out = pool.back();
    pool.pop_back();
    return MT_OK;
  }
  MT_CUDA_TRY(cudaMallocHost((void**)out, (size_t)C * 8));
  return MT_OK;
}

static void release_request(mt_server* s, SrvRequest* r) {
  if (r->g) graph_release(r->g, s->stream);
  r->g = nullptr;
  if (r->d_hist) cudaFreeAsync(r->d_hist, s->stream);
  r->d_hist = nullptr;
  if (r->state == 1 || r->state == 2) s->used -= std::min(s->used, r->bytes);
}

// A request that cannot run (its launch cannot be configured): it fails alone
// with `st`, its memory and slot are released.
static void fail_request(mt_server* s, RoundBuf& R, SrvRequest* r, mt_status st) {
  release_request(s, r);
  if (r->h_result) s->pinned_free[r->k - 3].push_back(r->h_result);
  r->h_result = nullptr;
  r->state = 3;
  r->status = st;
  r->t_done = now_ms(s);
  s->active.erase(std::find(s->active.begin(), s->active.end(), r));
  auto f = std::find(R.finishing.begin(), R.finishing.end(), r);
  if (f != R.finishing.end()) R.finishing.erase(f);
}

static void admit(mt_server* s) {
  bool loaded = false;
  while (!s->pending.empty() && (int)s->active.size() < s->max_slots) {
    SrvRequest* r = s->pending.front();
    const uint32_t C = table_classes(s->tables[r->k - 3]);
    r->bytes = request_bytes(r, C);
    if (r->bytes > s->budget) {  // can never fit
      s->pending.pop_front();
      r->state = 3;
      r->status = MT_EBUSY;
      r->t_done = now_ms(s);
      continue;
    }
    // the scratch r's k needs with r active, against what k holds now
    const int ki = r->k - 3;
    const size_t need_k = std::max(s->reserved[ki], scratch_need(s, ki, r));
    if (r->bytes + need_k > s->budget) {  // can never fit, even alone
      s->pending.pop_front();
      r->state = 3;
      r->status = MT_EBUSY;
      r->t_done = now_ms(s);
      continue;
    }
    if (s->used + r->bytes + reserved_total(s) - s->reserved[ki] + need_k > s->budget) break;
    s->pending.pop_front();
    mt_status st = graph_load_on(r->n, r->m, r->rp.data(), r->col.data(), s->load_stream, &r->g);
    if (st == MT_OK) st = acquire_pinned(s, r->k, C, &r->h_result);
    if (st == MT_OK) {
      cudaError_t e = cudaMallocAsync((void**)&r->d_hist, (size_t)C * 8, s->load_stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(r->d_hist, 0, (size_t)C * 8, s->load_stream);
      if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        st = MT_ECUDA;
      }
    }
    if (st != MT_OK) {
      if (r->g) graph_release(r->g, s->load_stream);
      r->g = nullptr;
      if (r->h_result) s->pinned_free[r->k - 3].push_back(r->h_result);
      r->h_result = nullptr;
      r->state = 3;
      r->status = st;
      r->t_done = now_ms(s);
      continue;
    }
    std::vector<int32_t>().swap(r->rp);
    std::vector<int32_t>().swap(r->col);
    s->used += r->bytes;
    s->reserved[ki] = need_k;
    r->state = 1;
    r->t_admit = now_ms(s);
    r->next_root = 0;
    s->active.push_back(r);
    loaded = true;
  }
  if (loaded) {
    cudaEventRecord(s->load_ev, s->load_stream);
    cudaStreamWaitEvent(s->stream, s->load_ev, 0);
  }
}

// Grow k's round scratch to this round's plan.  The admitted requests' plan
// bounds it, so what is allocated stays within the reservation charged to the
// budget.
static mt_status ensure_capacity(mt_server* s, int ki, size_t ws_need, size_t graphs) {
  if (s->ws_bytes[ki] < ws_need) {
    if (s->ws[ki]) MT_CUDA_TRY(cudaFreeAsync(s->ws[ki], s->stream));
    s->ws[ki] = nullptr;
    s->ws_bytes[ki] = 0;
    MT_CUDA_TRY(cudaMallocAsync(&s->ws[ki], ws_need, s->stream));
    s->ws_bytes[ki] = ws_need;
  }
  if (s->d_graphs_cap[ki] < graphs) {
    if (s->d_graphs[ki]) MT_CUDA_TRY(cudaFreeAsync(s->d_graphs[ki], s->stream));
    const size_t cap = graphs;
    MT_CUDA_TRY(cudaMallocAsync((void**)&s->d_graphs[ki], cap * sizeof(DevGraph), s->stream));
    s->d_graphs_cap[ki] = cap;
  }
  return MT_OK;
}

// Free k's round scratch once no active request of k is left (stream-ordered
// behind every launch enqueued so far) and drop its reservation.
static void release_idle_scratch(mt_server* s) {
  for (int ki = 0; ki < 4; ++ki) {
    bool any = false;
    for (const SrvRequest* r : s->active) any |= r->k == ki + 3;
    if (any) continue;
    if (s->ws[ki]) cudaFreeAsync(s->ws[ki], s->stream);
    if (s->d_graphs[ki]) cudaFreeAsync(s->d_graphs[ki], s->stream);
    s->ws[ki] = nullptr;
    s->ws_bytes[ki] = 0;
    s->d_graphs[ki] = nullptr;
    s->d_graphs_cap[ki] = 0;
    s->reserved[ki] = 0;
  }
}

static mt_status harvest(mt_server* s, RoundBuf& b, int32_t* completed) {
  if (!b.pending) return MT_OK;
  MT_CUDA_TRY(cudaEventSynchronize(b.ev));
  const double t = now_ms(s);
  // a launch that reported an error taints every request it ran a chunk of
  for (int ki = 0; ki < 4; ++ki) {
    if (b.h_err[ki])
      for (SrvRequest* r : b.chunked[ki]) r->taint |= b.h_err[ki];
    b.chunked[ki].clear();
  }
  for (SrvRequest* r : b.finishing) {
    release_request(s, r);  // while still active: its budget charge is returned
    if (r->taint) {
      r->state = 3;
      r->status = (r->taint & kErrWaitLimit) ? MT_ETIMEOUT : MT_EOVERFLOW;
      if (r->h_result) s->pinned_free[r->k - 3].push_back(r->h_result);
      r->h_result = nullptr;
    } else {
      r->state = 2;
      ++*completed;
    }
    r->t_done = t;
    s->active.erase(std::find(s->active.begin(), s->active.end(), r));
  }
  b.finishing.clear();
  b.pending = false;
  release_idle_scratch(s);
  return MT_OK;
}

static mt_status step(mt_server* s, int32_t* completed) {
  *completed = 0;
  admit(s);
  const int cur = (int)(s->round & 1);
  RoundBuf& R = s->rb[cur];
  // chunks: each active request with roots left gets a share of the round
  std::vector<SrvRequest*> open;
  for (SrvRequest* r : s->active)
    if (r->next_root < r->n) open.push_back(r);
  if (!open.empty()) {
    // water-filling: in ascending order of remaining cost, each request takes
    // the smaller of its remaining cost and an equal share of what is left
    std::vector<double> rem(open.size()), give(open.size());
    std::vector<size_t> order(open.size());
    for (size_t i = 0; i < open.size(); ++i) {
      rem[i] = open[i]->cum[open[i]->n] - open[i]->cum[open[i]->next_root];
      order[i] = i;
    }
    std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return rem[x] < rem[y]; });
    double budget = s->round_cost;
    size_t left = open.size();
    for (size_t i : order) {
      give[i] = std::min(rem[i], budget / (double)left);
      budget -= give[i];
      --left;
    }
    struct Chunk {
      SrvRequest* r;
      int a, b;
    };
    std::vector<Chunk> by_k[4];
    for (size_t i = 0; i < open.size(); ++i) {
      SrvRequest* r = open[i];
      const int a = r->next_root;
      int b = r->n;
      if (give[i] < rem[i]) {
        const double limit = r->cum[a] + give[i];
        b = (int)(std::upper_bound(r->cum.begin() + a + 1, r->cum.end(), limit) - r->cum.begin()) - 1;
        b = std::max(b, a + 1);
        b = std::min(b, r->n);
      }
      by_k[r->k - 3].push_back({r, a, b});
      R.chunked[r->k - 3].push_back(r);
      r->next_root = b;
      if (b == r->n) R.finishing.push_back(r);
    }
    size_t total = 0;
    for (auto& v : by_k) total += v.size();
    if (R.h_cap < total) {
      if (R.h_graphs) cudaFreeHost(R.h_graphs);
      R.h_graphs = nullptr;
      R.h_cap = 0;
      MT_CUDA_TRY(cudaMallocHost((void**)&R.h_graphs, std::max<size_t>(total, 64) * sizeof(DevGraph)));
      R.h_cap = std::max<size_t>(total, 64);
    }
    size_t off = 0;
    CountPlan plans[4];
    int nmaxs[4] = {0, 0, 0, 0};
    for (int ki = 0; ki < 4; ++ki) {
      auto& chunks = by_k[ki];
      if (chunks.empty()) continue;
      const int K = ki + 3;
      const mt_table* t = s->tables[ki];
      const uint32_t C = table_classes(t);
      int nmax = 1, dmax = 1, numax = 1;
      int64_t fwd = 0;
      for (auto& c : chunks) {
        nmax = std::max(nmax, c.r->g->n);
        dmax = std::max(dmax, c.r->g->dmax);
        numax = std::max(numax, c.r->g->nu);
        fwd += c.r->g->nu / 2 + 1;
      }
      CountPlan p;
      mt_tuning tun;
      tun.split_cost = 0.0;
      tun.split_scale = 0.0;
      tun.warps_per_block = 0;
      tun.stack_cap = 0;
      tun.method = s->method;
      mt_status cst =
          count_configure_tuned(&p, K, (int)chunks.size(), nmax, dmax, fwd, numax, C,
                                s->method == MT_METHOD_ENUMERATE ? nullptr : &tun, table_compact(t));
      if (cst == MT_OK) cst = ensure_capacity(s, ki, p.ws_bytes, chunks.size());
      if (cst == MT_OK)  // charge what is held, should the plan outgrow the reservation
        s->reserved[ki] = std::max(s->reserved[ki],
                                   s->ws_bytes[ki] + s->d_graphs_cap[ki] * sizeof(DevGraph));
      if (cst != MT_OK) {
        // this k cannot run (its table and the server's method do not go
        // together, e.g. the cell method on a compact k = 6 table, or its
        // scratch cannot be allocated): its requests fail alone, before any
        // of their roots is marked as counted
        for (auto& c : chunks) fail_request(s, R, c.r, cst);
        chunks.clear();
        R.chunked[ki].clear();
        cudaGetLastError();  // an allocation failure is not sticky: clear it
        continue;
      }
      DevGraph* hg = R.h_graphs + off;
      for (size_t i = 0; i < chunks.size(); ++i) {
        hg[i] = dev_view(chunks[i].r->g, chunks[i].r->d_hist);
        hg[i].root_begin = chunks[i].a;
        hg[i].root_end = chunks[i].b;
      }
      MT_CUDA_TRY(cudaMemcpyAsync(s->d_graphs[ki], hg, chunks.size() * sizeof(DevGraph),
                                  cudaMemcpyHostToDevice, s->stream));
      plans[ki] = p;
      nmaxs[ki] = nmax;
      off += chunks.size();
    }
    // fork: each k's launch waits for what the main stream holds (loads,
    // allocations, descriptors, the previous round), then joins back
    MT_CUDA_TRY(cudaEventRecord(s->fork_ev, s->stream));
    for (int ki = 0; ki < 4; ++ki) R.h_err[ki] = 0;  // this buffer's last round was harvested
    for (int ki = 0; ki < 4; ++ki) {
      if (by_k[ki].empty()) continue;
      MT_CUDA_TRY(cudaStreamWaitEvent(s->kstream[ki], s->fork_ev, 0));
      MT_TRY(count_enqueue(plans[ki], s->ws[ki], s->d_graphs[ki], table_view(s->tables[ki]), 0,
                           nmaxs[ki], s->kstream[ki]));
      MT_CUDA_TRY(cudaMemcpyAsync(R.h_err + ki, count_err_ptr(plans[ki], s->ws[ki]), 4,
                                  cudaMemcpyDeviceToHost, s->kstream[ki]));
      MT_CUDA_TRY(cudaEventRecord(s->kdone_ev[ki], s->kstream[ki]));
      MT_CUDA_TRY(cudaStreamWaitEvent(s->stream, s->kdone_ev[ki], 0));
    }
    for (SrvRequest* r : R.finishing) {
      const uint32_t C = table_classes(s->tables[r->k - 3]);
      MT_CUDA_TRY(cudaMemcpyAsync(r->h_result, r->d_hist, (size_t)C * 8, cudaMemcpyDeviceToHost,
                                  s->stream));
    }
    MT_CUDA_TRY(cudaEventRecord(R.ev, s->stream));
    R.pending = true;
  }
  // harvest the previous round while this one runs
  MT_TRY(harvest(s, s->rb[cur ^ 1], completed));
  s->round += 1;
  // when nothing new was launched, also settle the round just enqueued
  if (open.empty()) MT_TRY(harvest(s, R, completed));
  return MT_OK;
}

}  // namespace mt

using namespace mt;

extern "C" {

mt_status mt_server_create(const mt_table* t3, const mt_table* t4, const mt_table* t5,
                           const mt_table* t6, size_t memory_budget, int max_slots,
                           double round_cost, mt_server** out) {
  if (!out || max_slots < 1 || memory_budget == 0 || round_cost <= 0) return MT_EINVAL;
  const mt_table* ts[4] = {t3, t4, t5, t6};
  for (int i = 0; i < 4; ++i)
    if (ts[i] && table_k(ts[i]) != i + 3) return MT_EINVAL;
  mt_server* s = new mt_server();
  for (int i = 0; i < 4; ++i) s->tables[i] = ts[i];
  s->budget = memory_budget;
  s->max_slots = max_slots;
  s->round_cost = round_cost;
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->load_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->load_ev, cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&s->rb[i].ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s->rb[i].h_err, 4 * sizeof(uint32_t));
    if (e == cudaSuccess) std::fill(s->rb[i].h_err, s->rb[i].h_err + 4, 0u);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&s->kstream[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->kdone_ev[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    mt_server_free(s);
    return MT_ECUDA;
  }
  *out = s;
  return MT_OK;
}

mt_status mt_server_submit(mt_server* s, int k, int32_t n, int32_t m, const int32_t* row_ptr,
                           const int32_t* col, uint64_t* id) {
  if (!s || !id) return MT_EINVAL;
  if (k < 3 || k > 6 || !s->tables[k - 3]) return MT_EUNSUPPORTED;
  MT_TRY(validate_csr(n, m, row_ptr, col));
  SrvRequest* r = new SrvRequest();
  r->id = s->next_id++;
  r->k = k;
  r->n = n;
  r->m = m;
  r->rp.assign(row_ptr, row_ptr + n + 1);
  r->col.assign(col, col + m);
  root_costs(r);
  r->t_submit = now_ms(s);
  s->pending.push_back(r);
  s->all[r->id] = r;
  *id = r->id;
  return MT_OK;
}

mt_status mt_server_step(mt_server* s, int32_t* completed, int32_t* active, int32_t* pending) {
  if (!s) return MT_EINVAL;
  TraceRange tr("mt_server_step");
  int32_t done = 0;
  mt_status st = step(s, &done);
  if (completed) *completed = done;
  if (active) *active = (int32_t)s->active.size();
  if (pending) *pending = (int32_t)s->pending.size();
  return st;
}

mt_status mt_server_result(mt_server* s, uint64_t id, int32_t* state, uint64_t* hist,
                           double* latency_ms) {
  if (!s) return MT_EINVAL;
  auto it = s->all.find(id);
  if (it == s->all.end()) return MT_EINVAL;
  SrvRequest* r = it->second;
  if (state) *state = r->state;
  if (latency_ms) *latency_ms = r->state >= 2 ? r->t_done - r->t_submit : 0.0;
  if (r->state == 3) {
    const mt_status st = r->status;
    s->all.erase(it);
    delete r;
    return st;
  }
  if (r->state == 2 && hist) {
    const uint32_t C = table_classes(s->tables[r->k - 3]);
    std::copy(r->h_result, r->h_result + C, hist);
    s->pinned_free[r->k - 3].push_back(r->h_result);
    r->h_result = nullptr;
    s->all.erase(it);
    delete r;
  }
  return MT_OK;
}

mt_status mt_server_set_method(mt_server* s, int method) {
  if (!s || (method != MT_METHOD_ENUMERATE && method != MT_METHOD_CELLS)) return MT_EINVAL;
  s->method = method;
  return MT_OK;
}

mt_status mt_server_used_bytes(const mt_server* s, size_t* used) {
  if (!s || !used) return MT_EINVAL;
  *used = s->used + reserved_total(s);
  return MT_OK;
}

mt_status mt_server_free(mt_server* s) {
  if (!s) return MT_OK;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->load_stream) cudaStreamSynchronize(s->load_stream);
  for (auto& kv : s->all) {
    SrvRequest* r = kv.second;
    if (r->g) graph_release(r->g, s->stream);
    if (r->d_hist) cudaFreeAsync(r->d_hist, s->stream);
    if (r->h_result) cudaFreeHost(r->h_result);
    delete r;
  }
  for (int i = 0; i < 4; ++i) {
    if (s->ws[i]) cudaFreeAsync(s->ws[i], s->stream);
    if (s->d_graphs[i]) cudaFreeAsync(s->d_graphs[i], s->stream);
    for (uint64_t* p : s->pinned_free[i]) cudaFreeHost(p);
  }
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& b : s->rb) {
    if (b.ev) cudaEventDestroy(b.ev);
    if (b.h_graphs) cudaFreeHost(b.h_graphs);
    if (b.h_err) cudaFreeHost(b.h_err);
  }
  if (s->load_ev) cudaEventDestroy(s->load_ev);
  if (s->fork_ev) cudaEventDestroy(s->fork_ev);
  for (int i = 0; i < 4; ++i) {
    if (s->kstream[i]) {
      cudaStreamSynchronize(s->kstream[i]);
      cudaStreamDestroy(s->kstream[i]);
    }
    if (s->kdone_ev[i]) cudaEventDestroy(s->kdone_ev[i]);
  }
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->load_stream) cudaStreamDestroy(s->load_stream);
  delete s;
  return MT_OK;
}

}  // extern "C"
