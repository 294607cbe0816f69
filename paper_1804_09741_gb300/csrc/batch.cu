// Batched null model (the original graph and R randomised graphs, Sec. 1 steps
// (a)-(c); Sec. 4 runs such ensembles of 511 random graphs) and K5, the
// per-class z-scores.
//
// One step is:  randomise R graphs (K3, one block per graph) -> rebuild their
// sorted and undirected CSRs (K4, one block per graph) -> zero the R+1
// histograms -> plan work items over all R+1 graphs -> one persistent
// enumerate-and-classify launch over all items of all graphs (K2) -> z-scores
// (K5).  The step is captured once into a CUDA graph and replayed.
#include <algorithm>
#include <vector>

#include "count.cuh"
#include "trace.cuh"

namespace mt {
cudaError_t launch_randomize(int32_t n, int32_t m, int G, const int32_t* row_ptr,
                             const int32_t* col0, const uint64_t* seeds, uint64_t swaps,
                             int32_t* col_out, uint32_t* gscratch, int64_t* accepted,
                             cudaStream_t s);
size_t rand_gscratch_words(int32_t m, int G);
cudaError_t launch_randomize_dyads(int32_t n, int32_t m, int G, const int32_t* row_ptr,
                                   const int32_t* col0, const uint64_t* seeds, uint64_t attempts,
                                   int32_t* col_out, int32_t* scratch, uint32_t* gscratch,
                                   int64_t* accepted, cudaStream_t s);
size_t dyad_scratch_ints(int32_t n, int32_t m);
size_t rand_smem_bytes(int32_t m);
}  // namespace mt

struct mt_batch {
  const mt_graph* g0 = nullptr;
  const mt_table* t = nullptr;
  int R = 0;
  uint64_t swaps = 0;
  int K = 0;
  uint32_t C = 0;
  int32_t n = 0, m = 0;
  void* mem = nullptr;
  size_t mem_bytes = 0;
  // views into mem
  int32_t *col_rand = nullptr, *col_sorted = nullptr, *urow = nullptr, *usrc = nullptr,
          *ufwd = nullptr;
  uint32_t* ucol = nullptr;
  int32_t *in_ptr = nullptr, *in_tmp = nullptr, *in_col = nullptr, *cursor = nullptr;
  mt::BuildStats* stats = nullptr;
  uint32_t* rand_scratch = nullptr;
  int null_model = MT_NULL_ARC_SWAP;
  int32_t* dyad_scratch = nullptr;
  uint64_t* d_seeds = nullptr;
  mt::DevGraph* d_graphs = nullptr;
  unsigned long long* d_hists = nullptr;
  double* d_z = nullptr;
  void* ws = nullptr;
  uint64_t* h_seeds = nullptr;  // pinned
  mt::CountPlan plan;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  bool ran = false;
};

namespace mt {

// Fill the undirected-entry counts of the null graphs from the builder stats.
__global__ void k_fill_nu(DevGraph* graphs, const BuildStats* stats, int R) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R) graphs[r].nu = stats[r].nu;
}

// z_c = (H0_c - mu_c) / sigma_c, mu and sigma (ddof 0) over the R null rows, in
// float64 with every operation rounded on its own (no fused multiply-add), the
// squares summed in seed order.
__global__ void k_zscore(const unsigned long long* hists, int R, uint32_t C, double* z) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  unsigned long long s1 = 0;
  for (int r = 1; r <= R; ++r) s1 += hists[(size_t)r * C + c];
  const double Rd = (double)R;
  const double mu = __ddiv_rn(__ull2double_rn(s1), Rd);
  double acc = 0.0;
  for (int r = 1; r <= R; ++r) {
    const double d = __dsub_rn(__ull2double_rn(hists[(size_t)r * C + c]), mu);
    acc = __dadd_rn(acc, __dmul_rn(d, d));
  }
  const double var = __ddiv_rn(acc, Rd);
  const double sigma = __dsqrt_rn(var);
  const double diff = __dsub_rn(__ull2double_rn(hists[c]), mu);
  double out;
  if (sigma == 0.0) out = diff == 0.0 ? 0.0 : (diff > 0.0 ? __longlong_as_double(0x7FF0000000000000ll)
                                                          : __longlong_as_double((long long)0xFFF0000000000000ull));
  else out = __ddiv_rn(diff, sigma);
  z[c] = out;
}

static size_t r16(size_t x) { return (x + 15) & ~(size_t)15; }

static mt_status batch_create(const mt_graph* g0, const mt_table* t, int R, uint64_t swaps,
                              int null_model, const mt_tuning* tuning, mt_batch** out) {
  const int K = table_k(t);
  const uint32_t C = table_classes(t);
  const int32_t n = g0->n, m = g0->m;
  // degree bound valid for every null graph: out-degree + in-degree of the original
  std::vector<int32_t> rp(n + 1), col((size_t)std::max(m, 1));
  MT_TRY(mt_graph_copy_csr(g0, rp.data(), col.data(), nullptr));
  std::vector<int32_t> deg(n, 0);
  for (int v = 0; v < n; ++v) deg[v] += rp[v + 1] - rp[v];
  for (int32_t e = 0; e < m; ++e) deg[col[e]] += 1;
  int dbound = 0;
  for (int v = 0; v < n; ++v) dbound = std::max(dbound, deg[v]);
  dbound = std::max(dbound, g0->dmax);

  mt_batch* b = new mt_batch();
  b->g0 = g0; b->t = t; b->R = R; b->swaps = swaps; b->K = K; b->C = C; b->n = n; b->m = m;
  b->null_model = null_model;
  mt_status st = count_configure_tuned(&b->plan, K, R + 1, n, dbound,
                                       (int64_t)(R + 1) * std::max(m, 1),
                                       2 * (int64_t)std::max(m, 1), C, tuning, table_compact(t));
  if (st != MT_OK) {
    delete b;
    return st;
  }
  const size_t m1 = (size_t)std::max(m, 1);
  const size_t rs_words = rand_gscratch_words(m, R);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += r16(bytes);
    return o;
  };
  const size_t o_col_rand = take((size_t)R * m1 * 4);
  const size_t o_col_sorted = take((size_t)R * m1 * 4);
  const size_t o_urow = take((size_t)R * (n + 1) * 4);
  const size_t o_ucol = take((size_t)R * 2 * m1 * 4);
  const size_t o_usrc = take((size_t)R * 2 * m1 * 4);
  const size_t o_ufwd = take((size_t)R * n * 4);
  const size_t o_in_ptr = take((size_t)R * (n + 1) * 4);
  const size_t o_in_tmp = take((size_t)R * m1 * 4);
  const size_t o_in_col = take((size_t)R * m1 * 4);
  const size_t o_cursor = take((size_t)R * n * 4);
  const size_t o_stats = take((size_t)R * sizeof(BuildStats));
  const size_t o_rs = take(rs_words * 4);
  const size_t o_ds =
      take(null_model == MT_NULL_DYAD_SWAP ? (size_t)R * dyad_scratch_ints(n, m) * 4 : 0);
  const size_t o_seeds = take((size_t)R * 8);
  const size_t o_graphs = take((size_t)(R + 1) * sizeof(DevGraph));
  const size_t o_hists = take((size_t)(R + 1) * C * 8);
  const size_t o_z = take((size_t)C * 8);
  const size_t o_ws = take(b->plan.ws_bytes);
  b->mem_bytes = off;
  cudaError_t e = cudaMalloc(&b->mem, off);
  if (e != cudaSuccess) {
    delete b;
    set_last_error(cudaGetErrorString(e));
    return MT_ENOMEM;
  }
  char* base = (char*)b->mem;
  b->col_rand = (int32_t*)(base + o_col_rand);
  b->col_sorted = (int32_t*)(base + o_col_sorted);
  b->urow = (int32_t*)(base + o_urow);
  b->ucol = (uint32_t*)(base + o_ucol);
  b->usrc = (int32_t*)(base + o_usrc);
  b->ufwd = (int32_t*)(base + o_ufwd);
  b->in_ptr = (int32_t*)(base + o_in_ptr);
  b->in_tmp = (int32_t*)(base + o_in_tmp);
  b->in_col = (int32_t*)(base + o_in_col);
  b->cursor = (int32_t*)(base + o_cursor);
  b->stats = (BuildStats*)(base + o_stats);
  b->rand_scratch = rs_words ? (uint32_t*)(base + o_rs) : nullptr;
  b->dyad_scratch = null_model == MT_NULL_DYAD_SWAP ? (int32_t*)(base + o_ds) : nullptr;
  b->d_seeds = (uint64_t*)(base + o_seeds);
  b->d_graphs = (DevGraph*)(base + o_graphs);
  b->d_hists = (unsigned long long*)(base + o_hists);
  b->d_z = (double*)(base + o_z);
  b->ws = base + o_ws;
  e = cudaMallocHost(&b->h_seeds, (size_t)R * 8);
  if (e != cudaSuccess) {
    cudaFree(b->mem);
    delete b;
    return MT_ENOMEM;
  }
  // device graph table: entry 0 = the original, 1..R = the null graphs
  std::vector<DevGraph> hg(R + 1);
  hg[0] = dev_view(g0, b->d_hists);
  for (int r = 0; r < R; ++r) {
    DevGraph& d = hg[r + 1];
    d.n = n;
    d.m = m;
    d.nu = 0;
    d.root_begin = 0;
    d.root_end = n;
    d.pad = 0;
    d.row_ptr = g0->row_ptr;
    d.col = b->col_sorted + (size_t)r * m1;
    d.urow = b->urow + (size_t)r * (n + 1);
    d.ucol = b->ucol + (size_t)r * 2 * m1;
    d.usrc = b->usrc + (size_t)r * 2 * m1;
    d.ufwd = b->ufwd + (size_t)r * n;
    d.hist = b->d_hists + (size_t)(r + 1) * C;
  }
  e = cudaMemcpy(b->d_graphs, hg.data(), hg.size() * sizeof(DevGraph), cudaMemcpyHostToDevice);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&b->ev[i]);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    mt_batch_free(b);
    return MT_ECUDA;
  }
  *out = b;
  return MT_OK;
}

// Enqueue one whole step on s while s is being captured (the phase events are
// recorded as external event nodes so the host can read them after a replay).
static mt_status batch_enqueue(mt_batch* b, cudaStream_t s) {
  const int R = b->R;
  const int32_t n = b->n, m = b->m;
  const size_t m1 = (size_t)std::max(m, 1);
  MT_CUDA_TRY(cudaMemcpyAsync(b->d_seeds, b->h_seeds, (size_t)R * 8, cudaMemcpyHostToDevice, s));
  MT_CUDA_TRY(cudaEventRecordWithFlags(b->ev[0], s, cudaEventRecordExternal));
  if (b->null_model == MT_NULL_DYAD_SWAP)
    MT_CUDA_TRY(launch_randomize_dyads(n, m, R, b->g0->row_ptr, b->g0->col, b->d_seeds, b->swaps,
                                       b->col_rand, b->dyad_scratch, b->rand_scratch, nullptr, s));
  else
    MT_CUDA_TRY(launch_randomize(n, m, R, b->g0->row_ptr, b->g0->col, b->d_seeds, b->swaps,
                                 b->col_rand, b->rand_scratch, nullptr, s));
  BuildArgs a;
  a.n = n; a.m = m; a.G = R;
  a.row_ptr = b->g0->row_ptr; a.row_stride = 0;
  a.col_in = b->col_rand; a.col_out = b->col_sorted;
  a.in_ptr = b->in_ptr; a.in_tmp = b->in_tmp; a.in_col = b->in_col; a.cursor = b->cursor;
  a.urow = b->urow; a.ucol = b->ucol; a.usrc = b->usrc; a.ufwd = b->ufwd; a.stats = b->stats;
  (void)m1;
  MT_CUDA_TRY(launch_build(a, s));
  k_fill_nu<<<(R + 255) / 256, 256, 0, s>>>(b->d_graphs + 1, b->stats, R);
  MT_CUDA_TRY(cudaGetLastError());
  MT_CUDA_TRY(cudaEventRecordWithFlags(b->ev[1], s, cudaEventRecordExternal));
  MT_CUDA_TRY(cudaMemsetAsync(b->d_hists, 0, (size_t)(R + 1) * b->C * 8, s));
  if (n >= b->K) MT_TRY(count_enqueue(b->plan, b->ws, b->d_graphs, table_view(b->t), 0, n, s));
  MT_CUDA_TRY(cudaEventRecordWithFlags(b->ev[2], s, cudaEventRecordExternal));
  k_zscore<<<(b->C + 255) / 256, 256, 0, s>>>(b->d_hists, R, b->C, b->d_z);
  MT_CUDA_TRY(cudaGetLastError());
  MT_CUDA_TRY(cudaEventRecordWithFlags(b->ev[3], s, cudaEventRecordExternal));
  return MT_OK;
}

static mt_status batch_run(mt_batch* b, const uint64_t* seeds, uint64_t* hists, double* z,
                           cudaStream_t s) {
  // the previous replay may still read the pinned seed buffer
  if (b->ran) MT_CUDA_TRY(cudaEventSynchronize(b->ev[0]));
  std::copy(seeds, seeds + b->R, b->h_seeds);
  if (!b->exec) {
    cudaStream_t cs = s;
    bool own = false;
    if (cs == nullptr) {
      MT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      own = true;
    }
    MT_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    mt_status st = batch_enqueue(b, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (own) cudaStreamDestroy(cs);
    if (st != MT_OK) return st;
    MT_CUDA_TRY(e);
    b->graph = graph;
    MT_CUDA_TRY(cudaGraphInstantiate(&b->exec, graph, 0));
  }
  MT_CUDA_TRY(cudaGraphLaunch(b->exec, s));
  b->ran = true;
  const size_t hb = (size_t)(b->R + 1) * b->C * 8;
  bool sync = false;
  auto copy_out = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    cudaPointerAttributes attr;
    const bool dev = cudaPointerGetAttributes(&attr, dst) == cudaSuccess &&
                     (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (!dev) sync = true;
    return cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           s);
  };
  if (hists) MT_CUDA_TRY(copy_out(hists, b->d_hists, hb));
  if (z) MT_CUDA_TRY(copy_out(z, b->d_z, (size_t)b->C * 8));
  if (sync) {
    MT_CUDA_TRY(cudaStreamSynchronize(s));
    uint32_t err = 0;
    MT_CUDA_TRY(cudaMemcpy(&err, count_err_ptr(b->plan, b->ws), 4, cudaMemcpyDeviceToHost));
    if (err) return (err & kErrWaitLimit) ? MT_ETIMEOUT : MT_EOVERFLOW;
  }
  return MT_OK;
}

}  // namespace mt

using namespace mt;

extern "C" {

mt_status mt_batch_create(const mt_graph* g, const mt_table* t, int R, uint64_t swaps,
                          mt_batch** out) {
  if (!g || !t || !out || R < 1) return MT_EINVAL;
  return batch_create(g, t, R, swaps, MT_NULL_ARC_SWAP, nullptr, out);
}

mt_status mt_batch_create_ex(const mt_graph* g, const mt_table* t, int R, uint64_t swaps,
                             int null_model, const mt_tuning* tuning, mt_batch** out) {
  if (!g || !t || !out || R < 1) return MT_EINVAL;
  if (null_model != MT_NULL_ARC_SWAP && null_model != MT_NULL_DYAD_SWAP) return MT_EINVAL;
  if (tuning && (tuning->split_cost < 0 || tuning->split_scale < 0 ||
                 tuning->warps_per_block < 0 || tuning->warps_per_block > 32 ||
                 tuning->stack_cap < 0 || tuning->stack_cap > 65535 ||
                 tuning->method < 0 || tuning->method > 1))
    return MT_EINVAL;
  return batch_create(g, t, R, swaps, null_model, tuning, out);
}

mt_status mt_batch_create_tuned(const mt_graph* g, const mt_table* t, int R, uint64_t swaps,
                                const mt_tuning* tuning, mt_batch** out) {
  if (!g || !t || !out || R < 1) return MT_EINVAL;
  if (tuning && (tuning->split_cost < 0 || tuning->split_scale < 0 ||
                 tuning->warps_per_block < 0 || tuning->warps_per_block > 32 ||
                 tuning->stack_cap < 0 || tuning->stack_cap > 65535 ||
                 tuning->method < 0 || tuning->method > 1))
    return MT_EINVAL;
  return batch_create(g, t, R, swaps, MT_NULL_ARC_SWAP, tuning, out);
}

mt_status mt_batch_free(mt_batch* b) {
  if (!b) return MT_OK;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto& e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->h_seeds) cudaFreeHost(b->h_seeds);
  if (b->mem) cudaFree(b->mem);
  delete b;
  return MT_OK;
}

mt_status mt_batch_run(mt_batch* b, const uint64_t* seeds, uint64_t* hists, double* z,
                       void* stream) {
  if (!b || !seeds) return MT_EINVAL;
  TraceRange tr("mt_batch_run");
  return batch_run(b, seeds, hists, z, (cudaStream_t)stream);
}

mt_status mt_batch_phase_ms(const mt_batch* b, float out[3]) {
  if (!b || !out) return MT_EINVAL;
  if (!b->ran) {
    out[0] = out[1] = out[2] = 0.f;
    return MT_OK;
  }
  MT_CUDA_TRY(cudaEventSynchronize(b->ev[3]));
  MT_CUDA_TRY(cudaEventElapsedTime(&out[0], b->ev[0], b->ev[1]));
  MT_CUDA_TRY(cudaEventElapsedTime(&out[1], b->ev[1], b->ev[2]));
  MT_CUDA_TRY(cudaEventElapsedTime(&out[2], b->ev[2], b->ev[3]));
  return MT_OK;
}

mt_status mt_batch_error(const mt_batch* b, uint32_t* err) {
  if (!b || !err) return MT_EINVAL;
  MT_CUDA_TRY(cudaDeviceSynchronize());
  MT_CUDA_TRY(cudaMemcpy(err, count_err_ptr(b->plan, b->ws), 4, cudaMemcpyDeviceToHost));
  return MT_OK;
}

mt_status mt_count_batch(const mt_graph* g, const mt_table* t, const uint64_t* seeds, int R,
                         uint64_t swaps, uint64_t* hists, double* z, void* stream) {
  TraceRange tr("mt_count_batch");
  mt_batch* b = nullptr;
  MT_TRY(mt_batch_create(g, t, R, swaps, &b));
  mt_status st = mt_batch_run(b, seeds, hists, z, stream);
  if (st == MT_OK) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) st = MT_ECUDA;
  }
  mt_batch_free(b);
  return st;
}

}  // extern "C"
