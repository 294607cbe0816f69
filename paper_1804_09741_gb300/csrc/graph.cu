// Graph loading and the device graph builder.
//
// The builder turns a directed out-CSR whose rows may be unsorted into
//  * the same CSR with every row sorted ascending (duplicates flagged),
//  * the undirected neighbour CSR of Sec. 2: for each vertex v the sorted set
//    delta(v) = A(v) u B(v) u C(v), each entry tagged with which of the arcs
//    v->u, u->v exist,
//  * per entry its row vertex, per vertex the index of its first neighbour
//    larger than itself, and per graph the undirected degree maximum.
// One thread block builds one graph; G graphs of equal n and m build in one
// launch (the null graphs of a batch).
#include <cstring>
#include <mutex>
#include <vector>

#include "graph.cuh"
#include "trace.cuh"

namespace mt {

namespace {
thread_local std::string g_last_error;
}

void set_last_error(const std::string& s) { g_last_error = s; }

__device__ __forceinline__ int row_of(const int32_t* row_ptr, int n, int e) {
  // largest v with row_ptr[v] <= e (rows may be empty)
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(1024) k_build(BuildArgs a) {
  __shared__ int scan_tmp[33];
  __shared__ int s_dmax;
  __shared__ unsigned s_err;
  const int g = blockIdx.x;
  const int n = a.n, m = a.m;
  const int32_t* row_ptr = a.row_ptr + (size_t)g * a.row_stride;
  const int32_t* col_in = a.col_in + (size_t)g * m;
  int32_t* col_out = a.col_out + (size_t)g * m;
  int32_t* in_ptr = a.in_ptr + (size_t)g * (n + 1);
  int32_t* in_tmp = a.in_tmp + (size_t)g * m;
  int32_t* in_col = a.in_col + (size_t)g * m;
  int32_t* cursor = a.cursor + (size_t)g * n;
  int32_t* urow = a.urow + (size_t)g * (n + 1);
  uint32_t* ucol = a.ucol + (size_t)g * 2 * m;
  int32_t* usrc = a.usrc + (size_t)g * 2 * m;
  int32_t* ufwd = a.ufwd + (size_t)g * n;
  const int tid = threadIdx.x, nt = blockDim.x;

  if (tid == 0) { s_dmax = 0; s_err = 0; }
  for (int v = tid; v <= n; v += nt) in_ptr[v] = 0;
  __syncthreads();
  // in-degrees
  for (int e = tid; e < m; e += nt) atomicAdd(&in_ptr[col_in[e]], 1);
  __syncthreads();
  block_exclusive_scan(in_ptr, n + 1, scan_tmp);
  for (int v = tid; v < n; v += nt) cursor[v] = in_ptr[v];
  __syncthreads();
  // scatter sources into in-rows (unordered), rank-sort the out-rows
  for (int e = tid; e < m; e += nt) {
    const int v = row_of(row_ptr, n, e);
    const int x = col_in[e];
    const int pos = atomicAdd(&cursor[x], 1);
    in_tmp[pos] = v;
    int rank = 0;
    bool dup = false;
    for (int f = row_ptr[v]; f < row_ptr[v + 1]; ++f) {
      const int y = col_in[f];
      rank += y < x;
      dup |= (y == x) && (f != e);
    }
    if (dup) atomicOr(&s_err, kErrDuplicateArc);
    else col_out[row_ptr[v] + rank] = x;
  }
  __syncthreads();
  // rank-sort the in-rows (sources of a vertex are distinct unless duplicated)
  for (int e = tid; e < m; e += nt) {
    const int x = row_of(in_ptr, n, e);
    const int y0 = in_tmp[e];
    int rank = 0;
    for (int f = in_ptr[x]; f < in_ptr[x + 1]; ++f) rank += in_tmp[f] < y0;
    in_col[in_ptr[x] + rank] = y0;
  }
  __syncthreads();
  if (s_err) {
    if (tid == 0) {
      a.stats[g].err = s_err;
      a.stats[g].nu = 0;
      a.stats[g].dmax = 0;
    }
    return;
  }
  // undirected degree = size of the union of the sorted out- and in-rows
  for (int v = tid; v < n; v += nt) {
    int i = row_ptr[v], ie = row_ptr[v + 1], j = in_ptr[v], je = in_ptr[v + 1], c = 0;
    while (i < ie || j < je) {
      const int x = i < ie ? col_out[i] : 0x7FFFFFFF;
      const int y = j < je ? in_col[j] : 0x7FFFFFFF;
      if (x <= y) ++i;
      if (y <= x) ++j;
      ++c;
    }
    urow[v] = c;
    atomicMax(&s_dmax, c);
  }
  if (tid == 0) urow[n] = 0;
  __syncthreads();
  const long long nu = block_exclusive_scan(urow, n + 1, scan_tmp);
  // write the labelled undirected rows
  for (int v = tid; v < n; v += nt) {
    int i = row_ptr[v], ie = row_ptr[v + 1], j = in_ptr[v], je = in_ptr[v + 1];
    int o = urow[v];
    int fwd = -1;
    while (i < ie || j < je) {
      const int x = i < ie ? col_out[i] : 0x7FFFFFFF;
      const int y = j < je ? in_col[j] : 0x7FFFFFFF;
      const int u = x < y ? x : y;
      uint32_t code = 0;
      if (x <= y) { code |= 1u << 30; ++i; }   // arc v -> u
      if (y <= x) { code |= 1u << 31; ++j; }   // arc u -> v
      if (fwd < 0 && u > v) fwd = o - urow[v];
      ucol[o] = code | (uint32_t)u;
      usrc[o] = v;
      ++o;
    }
    ufwd[v] = fwd < 0 ? o - urow[v] : fwd;
  }
  if (tid == 0) {
    a.stats[g].err = 0;
    a.stats[g].nu = (int32_t)nu;
    a.stats[g].dmax = s_dmax;
  }
}

cudaError_t launch_build(const BuildArgs& a, cudaStream_t s) {
  if (a.G <= 0) return cudaSuccess;
  k_build<<<a.G, 1024, 0, s>>>(a);
  return cudaGetLastError();
}

DevGraph dev_view(const mt_graph* g, unsigned long long* hist) {
  DevGraph d;
  d.n = g->n;
  d.m = g->m;
  d.nu = g->nu;
  d.root_begin = 0;
  d.root_end = g->n;
  d.pad = 0;
  d.row_ptr = g->row_ptr;
  d.col = g->col;
  d.urow = g->urow;
  d.ucol = g->ucol;
  d.usrc = g->usrc;
  d.ufwd = g->ufwd;
  d.hist = hist;
  return d;
}

size_t graph_device_bytes(int32_t n, int32_t m) {
  const size_t m1 = (size_t)(m > 0 ? m : 1);
  const size_t ints = (size_t)(n + 1) + m1 + (size_t)(n + 1) + 2 * m1 + 2 * m1 + (size_t)n;
  return ints * 4 + 256;
}

// Allocate the device arrays of a graph with n vertices and m arcs (with
// cudaMallocAsync on `s` when `pooled`).
static mt_status graph_alloc_impl(int32_t n, int32_t m, bool pooled, cudaStream_t s,
                                  mt_graph** out) {
  mt_graph* g = new mt_graph();
  g->n = n;
  g->m = m;
  const size_t m1 = (size_t)(m > 0 ? m : 1);
  void* mem = nullptr;
  cudaError_t e = pooled ? cudaMallocAsync(&mem, graph_device_bytes(n, m), s)
                         : cudaMalloc(&mem, graph_device_bytes(n, m));
  if (e != cudaSuccess) {
    delete g;
    set_last_error(cudaGetErrorString(e));
    return MT_ENOMEM;
  }
  g->mem = mem;
  g->pooled = pooled;
  int32_t* p = (int32_t*)mem;
  g->row_ptr = p; p += n + 1;
  g->col = p; p += m1;
  g->urow = p; p += n + 1;
  g->ucol = (uint32_t*)p; p += 2 * m1;
  g->usrc = p; p += 2 * m1;
  g->ufwd = p; p += n;
  *out = g;
  return MT_OK;
}

mt_status graph_alloc(int32_t n, int32_t m, mt_graph** out) {
  return graph_alloc_impl(n, m, false, nullptr, out);
}

void graph_release(mt_graph* g, cudaStream_t s) {
  if (!g) return;
  if (g->pooled) {
    if (g->mem) cudaFreeAsync(g->mem, s);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    delete g;
  } else {
    mt_graph_free(g);
  }
}

mt_status validate_csr(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col) {
  if (!row_ptr || (m > 0 && !col) || n < 1 || m < 0) return MT_EINVAL;
  if (n > kMaxVertices) return MT_EUNSUPPORTED;
  if (row_ptr[0] != 0 || row_ptr[n] != m) return MT_EINVAL;
  for (int32_t v = 0; v < n; ++v) {
    if (row_ptr[v + 1] < row_ptr[v]) return MT_EINVAL;
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
      if (col[e] < 0 || col[e] >= n || col[e] == v) return MT_EINVAL;
  }
  return MT_OK;
}

mt_status graph_build_sync(mt_graph* g, const int32_t* col_in, cudaStream_t s);

static mt_status graph_load_impl(int32_t n, int32_t m, const int32_t* row_ptr,
                                 const int32_t* col, bool pooled, cudaStream_t s,
                                 mt_graph** out) {
  MT_TRY(validate_csr(n, m, row_ptr, col));
  mt_graph* g = nullptr;
  MT_TRY(graph_alloc_impl(n, m, pooled, s, &g));
  int32_t* col_in = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&col_in, (size_t)(m > 0 ? m : 1) * 4, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->row_ptr, row_ptr, (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && m > 0)
    e = cudaMemcpyAsync(col_in, col, (size_t)m * 4, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    if (col_in) cudaFreeAsync(col_in, s);
    graph_release(g, s);
    return MT_ECUDA;
  }
  mt_status st = graph_build_sync(g, col_in, s);
  cudaFreeAsync(col_in, s);
  if (st != MT_OK) {
    graph_release(g, s);
    return st;
  }
  *out = g;
  return MT_OK;
}

mt_status graph_load_on(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col,
                        cudaStream_t s, mt_graph** out) {
  return graph_load_impl(n, m, row_ptr, col, true, s, out);
}

// Build the sorted and undirected CSRs of `g` from unsorted destinations
// `col_in` (device, m) using its own row_ptr, then read back the stats.
mt_status graph_build_sync(mt_graph* g, const int32_t* col_in, cudaStream_t s) {
  const size_t m1 = (size_t)(g->m > 0 ? g->m : 1);
  const size_t scratch_ints = (size_t)(g->n + 1) + 2 * m1 + (size_t)g->n;
  void* scratch = nullptr;
  MT_CUDA_TRY(cudaMallocAsync(&scratch, scratch_ints * 4 + sizeof(BuildStats) + 256, s));
  int32_t* p = (int32_t*)scratch;
  BuildArgs a;
  a.n = g->n; a.m = g->m; a.G = 1;
  a.row_ptr = g->row_ptr; a.row_stride = 0;
  a.col_in = col_in; a.col_out = g->col;
  a.in_ptr = p; p += g->n + 1;
  a.in_tmp = p; p += m1;
  a.in_col = p; p += m1;
  a.cursor = p; p += g->n;
  a.stats = (BuildStats*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  a.urow = g->urow; a.ucol = g->ucol; a.usrc = g->usrc; a.ufwd = g->ufwd;
  cudaError_t e = launch_build(a, s);
  BuildStats st{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, a.stats, sizeof(st), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return MT_ECUDA;
  }
  if (st.err & kErrDuplicateArc) return MT_EINVAL;
  g->nu = st.nu;
  g->dmax = st.dmax;
  return MT_OK;
}

}  // namespace mt

using namespace mt;

extern "C" {

const char* mt_status_str(mt_status s) {
  switch (s) {
    case MT_OK: return "ok";
    case MT_EINVAL: return "invalid argument or malformed graph";
    case MT_EUNSUPPORTED: return "unsupported size (k outside 3..6, n > 65535 or degree too large)";
    case MT_ENOMEM: return "out of memory";
    case MT_ECUDA: return "CUDA error";
    case MT_ETIMEOUT: return "bounded device wait expired";
    case MT_EOVERFLOW: return "device stack or queue overflow";
    case MT_EBUSY: return "admission refused (budget or slots)";
  }
  return "unknown status";
}

const char* mt_last_error(void) { return g_last_error.c_str(); }

mt_status mt_graph_load_csr(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col,
                            void* stream, mt_graph** out) {
  if (!out) return MT_EINVAL;
  TraceRange tr("mt_graph_load_csr");
  return graph_load_impl(n, m, row_ptr, col, false, (cudaStream_t)stream, out);
}

mt_status mt_graph_free(mt_graph* g) {
  if (!g) return MT_OK;
  cudaDeviceSynchronize();
  if (g->mem) cudaFree(g->mem);
  if (g->ws && g->ws_owned) cudaFree(g->ws);
  if (g->ev0) cudaEventDestroy(g->ev0);
  if (g->ev1) cudaEventDestroy(g->ev1);
  delete g;
  return MT_OK;
}

mt_status mt_graph_info(const mt_graph* g, int32_t* n, int32_t* m, int32_t* m_undirected,
                        int32_t* max_degree) {
  if (!g) return MT_EINVAL;
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (m_undirected) *m_undirected = g->nu / 2;
  if (max_degree) *max_degree = g->dmax;
  return MT_OK;
}

mt_status mt_graph_copy_csr(const mt_graph* g, int32_t* row_ptr, int32_t* col, void* stream) {
  if (!g || !row_ptr || (g->m > 0 && !col)) return MT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  MT_CUDA_TRY(cudaMemcpyAsync(row_ptr, g->row_ptr, (size_t)(g->n + 1) * 4,
                              cudaMemcpyDeviceToHost, s));
  if (g->m > 0)
    MT_CUDA_TRY(cudaMemcpyAsync(col, g->col, (size_t)g->m * 4, cudaMemcpyDeviceToHost, s));
  MT_CUDA_TRY(cudaStreamSynchronize(s));
  return MT_OK;
}

}  // extern "C"
