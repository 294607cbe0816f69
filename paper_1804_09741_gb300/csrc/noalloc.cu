// mt_count_noalloc: the counting call for programs that must not allocate GPU
// memory while they run.
//
// mt_count keeps its planner and work-queue scratch in memory it allocates on
// the graph handle the first time it needs it.  Some callers cannot accept that:
// a service that reserves its whole device-memory budget up front (through its
// own pool or a framework's caching allocator) has nothing left for an
// unplanned cudaMalloc, and a latency-sensitive loop cannot afford one either,
// because cudaMalloc/cudaFree may synchronise the device.  This entry point
// runs the same planner and enumerator kernels with their scratch taken from a
// fixed array compiled into the library, and allocates nothing.
//
// The fixed array holds kNoAllocScratchBytes (8 MiB).  Every GPU that loads the
// library reserves it until the process exits.  All calls share it, so calls
// that overlap on the GPU (different streams, different threads) race and give
// wrong counts: order them on one stream or synchronise between them.
//
// The launch's status word (stack or queue overflow, an expired idle wait)
// stays in the array's header until the next call; mt_count_noalloc_error
// copies it out, because the count itself returns before the kernels run.
#include <mutex>

#include "count.cuh"

namespace mt {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array, looked up once per device.  In host code the
// array's name is only a host-side stand-in; kernels need the address that
// cudaGetSymbolAddress returns for the current device.
static void* g_scratch_addr[kNoAllocMaxDevices] = {};
static std::mutex g_scratch_mu;

static mt_status scratch_address(void** out) {
  int dev = 0;
  MT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return MT_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_last_error(std::string("cudaGetSymbolAddress(noalloc scratch): ") +
                     cudaGetErrorString(e));
      return MT_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return MT_OK;
}

// Writes the graph descriptor into the fixed scratch (no host staging copy).
__global__ void k_put_graph(DevGraph* dst, DevGraph src) { *dst = src; }

static mt_status count_noalloc(const mt_graph* g, const mt_table* t, uint64_t* hist,
                               cudaStream_t s) {
  int dev = 0;
  MT_CUDA_TRY(cudaGetDevice(&dev));
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, hist) != cudaSuccess ||
      (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    set_last_error("mt_count_noalloc: hist must be device memory");
    return MT_EINVAL;
  }
  if (attr.type == cudaMemoryTypeDevice && attr.device != dev) {
    // this device's kernels would write another GPU's memory
    set_last_error("mt_count_noalloc: hist is memory of device " + std::to_string(attr.device) +
                   ", the current device is " + std::to_string(dev));
    return MT_EINVAL;
  }
  void* scratch = nullptr;
  MT_TRY(scratch_address(&scratch));
  const int K = table_k(t);
  const uint32_t C = table_classes(t);
  CountPlan p;
  MT_TRY(count_configure(&p, K, 1, g->n, g->dmax, g->nu / 2 + 1, g->nu > 0 ? g->nu : 1, C, 0.0, 0,
                         table_compact(t)));
  const size_t desc_off = (p.ws_bytes + 255) & ~(size_t)255;
  const size_t need = desc_off + 256;
  if (need > kNoAllocScratchBytes) {
    set_last_error("mt_count_noalloc: this graph needs " + std::to_string(need) +
                   " bytes of scratch; the fixed scratch holds " +
                   std::to_string(kNoAllocScratchBytes) + " bytes (use mt_count)");
    return MT_EUNSUPPORTED;
  }
  DevGraph* dg = (DevGraph*)((char*)scratch + desc_off);
  k_put_graph<<<1, 1, 0, s>>>(dg, dev_view(g, (unsigned long long*)hist));
  MT_CUDA_TRY(cudaGetLastError());
  MT_CUDA_TRY(cudaMemsetAsync(hist, 0, (size_t)C * 8, s));
  if (g->n >= K) {
    MT_TRY(count_enqueue(p, scratch, dg, table_view(t), 0, g->n, s));
  } else {
    // no launch: clear the status word a previous call left behind
    MT_CUDA_TRY(cudaMemsetAsync(count_err_ptr(p, scratch), 0, 4, s));
  }
  return MT_OK;
}

// Status word of the last count that used the fixed scratch: its planner and
// enumerator write their error bits into the header at the start of the array.
static mt_status noalloc_error(uint32_t* err, cudaStream_t s) {
  void* scratch = nullptr;
  MT_TRY(scratch_address(&scratch));
  uint32_t word = 0;
  MT_CUDA_TRY(cudaMemcpyAsync(&word, count_err_ptr(CountPlan{}, scratch), 4,
                              cudaMemcpyDeviceToHost, s));
  MT_CUDA_TRY(cudaStreamSynchronize(s));
  if (err) *err = word;
  if (word == 0) return MT_OK;
  return (word & kErrWaitLimit) ? MT_ETIMEOUT : MT_EOVERFLOW;
}

}  // namespace mt

extern "C" mt_status mt_count_noalloc_error(uint32_t* err, void* stream) {
  return mt::noalloc_error(err, (cudaStream_t)stream);
}

extern "C" mt_status mt_count_noalloc(const mt_graph* g, const mt_table* t, uint64_t* hist,
                                      void* stream) {
  if (!g || !t || !hist) return MT_EINVAL;
  return mt::count_noalloc(g, t, hist, (cudaStream_t)stream);
}
