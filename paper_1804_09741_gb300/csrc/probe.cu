// Measured ceilings of the two memory operations the classification step
// performs per subgraph (Sec. 3.2: one table read; Problem 1: one histogram
// add): random 4-byte reads from a table of a given size, and random 64-bit
// atomic adds into a histogram of a given size.  Indices come from a hash of
// the thread and iteration (no index stream), so the rate is that of the
// gather or atomic path itself (L2 when the buffer fits in it).
#include <algorithm>

#include "common.cuh"

namespace mt {

__device__ __forceinline__ uint32_t probe_hash(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return x;
}

__global__ void __launch_bounds__(256) k_probe_gather(const uint32_t* __restrict__ table,
                                                      uint32_t mask, int iters, uint32_t* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  uint32_t h = probe_hash(tid);
#pragma unroll 8
  for (int i = 0; i < iters; ++i) {
    h = probe_hash(h + (uint32_t)i);
    acc += __ldg(&table[h & mask]);
  }
  if (acc == 0x12345678u) sink[tid & 1023] = acc;  // keeps the loads alive
}

__global__ void __launch_bounds__(256) k_probe_atomic(unsigned long long* hist, uint32_t mask,
                                                      int iters) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t h = probe_hash(tid ^ 0x9E3779B9u);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
    h = probe_hash(h + (uint32_t)i);
    atomicAdd(&hist[h & mask], 1ull);
  }
}

}  // namespace mt

using namespace mt;

extern "C" mt_status mt_probe_rates(uint64_t table_words, uint64_t hist_words, double* gathers_per_s,
                                    double* atomics_per_s) {
  if (table_words == 0 || hist_words == 0 || (table_words & (table_words - 1)) ||
      (hist_words & (hist_words - 1)) || table_words > (1ull << 30) || hist_words > (1ull << 28))
    return MT_EINVAL;
  int dev = 0, sms = 0;
  MT_CUDA_TRY(cudaGetDevice(&dev));
  MT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  uint32_t* table = nullptr;
  unsigned long long* hist = nullptr;
  uint32_t* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mt_status st = MT_OK;
  float ms_g = 0.f, ms_a = 0.f;
  const int blocks = sms * 8, threads = 256;
  const int iters_g = 4096, iters_a = 1024;
  do {
    cudaError_t e = cudaMalloc(&table, table_words * 4);
    if (e == cudaSuccess) e = cudaMalloc(&hist, hist_words * 8);
    if (e == cudaSuccess) e = cudaMalloc(&sink, 4096);
    if (e == cudaSuccess) e = cudaMemset(table, 1, table_words * 4);
    if (e == cudaSuccess) e = cudaMemset(hist, 0, hist_words * 8);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
      set_last_error(cudaGetErrorString(e));
      st = e == cudaErrorMemoryAllocation ? MT_ENOMEM : MT_ECUDA;
      break;
    }
    // warm-up, then timed runs
    k_probe_gather<<<blocks, threads>>>(table, (uint32_t)(table_words - 1), iters_g / 8, sink);
    k_probe_atomic<<<blocks, threads>>>(hist, (uint32_t)(hist_words - 1), iters_a / 8);
    cudaEventRecord(e0);
    k_probe_gather<<<blocks, threads>>>(table, (uint32_t)(table_words - 1), iters_g, sink);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_g, e0, e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0);
    k_probe_atomic<<<blocks, threads>>>(hist, (uint32_t)(hist_words - 1), iters_a);
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_a, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_last_error(cudaGetErrorString(e));
      st = MT_ECUDA;
      break;
    }
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (table) cudaFree(table);
  if (hist) cudaFree(hist);
  if (sink) cudaFree(sink);
  if (st != MT_OK) return st;
  const double n = (double)blocks * threads;
  if (gathers_per_s) *gathers_per_s = n * iters_g / (ms_g * 1e-3);
  if (atomics_per_s) *atomics_per_s = n * iters_a / (ms_a * 1e-3);
  return MT_OK;
}
