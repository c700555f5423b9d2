// Random-access ceiling of the device: uniformly random 8-byte loads,
// stores and 64-bit compare-and-swaps over a large buffer.  The global switch
// round is dominated by exactly these accesses (gathers of E, probes and
// claims of the dependency table), so their sustained rate, in 32-byte
// sectors per second, is the denominator of its random-access roofline.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gesmc_microbench.h"

namespace {

__device__ __forceinline__ unsigned long long mix(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

constexpr int kIlp = 4;

__global__ void k_fill(unsigned long long *buf, unsigned long long words, unsigned long long value) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < words;
       i += (unsigned long long)gridDim.x * blockDim.x)
    buf[i] = value;
}

// kind 0: loads, 1: stores, 2: CAS, 3: 32-bit atomic add with return, 4: the
// same without return.  Each thread issues `per_thread` accesses
// in groups of kIlp independent ones.
__global__ void k_random(unsigned long long *buf, unsigned long long words, int kind, uint32_t per_thread,
                         unsigned long long salt, unsigned long long *sink) {
  const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  unsigned long long acc = 0;
  for (uint32_t it = 0; it < per_thread; it += kIlp) {
    unsigned long long idx[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) idx[u] = __umul64hi(mix(salt ^ (tid * per_thread + it + u)), words);
    if (kind == 0) {
#pragma unroll
      for (int u = 0; u < kIlp; ++u) acc += __ldcg(&buf[idx[u]]);
    } else if (kind == 1) {
#pragma unroll
      for (int u = 0; u < kIlp; ++u) __stcg(&buf[idx[u]], idx[u]);
    } else if (kind == 2) {
#pragma unroll
      for (int u = 0; u < kIlp; ++u) acc += atomicCAS(&buf[idx[u]], ~0ull, idx[u]);
    } else if (kind == 3) {  // 32-bit add with return (a cursor), counters at 8-byte spacing
#pragma unroll
      for (int u = 0; u < kIlp; ++u) acc += atomicAdd(reinterpret_cast<unsigned int *>(&buf[idx[u]]), 1u);
    } else {  // 32-bit add without return (a histogram count)
#pragma unroll
      for (int u = 0; u < kIlp; ++u) atomicAdd(reinterpret_cast<unsigned int *>(&buf[idx[u]]), 1u);
    }
  }
  if (acc == 0x123456789ull) *sink = acc;  // keeps the loads alive
}

}  // namespace

extern "C" int gesmc_probe_random_access(uint64_t bytes, int kind, uint64_t accesses, double *accesses_per_s) {
  if (!accesses_per_s || kind < 0 || kind > 4 || bytes < 4096 || accesses == 0) return -1;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return -6;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned long long words = bytes / 8;
  unsigned long long *buf = nullptr, *sink = nullptr;
  if (cudaMalloc(&buf, words * 8) != cudaSuccess) {
    cudaGetLastError();
    return -5;
  }
  if (cudaMalloc(&sink, 8) != cudaSuccess) {
    cudaFree(buf);
    cudaGetLastError();
    return -5;
  }
  const int threads = 256, blocks = sms * 8;
  const unsigned long long nthreads = (unsigned long long)threads * blocks;
  uint32_t per_thread = (uint32_t)((accesses + nthreads - 1) / nthreads);
  per_thread = (per_thread + kIlp - 1) / kIlp * kIlp;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f, best = 1e30f;
  bool ok = true;
  for (int rep = 0; rep < 4 && ok; ++rep) {
    k_fill<<<sms * 16, 256>>>(buf, words, ~0ull);
    cudaEventRecord(e0);
    k_random<<<blocks, threads>>>(buf, words, kind, per_thread, 0x9E3779B97F4A7C15ull * (rep + 1), sink);
    cudaEventRecord(e1);
    ok = cudaEventSynchronize(e1) == cudaSuccess;
    if (ok && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  cudaFree(sink);
  if (!ok || cudaGetLastError() != cudaSuccess) return -6;
  *accesses_per_s = (double)nthreads * per_thread / (best / 1e3);
  return 0;
}
