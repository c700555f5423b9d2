// G(n, p) starting graphs generated on the GPU (the SynGnp inputs of
// Sec. 6), for chains too large to generate and copy from the host quickly.
// Two passes over the same deterministic chunks: count the edges of every
// chunk, scan the counts, then regenerate each chunk into its offset.
#include <math.h>

#include "../../include/gesmc_gen.h"
#include "device_util.cuh"

namespace gesmc {
namespace {

struct GnpArgs {
  unsigned long long n, pairs, chunk, chunks, seed;
  double log_q;  // log(1 - p)
  int all;       // p == 1: every pair
};

// Offset of row u's first pair {u, u + 1} in the row-by-row numbering.
__device__ __forceinline__ unsigned long long row_start(unsigned long long n, unsigned long long u) {
  return u * (2 * n - u - 1) / 2;
}

// Row u holding pair t: the float estimate from the quadratic, then fixed
// exactly with integer row offsets.
__device__ __forceinline__ unsigned long long row_of(unsigned long long n, unsigned long long t) {
  const double a = 2.0 * (double)n - 1.0;
  double est = (a - sqrt(a * a - 8.0 * (double)t)) * 0.5;
  unsigned long long u = est < 0 ? 0 : (unsigned long long)est;
  if (u > n - 2) u = n - 2;
  while (u > 0 && row_start(n, u) > t) --u;
  while (u + 1 <= n - 2 && row_start(n, u + 1) <= t) ++u;
  return u;
}

// The chunk's edges in pair order; write = false only counts them.  Not
// inlined: the counting and the writing pass run the same code, so they
// agree on every chunk's count.
__device__ __noinline__ unsigned long long walk_chunk(const GnpArgs &g, unsigned long long c, unsigned long long *out,
                                         bool write) {
  const unsigned long long beg = c * g.chunk;
  const unsigned long long end = min(beg + g.chunk, g.pairs);
  unsigned long long cnt = 0, u = 0, u_end = 0, t = beg;
  bool have_row = false;
  U64x4 w;
  for (unsigned long long d = 0;; ++d) {
    if (g.all) {
      if (d > 0) ++t;
    } else {
      if ((d & 3) == 0) w = philox(c, d >> 2, 3, 0, g.seed, 0);
      const double U = (double)(word_of(w, (uint32_t)(d & 3)) >> 11) * 0x1.0p-53;
      const double skip = floor(log1p(-U) / g.log_q);
      // the first draw lands on pair beg + skip, later ones on t + 1 + skip
      const double step = (d ? 1.0 : 0.0) + skip;
      if (step >= (double)(end - t)) break;
      t += (unsigned long long)step;
    }
    if (t >= end) break;
    if (write) {
      if (!have_row || t >= u_end) {
        u = have_row ? u : row_of(g.n, t);
        while (row_start(g.n, u + 1) <= t) ++u;
        u_end = row_start(g.n, u + 1);
        have_row = true;
      }
      const unsigned long long v = u + 1 + (t - row_start(g.n, u));
      out[cnt] = (u << 32) | v;
    }
    ++cnt;
  }
  return cnt;
}

__global__ void k_gnp_count(GnpArgs g, unsigned long long *counts) {
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < g.chunks;
       c += (unsigned long long)gridDim.x * blockDim.x)
    counts[c] = walk_chunk(g, c, nullptr, false);
}

// Exclusive scan of the chunk counts by one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_gnp_scan(unsigned long long *counts, unsigned long long chunks,
                                                   unsigned long long *total) {
  __shared__ unsigned long long part[1024];
  const unsigned long long per = (chunks + 1023) / 1024;
  const unsigned long long b = min(threadIdx.x * per, chunks), e = min(b + per, chunks);
  unsigned long long sum = 0;
  for (unsigned long long c = b; c < e; ++c) sum += counts[c];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    const unsigned long long v = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = part[threadIdx.x] - sum;
  for (unsigned long long c = b; c < e; ++c) {
    const unsigned long long x = counts[c];
    counts[c] = run;
    run += x;
  }
  if (threadIdx.x == 1023) *total = part[1023];
}

__global__ void k_gnp_write(GnpArgs g, const unsigned long long *offsets, unsigned long long *out) {
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < g.chunks;
       c += (unsigned long long)gridDim.x * blockDim.x)
    walk_chunk(g, c, out + offsets[c], true);
}

}  // namespace
}  // namespace gesmc

extern "C" int gesmc_generate_gnp(uint64_t n, double p, uint64_t seed, uint64_t *out, uint64_t capacity,
                                  uint64_t *m_out, void *stream) {
  using namespace gesmc;
  if (!m_out || n < 2 || n > (1ull << 31) || !(p >= 0.0 && p <= 1.0) || (capacity > 0 && !out)) return -1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GnpArgs g;
  g.n = n;
  g.pairs = n * (n - 1) / 2;
  g.seed = seed;
  g.all = p >= 1.0 ? 1 : 0;
  if (p <= 0.0) {
    *m_out = 0;
    return 0;
  }
  g.log_q = g.all ? 0.0 : log1p(-p);
  const double want = ceil(128.0 / p);
  g.chunk = want >= (double)g.pairs ? g.pairs : (unsigned long long)want;
  if (g.chunk == 0) g.chunk = 1;
  g.chunks = (g.pairs + g.chunk - 1) / g.chunk;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return -6;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  unsigned long long *scratch = nullptr;
  if (cudaMallocAsync(&scratch, 8 * (g.chunks + 1), s) != cudaSuccess) {
    cudaGetLastError();
    return -6;
  }
  unsigned long long *counts = scratch, *total = scratch + g.chunks;
  const unsigned long long blocks = min((g.chunks + 255) / 256, (unsigned long long)sms * 16);
  k_gnp_count<<<(unsigned)(blocks ? blocks : 1), 256, 0, s>>>(g, counts);
  k_gnp_scan<<<1, 1024, 0, s>>>(counts, g.chunks, total);
  unsigned long long m = 0;
  bool ok = cudaMemcpyAsync(&m, total, 8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaStreamSynchronize(s) == cudaSuccess;
  int rc = ok ? 0 : -6;
  if (ok) {
    *m_out = m;
    if (m > capacity) {
      rc = -5;
    } else if (m > 0) {
      k_gnp_write<<<(unsigned)(blocks ? blocks : 1), 256, 0, s>>>(g, counts, reinterpret_cast<unsigned long long *>(out));
      ok = cudaStreamSynchronize(s) == cudaSuccess;
      if (!ok) rc = -6;
    }
  }
  cudaFreeAsync(scratch, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = -6;
  return rc;
}
