// Device helpers shared by the kernels of libgesmc (global switch rounds and
// ParES): the Philox4x64-10 generator, the 64-bit mixer that picks hash
// slots, canonical edge ids and the edge switch tau of Def. 1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gesmc {

// ---------------------------------------------------------------- Philox4x64-10
// Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11): ten
// rounds, each multiplying counter words 0 and 2 by fixed 64-bit constants,
// xor-ing the high halves into words 1 and 3 with the round key, and
// permuting; the key is advanced by two Weyl increments between rounds.
struct U64x4 {
  unsigned long long w[4];
};

__device__ __forceinline__ U64x4 philox(unsigned long long c0, unsigned long long c1, unsigned long long c2,
                                        unsigned long long c3, unsigned long long k0, unsigned long long k1) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const unsigned long long n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  U64x4 out;
  out.w[0] = c0;
  out.w[1] = c1;
  out.w[2] = c2;
  out.w[3] = c3;
  return out;
}

// Word t of a block, t in 0..3 (selects, so the block stays in registers).
__device__ __forceinline__ unsigned long long word_of(const U64x4 &w, uint32_t t) {
  const unsigned long long lo = (t & 1) ? w.w[1] : w.w[0];
  const unsigned long long hi = (t & 1) ? w.w[3] : w.w[2];
  return (t & 2) ? hi : lo;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long k) {
  // MurmurHash3's 64-bit finaliser (Appleby): a bijective avalanche mixer
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ unsigned long long pack_edge(uint32_t a, uint32_t b) {
  const uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
  return ((unsigned long long)lo << 32) | hi;
}

// Edge switch with direction bit g on e1 = (u, v), e2 = (x, y) (Def. 1):
// g = 0 gives (u, x), (v, y); g = 1 gives (u, y), (v, x), as canonical ids
// e3, e4.  Returns the outright-reject code: a new edge is a loop, or the
// sources share a node (then every outcome of tau is a loop or re-creates
// the two source edges, which are in E when the switch runs); else 0.
__device__ __forceinline__ uint32_t tau_g(uint32_t g, unsigned long long e1, unsigned long long e2,
                                          unsigned long long &e3, unsigned long long &e4) {
  const uint32_t u = (uint32_t)(e1 >> 32), v = (uint32_t)e1;
  const uint32_t x = (uint32_t)(e2 >> 32), y = (uint32_t)e2;
  const uint32_t a3 = u, b3 = g ? y : x, a4 = v, b4 = g ? x : y;
  e3 = pack_edge(a3, b3);
  e4 = pack_edge(a4, b4);
  if (a3 == b3 || a4 == b4) return 1u;  // a loop
  if (u == x || u == y || v == x || v == y) return 2u;  // shared node
  return 0;
}

// ---------------------------------------------------------------- bulk copies
// One-dimensional bulk copy (the TMA engine, cp.async.bulk) of `bytes` from
// global memory into this CTA's shared memory, completing on an mbarrier.
// Addresses must be 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The barrier's memory may be put to another use after this.
__device__ __forceinline__ void mbar_inval(unsigned long long *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// The calling thread arrives and announces `bytes` of copies that complete
// on the barrier's current phase.
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bulk prefetch of `bytes` of global memory into L2 (no destination, no
// completion to wait for); 16-byte aligned address, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Wait for phase `parity` of the barrier to complete, at most `limit` polls;
// false if it did not (the caller reports an error instead of spinning on).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, uint32_t limit) {
  const uint32_t addr = smem_addr(bar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace gesmc
