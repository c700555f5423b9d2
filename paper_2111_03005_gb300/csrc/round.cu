// One global switch round (Def. 2 of arXiv 2111.03005) on one GB300.
//
// Steps (the round of Algorithm 3, with Algorithm 1 as its superstep):
//   k_clear      empty the dependency table T, switch statuses, bucket counts
//   k_hist       Philox keys of all positions -> bucket histogram
//   k_scan       bucket offsets
//   k_scatter    positions into buckets (32 further key bits carried along)
//   k_sortpair   per bucket: exact in-shared-memory sort by (key, position),
//                then for every pair of consecutive slots (one edge switch,
//                Def. 1) gather both source edges, apply tau and the loop
//                rule, and record the four tuples of Algorithm 1 in T
//   k_boundary   the same for pairs whose two slots lie in different buckets
//   k_decide1    wave 1 of the decide/delay loop over all switches: decide
//                what is decidable, rewire legal switches, list the rest
//   k_tail       waves 2, 3, ... until no switch is undecided
//
// The waves are Jacobi steps: a switch decided in wave w only uses decisions
// of waves < w (status words carry their wave), so the result and the wave
// count do not depend on thread timing.  The edge list after the round is
// the one the sequential loop of Def. 2 produces.
#include "gesmc_internal.cuh"

namespace gesmc {
namespace {

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

// Permutation keys of positions 4b .. 4b+3 of round `round`.
__device__ __forceinline__ U64x4 perm_block(unsigned long long seed, unsigned long long round, unsigned long long b) {
  return philox(b, round, 0, 0, seed, 0);
}

// Word t of a block, t in 0..3 (selects, so the block stays in registers).
__device__ __forceinline__ unsigned long long word_of(const U64x4 &w, uint32_t t) {
  const unsigned long long lo = (t & 1) ? w.w[1] : w.w[0];
  const unsigned long long hi = (t & 1) ? w.w[3] : w.w[2];
  return (t & 2) ? hi : lo;
}

__device__ __forceinline__ unsigned long long perm_key(unsigned long long seed, unsigned long long round,
                                                       uint32_t i) {
  return word_of(perm_block(seed, round, i >> 2), i & 3);
}

__device__ __forceinline__ bool is_lazy(const RoundArgs &a, uint32_t k) {
  if (a.lazy_threshold == 0) return false;
  return word_of(philox(k >> 2, a.round, 1, 0, a.seed, 0), k & 3) < a.lazy_threshold;
}

__device__ __forceinline__ uint32_t bucket_of(unsigned long long key, uint32_t B) {
  return B ? (uint32_t)(key >> (64 - B)) : 0u;
}

// The 32 key bits after the bucket bits.
__device__ __forceinline__ uint32_t mid_of(unsigned long long key, uint32_t B) {
  return (uint32_t)((key << B) >> 32);
}

// ---------------------------------------------------------------- table T
__device__ __forceinline__ unsigned long long mix64(unsigned long long k) {
  // MurmurHash3's 64-bit finaliser (Appleby): a bijective avalanche mixer
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ unsigned long long home_slot(unsigned long long key, unsigned long long cap) {
  return __umul64hi(mix64(key), cap);
}

__device__ __forceinline__ unsigned long long ld_cg(const unsigned long long *p) { return __ldcg(p); }

// Slot holding `key`, claiming an empty one if the key is absent.  Returns
// cap if every slot was visited (table full; cannot happen when the table
// has more slots than keys).
__device__ __forceinline__ unsigned long long find_or_claim(Slot *T, unsigned long long cap, unsigned long long key) {
  unsigned long long s = home_slot(key, cap);
  for (unsigned long long n = 0; n < cap; ++n) {
    const unsigned long long cur = ld_cg(&T[s].key);
    if (cur == key) return s;
    if (cur == kEmptyKey) {
      const unsigned long long prev = atomicCAS(&T[s].key, kEmptyKey, key);
      if (prev == kEmptyKey || prev == key) return s;
    }
    if (++s == cap) s = 0;
  }
  return cap;
}

__device__ __forceinline__ unsigned long long pack_edge(uint32_t a, uint32_t b) {
  const uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
  return ((unsigned long long)lo << 32) | hi;
}

// Build switch k = (i, j, g = [i < j]) (Def. 2): gather its source edges,
// compute its targets with tau (Def. 1), and store Algorithm 1's tuples:
// (e1, k, ERASE), (e2, k, ERASE), (e3, k, INSERT), (e4, k, INSERT).
// Switches rejected outright (loop, shared node, lazy) store their sources
// as never erased and no targets.
__device__ __forceinline__ void build_switch(const RoundArgs &a, uint32_t k, uint32_t i, uint32_t j) {
  const unsigned long long e1 = __ldcg(&a.E[i]);
  const unsigned long long e2 = __ldcg(&a.E[j]);
  uint32_t code = 0;
  uint32_t a3 = 0, b3 = 0, a4 = 0, b4 = 0;
  if (is_lazy(a, k)) {
    code = kSwLazy;
  } else {
    const uint32_t u = (uint32_t)(e1 >> 32), v = (uint32_t)e1;
    const uint32_t x = (uint32_t)(e2 >> 32), y = (uint32_t)e2;
    if (i < j) {  // g = 1: (u, y), (v, x)
      a3 = u; b3 = y; a4 = v; b4 = x;
    } else {      // g = 0: (u, x), (v, y)
      a3 = u; b3 = x; a4 = v; b4 = y;
    }
    if (a3 == b3 || a4 == b4) code = kSwLoop;
    else if (u == x || u == y || v == x || v == y) code = kSwShared;
  }
  const uint32_t p = code ? kPKeep : k;
  const unsigned long long s1 = find_or_claim(a.T, a.cap, e1);
  const unsigned long long s2 = find_or_claim(a.T, a.cap, e2);
  unsigned long long s3 = 0, s4 = 0;
  if (!code) {
    s3 = find_or_claim(a.T, a.cap, pack_edge(a3, b3));
    s4 = find_or_claim(a.T, a.cap, pack_edge(a4, b4));
  }
  bool full = (s1 == a.cap) || (s2 == a.cap) || (!code && (s3 == a.cap || s4 == a.cap));
  if (full) {
    atomicOr(&a.ctl->err, kErrTableFull);
    a.sw[k] = make_uint4(i, j, kSwLoop, 0);  // keeps later kernels in bounds
    return;
  }
  a.T[s1].p = p;
  a.T[s2].p = p;
  if (!code) {
    atomicMin(&a.T[s3].q, k);
    atomicMin(&a.T[s4].q, k);
    a.sw[k] = make_uint4(i, j, (uint32_t)s3, (uint32_t)s4);
  } else {
    a.sw[k] = make_uint4(i, j, code, 0);
  }
}

// An edge of E that no switch of the round touches keeps p = kPKeep.
__device__ __forceinline__ void keep_source(const RoundArgs &a, uint32_t i) {
  const unsigned long long e = __ldcg(&a.E[i]);
  const unsigned long long s = find_or_claim(a.T, a.cap, e);
  if (s == a.cap) {
    atomicOr(&a.ctl->err, kErrTableFull);
    return;
  }
  a.T[s].p = kPKeep;
}

// ---------------------------------------------------------------- decide
__device__ __forceinline__ Slot load_slot(const Slot *p) {
  const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(p));
  Slot s;
  s.key = ((unsigned long long)v.y << 32) | v.x;
  s.p = v.z;
  s.q = v.w;
  return s;
}

constexpr int kOk = 0, kWait = 1, kBad = 2;

__device__ __forceinline__ bool decided_before(uint32_t st, uint32_t wave) {
  const uint32_t w = st >> 2;
  return w != 0 && w < wave;
}

// Algorithm 1's test of one target edge of switch k in wave `wave`, reading
// the table slot (p, q): kBad if the edge exists when k runs, kOk if it
// certainly does not, kWait if that depends on an undecided switch.
__device__ __forceinline__ int check_target(const RoundArgs &a, uint32_t k, uint32_t p, uint32_t q, uint32_t wave) {
  int res = kOk;
  if (p != kPNone) {             // the edge is in E at the start of the round
    if (p >= k) return kBad;     // erased later than k, or never
    const uint32_t sp = __ldcg(&a.status[p]);
    if (decided_before(sp, wave)) {
      if ((sp & 3u) == kIllegal) return kBad;  // its eraser failed: still there
    } else {
      res = kWait;
    }
  }
  if (q != k) {
    if (q < k) {                 // an earlier switch may insert it first
      const uint32_t sq = __ldcg(&a.status[q]);
      if (decided_before(sq, wave) && (sq & 3u) == kLegal) return kBad;
    }
    res = kWait;                 // q undecided, illegal but not yet replaced, or being replaced
  }
  return res;
}

struct Tally {
  uint32_t accepted = 0, rej_loop = 0, rej_exists = 0, lazy = 0;
};

// Decide switch k in wave `wave`.  Returns kOk (legal), kBad (illegal) or
// kWait.  Legal switches rewire E at once: positions i and j belong to k
// alone in this round, and their old values were read when k was built.
__device__ __forceinline__ int decide_one(const RoundArgs &a, uint32_t k, uint32_t wave, Tally &t) {
  const uint4 rec = __ldcg(&a.sw[k]);
  if (rec.z < kSwCodeMin && (rec.z >= a.cap || rec.w >= a.cap || rec.x >= a.m || rec.y >= a.m)) {
    // a record the round did not write (only after a reported bucket overflow)
    atomicOr(&a.ctl->err, kErrRecord);
    a.status[k] = (wave << 2) | kIllegal;
    return kBad;
  }
  if (rec.z >= kSwCodeMin) {
    a.status[k] = (wave << 2) | kIllegal;
    if (rec.z == kSwLazy) ++t.lazy;
    else if (rec.z == kSwLoop) ++t.rej_loop;
    else ++t.rej_exists;
    return kBad;
  }
  // through L2: inside k_tail the slots change between waves (atomics)
  const Slot s3 = load_slot(&a.T[rec.z]);
  const Slot s4 = load_slot(&a.T[rec.w]);
  const int r3 = check_target(a, k, s3.p, s3.q, wave);
  const int r4 = check_target(a, k, s4.p, s4.q, wave);
  if (r3 == kBad || r4 == kBad) {
    a.status[k] = (wave << 2) | kIllegal;
    // an illegal switch no longer counts as an inserter: if it was the
    // smallest one, clear the field; the waiting inserters re-register
    if (s3.q == k) atomicCAS(&a.T[rec.z].q, k, kQNone);
    if (s4.q == k) atomicCAS(&a.T[rec.w].q, k, kQNone);
    ++t.rej_exists;
    return kBad;
  }
  if (r3 == kWait || r4 == kWait) return kWait;
  a.E[rec.x] = s3.key;
  a.E[rec.y] = s4.key;
  a.status[k] = (wave << 2) | kLegal;
  ++t.accepted;
  return kOk;
}

__device__ __forceinline__ void flush_tally(const RoundArgs &a, Tally t) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    t.accepted += __shfl_down_sync(0xffffffffu, t.accepted, off);
    t.rej_loop += __shfl_down_sync(0xffffffffu, t.rej_loop, off);
    t.rej_exists += __shfl_down_sync(0xffffffffu, t.rej_exists, off);
    t.lazy += __shfl_down_sync(0xffffffffu, t.lazy, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (t.accepted) atomicAdd(&a.st->accepted, (unsigned long long)t.accepted);
    if (t.rej_loop) atomicAdd(&a.st->rej_loop, (unsigned long long)t.rej_loop);
    if (t.rej_exists) atomicAdd(&a.st->rej_exists, (unsigned long long)t.rej_exists);
    if (t.lazy) atomicAdd(&a.st->lazy, (unsigned long long)t.lazy);
  }
}

// Warp-aggregated append of k to a list (all lanes of the warp must call).
__device__ __forceinline__ void append_if(bool take, uint32_t k, uint32_t *list, uint32_t *count) {
  const unsigned mask = __ballot_sync(0xffffffffu, take);
  if (!mask) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (take) list[base + __popc(mask & ((1u << lane) - 1u))] = k;
}

// ---------------------------------------------------------------- kernels

__global__ void k_clear(RoundArgs a) {
  const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
  uint4 *T4 = reinterpret_cast<uint4 *>(a.T);
  const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
  for (unsigned long long s = tid; s < a.cap; s += nth) __stcg(&T4[s], ones);
  for (unsigned long long k = tid; k < a.L; k += nth) a.status[k] = 0;
  for (unsigned long long b = tid; b < a.nb; b += nth) a.bucket_cnt[b] = 0;
  if (tid == 0) {
    a.ctl->pending[0] = 0;
    a.ctl->pending[1] = 0;
    a.ctl->boundary = 0;
    a.ctl->waves = 0;
  }
}

constexpr int kHistSmem = 4096;

__global__ void k_hist(RoundArgs a) {
  __shared__ uint32_t h[kHistSmem];
  const bool local = a.nb <= kHistSmem;
  if (local) {
    for (uint32_t b = threadIdx.x; b < a.nb; b += blockDim.x) h[b] = 0;
    __syncthreads();
  }
  const uint32_t nblk = (a.m + 3) >> 2;
  for (uint32_t blk = blockIdx.x * blockDim.x + threadIdx.x; blk < nblk; blk += gridDim.x * blockDim.x) {
    const U64x4 w = perm_block(a.seed, a.round, blk);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (4 * blk + t < a.m) {
        const uint32_t b = bucket_of(w.w[t], a.B);
        if (local) atomicAdd(&h[b], 1u);
        else atomicAdd(&a.bucket_cnt[b], 1u);
      }
    }
  }
  if (local) {
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < a.nb; b += blockDim.x)
      if (h[b]) atomicAdd(&a.bucket_cnt[b], h[b]);
  }
}

// Exclusive scan of the bucket counts (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) k_scan(RoundArgs a) {
  __shared__ uint32_t part[1024];
  const uint32_t tid = threadIdx.x;
  const uint32_t per = (a.nb + 1023) / 1024;
  const uint32_t beg = min(tid * per, a.nb), end = min(beg + per, a.nb);
  uint32_t sum = 0;
  bool over = false;
  for (uint32_t b = beg; b < end; ++b) {
    const uint32_t c = a.bucket_cnt[b];
    sum += c;
    over |= c > (uint32_t)kBucketCap;
  }
  if (over) atomicOr(&a.ctl->err, kErrBucket);
  part[tid] = sum;
  __syncthreads();
  for (uint32_t d = 1; d < 1024; d <<= 1) {
    const uint32_t v = tid >= d ? part[tid - d] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  uint32_t run = part[tid] - sum;  // exclusive prefix
  for (uint32_t b = beg; b < end; ++b) {
    a.bucket_off[b] = run;
    a.cursor[b] = run;
    run += a.bucket_cnt[b];
  }
  if (tid == 1023) a.bucket_off[a.nb] = part[1023];
}

__global__ void k_scatter(RoundArgs a) {
  const uint32_t nblk = (a.m + 3) >> 2;
  for (uint32_t blk = blockIdx.x * blockDim.x + threadIdx.x; blk < nblk; blk += gridDim.x * blockDim.x) {
    const U64x4 w = perm_block(a.seed, a.round, blk);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint32_t i = 4 * blk + t;
      if (i < a.m) {
        const uint32_t b = bucket_of(w.w[t], a.B);
        const uint32_t pos = atomicAdd(&a.cursor[b], 1u);
        a.buf[pos] = ((unsigned long long)mid_of(w.w[t], a.B) << 32) | i;
      }
    }
  }
}

// In-place exclusive scan of n = 2^kSubBits counters by a CTA of
// kSortThreads threads (each owns a contiguous run of n / kSortThreads).
__device__ __forceinline__ void cta_exclusive_scan(uint32_t *h, uint32_t *warp_tot) {
  constexpr int n = 1 << kSubBits;
  constexpr int per = n / kSortThreads;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t loc[per];
  uint32_t sum = 0;
#pragma unroll
  for (int r = 0; r < per; ++r) {
    loc[r] = h[tid * per + r];
    sum += loc[r];
  }
  uint32_t incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < kSortThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, t, d);
      if (lane >= d) t += v;
    }
    if (lane < kSortThreads / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  uint32_t run = incl - sum + (warp ? warp_tot[warp - 1] : 0);
#pragma unroll
  for (int r = 0; r < per; ++r) {
    h[tid * per + r] = run;
    run += loc[r];
  }
}

__device__ __forceinline__ bool full_key_less(const RoundArgs &a, uint32_t i, uint32_t j) {
  const unsigned long long ki = perm_key(a.seed, a.round, i), kj = perm_key(a.seed, a.round, j);
  return ki < kj || (ki == kj && i < j);
}

// One CTA per bucket: exact sort of the bucket by (key, position), then the
// edge switches of every pair of consecutive slots inside the bucket.
__global__ void __launch_bounds__(kSortThreads) k_sortpair(RoundArgs a) {
  __shared__ unsigned long long sorted[kBucketCap];
  __shared__ uint32_t hist[1 << kSubBits];
  __shared__ uint32_t warp_tot[kSortThreads / 32];
  const int tid = threadIdx.x;
  constexpr int nsub = 1 << kSubBits;
  for (uint32_t b = blockIdx.x; b < a.nb; b += gridDim.x) {
    const uint32_t off = a.bucket_off[b];
    const uint32_t cnt = a.bucket_off[b + 1] - off;
    if (cnt > (uint32_t)kBucketCap) {  // reported by k_scan; the round is void
      continue;
    }
    for (int s = tid; s < nsub; s += kSortThreads) hist[s] = 0;
    unsigned long long v[kPerThread];
#pragma unroll
    for (int r = 0; r < kPerThread; ++r) {
      const uint32_t idx = tid + r * kSortThreads;
      v[r] = idx < cnt ? __ldcs(&a.buf[off + idx]) : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPerThread; ++r) {
      const uint32_t idx = tid + r * kSortThreads;
      if (idx < cnt) atomicAdd(&hist[(uint32_t)(v[r] >> (64 - kSubBits))], 1u);
    }
    __syncthreads();
    cta_exclusive_scan(hist, warp_tot);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPerThread; ++r) {
      const uint32_t idx = tid + r * kSortThreads;
      if (idx < cnt) {
        const uint32_t pos = atomicAdd(&hist[(uint32_t)(v[r] >> (64 - kSubBits))], 1u);
        sorted[pos] = v[r];
      }
    }
    __syncthreads();
    // hist[s] is now the end of sub-bucket s; sort each (a handful of items)
    for (int s = tid; s < nsub; s += kSortThreads) {
      const uint32_t beg = s ? hist[s - 1] : 0, end = hist[s];
      for (uint32_t x = beg + 1; x < end; ++x) {
        const unsigned long long val = sorted[x];
        uint32_t y = x;
        while (y > beg && sorted[y - 1] > val) {
          sorted[y] = sorted[y - 1];
          --y;
        }
        sorted[y] = val;
      }
    }
    __syncthreads();
    // equal 32-bit key parts: order those runs by the full key
    for (uint32_t t = tid; t + 1 < cnt; t += kSortThreads) {
      const uint32_t mt = (uint32_t)(sorted[t] >> 32);
      if ((uint32_t)(sorted[t + 1] >> 32) == mt && (t == 0 || (uint32_t)(sorted[t - 1] >> 32) != mt)) {
        uint32_t e = t + 2;
        while (e < cnt && (uint32_t)(sorted[e] >> 32) == mt) ++e;
        for (uint32_t x = t + 1; x < e; ++x) {
          const unsigned long long val = sorted[x];
          uint32_t y = x;
          while (y > t && full_key_less(a, (uint32_t)val, (uint32_t)sorted[y - 1])) {
            sorted[y] = sorted[y - 1];
            --y;
          }
          sorted[y] = val;
        }
      }
    }
    __syncthreads();
    // slots off .. off+cnt-1 now hold pi in order
    const uint32_t t0 = off & 1u;
    const uint32_t npairs = cnt > t0 ? (cnt - t0) >> 1 : 0;
    for (uint32_t pidx = tid; pidx < npairs; pidx += kSortThreads) {
      const uint32_t t = t0 + 2 * pidx;
      build_switch(a, (off + t) >> 1, (uint32_t)sorted[t], (uint32_t)sorted[t + 1]);
    }
    if (tid == 0 && cnt > 0) {
      if (t0 == 1) {  // slot off is the second of a pair started in an earlier bucket
        a.pib[off] = (uint32_t)sorted[0];
        const uint32_t idx = atomicAdd(&a.ctl->boundary, 1u);
        a.bnd[idx] = (off - 1) >> 1;
      }
      const uint32_t last = off + cnt - 1;
      if ((last & 1u) == 0) {  // first of a pair whose partner is in a later bucket
        if (last + 1 == a.m) keep_source(a, (uint32_t)sorted[cnt - 1]);  // odd m: unpaired
        else a.pib[last] = (uint32_t)sorted[cnt - 1];
      }
    }
    __syncthreads();
  }
}

__global__ void k_boundary(RoundArgs a) {
  const uint32_t n = a.ctl->boundary;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const uint32_t k = a.bnd[idx];
    const uint32_t i = a.pib[2 * k], j = a.pib[2 * k + 1];
    if (k >= a.L || i >= a.m || j >= a.m) {  // only after a reported bucket overflow
      atomicOr(&a.ctl->err, kErrRecord);
      continue;
    }
    build_switch(a, k, i, j);
  }
}

__global__ void k_decide1(RoundArgs a) {
  Tally t;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < a.L; base += stride) {
    const uint32_t k = base + threadIdx.x;
    int r = kOk;
    if (k < a.L) r = decide_one(a, k, 1u, t);
    append_if(k < a.L && r == kWait, k, a.list0, &a.ctl->pending[0]);
  }
  flush_tally(a, t);
}

// Waves 2, 3, ... on one CTA: undecided switches re-register as inserters
// (the table's q fields of illegal minima were cleared), then decide.
__global__ void __launch_bounds__(1024) k_tail(RoundArgs a) {
  __shared__ uint32_t s_n;
  Tally t;
  uint32_t cur = 0, wave = 2, prev_n = a.L + 1;
  volatile uint32_t *pend = a.ctl->pending;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_n = pend[cur];
    __syncthreads();
    const uint32_t n = s_n;
    if (n == 0) break;
    if (wave > (a.max_waves ? a.max_waves : kDefaultWaveCap)) {
      if (threadIdx.x == 0) atomicOr(&a.ctl->err, kErrWaveCap);
      break;
    }
    if (n >= prev_n) {  // no switch was decided in the last wave: impossible
      if (threadIdx.x == 0) atomicOr(&a.ctl->err, kErrNoProgress);
      break;
    }
    prev_n = n;
    const uint32_t *in = cur ? a.list1 : a.list0;
    uint32_t *out = cur ? a.list0 : a.list1;
    for (uint32_t idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const uint32_t k = in[idx];
      const uint4 rec = __ldcg(&a.sw[k]);
      if (rec.z < a.cap && rec.w < a.cap) {  // always true for a listed switch
        atomicMin(&a.T[rec.z].q, k);
        atomicMin(&a.T[rec.w].q, k);
      }
    }
    if (threadIdx.x == 0) {
      pend[cur ^ 1] = 0;
      if (wave < kWaveHist) a.st->last_pending[wave] = n;
    }
    __syncthreads();
    for (uint32_t base = 0; base < n; base += blockDim.x) {
      const uint32_t idx = base + threadIdx.x;
      int r = kOk;
      uint32_t k = 0;
      if (idx < n) {
        k = in[idx];
        r = decide_one(a, k, wave, t);
      }
      append_if(idx < n && r == kWait, k, out, (uint32_t *)&pend[cur ^ 1]);
    }
    cur ^= 1;
    ++wave;
  }
  flush_tally(a, t);
  if (threadIdx.x == 0) {
    const uint32_t waves = a.L ? wave - 1 : 0;
    a.ctl->waves = waves;
    a.st->waves_total += waves;
    if (waves > a.st->waves_max) a.st->waves_max = waves;
    a.st->wave_hist[waves < kWaveHist ? waves : kWaveHist - 1] += 1;
    a.st->last_pending[1] = a.L;
    for (uint32_t w = wave; w < kWaveHist; ++w) a.st->last_pending[w] = 0;
  }
}

// ---------------------------------------------------------------- create-time checks

__global__ void k_canonicalise(unsigned long long *E, uint32_t m, unsigned long long n_bound, uint32_t *flags,
                               uint32_t *max_id) {
  uint32_t f = 0, mx = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const unsigned long long e = E[i];
    const uint32_t x = (uint32_t)(e >> 32), y = (uint32_t)e;
    if (x == y) f |= kFlagLoop;
    if (n_bound && (x >= n_bound || y >= n_bound)) f |= kFlagRange;
    mx = max(mx, max(x, y));
    E[i] = pack_edge(x, y);
  }
  if (f) atomicOr(flags, f);
  if (m) atomicMax(max_id, mx);
}

__global__ void k_duplicates(const unsigned long long *E, uint32_t m, Slot *T, unsigned long long cap,
                             uint32_t *flags) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const unsigned long long key = E[i];
    unsigned long long s = home_slot(key, cap);
    bool placed = false;
    for (unsigned long long n = 0; n < cap && !placed; ++n) {
      const unsigned long long prev = atomicCAS(&T[s].key, kEmptyKey, key);
      if (prev == kEmptyKey) placed = true;
      else if (prev == key) {
        atomicOr(flags, kFlagMulti);
        placed = true;
      } else if (++s == cap) {
        s = 0;
      }
    }
    if (!placed) atomicOr(flags, kFlagTableFull);
  }
}

__global__ void k_clear_table(Slot *T, unsigned long long cap) {
  uint4 *T4 = reinterpret_cast<uint4 *>(T);
  const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
  for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s < cap;
       s += (unsigned long long)gridDim.x * blockDim.x)
    T4[s] = ones;
}

inline int grid_for(unsigned long long work, int threads, int num_sms, int per_sm) {
  unsigned long long g = (work + threads - 1) / threads;
  const unsigned long long lim = (unsigned long long)num_sms * per_sm;
  if (g > lim) g = lim;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t launch_round(const RoundArgs &a, cudaStream_t s, int num_sms, cudaEvent_t *ev, uint32_t *launches) {
  // ev (optional) receives kNumStages + 1 stage boundaries; stages that do
  // not run for tiny m still get both of their events (zero duration).
  auto mark = [&](int stage) {
    if (ev) cudaEventRecord(ev[stage], s);
  };
  uint32_t n = 0;
  const unsigned long long clear_work = a.cap > a.L ? a.cap : a.L;
  const bool work = a.m >= 2;
  const uint32_t nblk = (a.m + 3) / 4;
  mark(kStageClear);
  k_clear<<<grid_for(clear_work, 256, num_sms, 16), 256, 0, s>>>(a);
  ++n;
  mark(kStageHist);
  if (work) { k_hist<<<grid_for(nblk, 256, num_sms, 8), 256, 0, s>>>(a); ++n; }
  mark(kStageScan);
  if (work) { k_scan<<<1, 1024, 0, s>>>(a); ++n; }
  mark(kStageScatter);
  if (work) { k_scatter<<<grid_for(nblk, 256, num_sms, 8), 256, 0, s>>>(a); ++n; }
  mark(kStageSortPair);
  if (work) { k_sortpair<<<a.nb, kSortThreads, 0, s>>>(a); ++n; }
  mark(kStageBoundary);
  if (work) { k_boundary<<<grid_for(a.nb, 256, num_sms, 2), 256, 0, s>>>(a); ++n; }
  mark(kStageDecide1);
  if (work) { k_decide1<<<grid_for(a.L, 256, num_sms, 16), 256, 0, s>>>(a); ++n; }
  mark(kStageTail);
  if (work) { k_tail<<<1, 1024, 0, s>>>(a); ++n; }
  mark(kNumStages);
  if (launches) *launches += n;
  return cudaGetLastError();
}

cudaError_t launch_canonicalise(unsigned long long *E, uint32_t m, unsigned long long n_bound, uint32_t *flags,
                                uint32_t *max_id, cudaStream_t s, int num_sms) {
  k_canonicalise<<<grid_for(m, 256, num_sms, 8), 256, 0, s>>>(E, m, n_bound, flags, max_id);
  return cudaGetLastError();
}

cudaError_t launch_duplicate_check(const unsigned long long *E, uint32_t m, Slot *T, unsigned long long cap,
                                   uint32_t *flags, cudaStream_t s, int num_sms) {
  k_duplicates<<<grid_for(m, 256, num_sms, 8), 256, 0, s>>>(E, m, T, cap, flags);
  return cudaGetLastError();
}

cudaError_t launch_clear_table(Slot *T, unsigned long long cap, cudaStream_t s, int num_sms) {
  k_clear_table<<<grid_for(cap, 256, num_sms, 16), 256, 0, s>>>(T, cap);
  return cudaGetLastError();
}

}  // namespace gesmc
