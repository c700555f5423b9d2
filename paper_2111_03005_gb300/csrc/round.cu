// One global switch round (Def. 2 of arXiv 2111.03005) of every chain of a
// pool, on one GB300, laid out as streaming passes so that no step needs a
// random DRAM access per switch.
//
//   k_clear          zero the per-round counters
//   k_permute        read the list in last-round slot order (applying the
//                    last round's legal switches on the fly), compute each
//                    position's Philox key and append (key bits, position,
//                    edge) to its bucket; the buckets' write frontiers stay
//                    in L2, so DRAM sees whole lines
//   k_scan_perm      bucket slot offsets
//   k_sortpair       per bucket: exact sort by (key, position) in shared
//                    memory; write the list back in this round's slot order;
//                    for each pair of slots (edge switch sigma_k, Def. 1)
//                    apply tau, the loop and shared-node rules and laziness,
//                    and append Algorithm 1's four tuples (e1, k, ERASE),
//                    (e2, k, ERASE), (e3, k, INSERT), (e4, k, INSERT) to
//                    the hash partitions of their edge ids
//   k_boundary       the same for pairs whose slots lie in two buckets
//   k_sources        the sources (ERASE tuples) of all switches, from the
//                    list in slot order, but only those whose edge id some
//                    target of the round may equal (target filter)
//   k_overflow_*     group the (rare) tuples that found their partition full
//   k_group          per partition: group by edge id in a shared-memory
//                    table and decide every target of wave 1 (Algorithm 1's
//                    first round): certainly present, free, or dependent on
//                    an undecided switch; edge ids with a dependency get an
//                    entry {p, q} for the later waves
//   k_wave1          per switch: legal, illegal or pending
//   k_wave_register  waves 2, 3, ... over the pending switches on the whole
//   k_wave_decide    GPU, one pair of kernels per wave
//   k_tail           any remaining waves, on one CTA
//
// The waves are Jacobi steps: a switch decided in wave w only uses decisions
// of waves < w (status words carry their wave), so the result and the wave
// count do not depend on thread timing.  The list after the round is the one
// the sequential loop of Def. 2 produces.
#include <algorithm>

#include "device_util.cuh"
#include "gesmc_internal.cuh"

namespace gesmc {
namespace {

// Permutation key K(i) of round `round` (purpose 0).
__device__ __forceinline__ unsigned long long perm_key(unsigned long long seed, unsigned long long round,
                                                       uint32_t i) {
  return word_of(philox(i >> 2, round, 0, 0, seed, 0), i & 3);
}

__device__ __forceinline__ uint32_t bucket_of(unsigned long long key, uint32_t B) {
  return B ? (uint32_t)(key >> (64 - B)) : 0u;
}

// The 32 key bits after the bucket bits.
__device__ __forceinline__ uint32_t mid_of(unsigned long long key, uint32_t B) {
  return (uint32_t)((key << B) >> 32);
}

// ---------------------------------------------------------------- edges
__device__ __forceinline__ uint32_t partition_of(unsigned long long h, uint32_t P) {
  return P ? (uint32_t)(h >> (64 - P)) : 0u;
}

// Edge switch (i, j, g = [i < j]) of a global switch (Def. 2): tau with the
// direction bit the permutation gives.
__device__ __forceinline__ uint32_t tau(uint32_t i, uint32_t j, unsigned long long e1, unsigned long long e2,
                                        unsigned long long &e3, unsigned long long &e4) {
  return tau_g(i < j ? 1u : 0u, e1, e2, e3, e4);
}


// ---------------------------------------------------------------- chains
// Round number of a chain in the current pool round, and whether status[]
// holds decisions of the chain's last round that still have to be applied.
__device__ __forceinline__ unsigned long long chain_round(const ChainDesc &ch, unsigned long long pool_round) {
  return ch.start_round + (pool_round - ch.join);
}
__device__ __forceinline__ bool chain_apply(const ChainDesc &ch, unsigned long long pool_round) {
  return pool_round > ch.added;
}

// Laziness word of switch k (the chain's own index): Philox, purpose 1.
__device__ __forceinline__ unsigned long long lazy_word(const ChainDesc &ch, unsigned long long round, uint32_t k) {
  return word_of(philox(k >> 2, round, 1, 0, ch.seed, 0), k & 3);
}

// Laziness (Def. 2, P_L).  Per-switch form: switch k is skipped iff its word
// is below the chain's threshold.  Exact l: the round runs its first ell
// switches only, ell = the number of words that pass (counted beforehand).
__device__ __forceinline__ bool is_lazy(const ChainDesc &ch, unsigned long long round, uint32_t k, uint32_t ell) {
  if (ch.lazy_threshold == 0) return false;
  if (ch.exact_ell) return k >= ell;
  return lazy_word(ch, round, k) < ch.lazy_threshold;
}

// The values of slots 2k, 2k+1 of a chain at the start of this round: the
// chain's last-round switch k rewired them if it was legal.
__device__ __forceinline__ void apply_last(const RoundArgs &a, const ChainDesc &ch, bool apply, uint32_t k,
                                           uint32_t i, uint32_t j, unsigned long long &e1, unsigned long long &e2) {
  if (apply && k < ch.L && (__ldcs(&a.status[ch.switch_base + k]) & 3u) == kLegal) {
    unsigned long long e3, e4;
    tau(i, j, e1, e2, e3, e4);
    e1 = e3;
    e2 = e4;
  }
}

// ---------------------------------------------------------------- build
// Append tuples to their hash partitions: partition ids and cursor atomics
// first (independent, in flight together), then the 16-byte stores.  A
// tuple in its partition is {id lo, id hi, value, low 32 bits of the id's
// hash} (the grouping kernel probes its table with those bits); one that
// finds its partition full goes to the overflow list with its partition id
// in place of the hash bits.
// The target filter's bit of an edge id with hash h.
__device__ __forceinline__ uint32_t filter_bit(const RoundArgs &a, unsigned long long h) {
  return (uint32_t)(h >> 24) & a.tfilter_mask;
}

template <int N>
__device__ __forceinline__ void emit_tuples(const RoundArgs &a, const ChainDesc &ch,
                                            const unsigned long long (&key)[N], const unsigned long long (&hash)[N],
                                            const uint32_t (&val)[N]) {
  uint32_t part[N], hlo[N], idx[N];
#pragma unroll
  for (int t = 0; t < N; ++t) {
    const unsigned long long h = hash[t];
    part[t] = partition_of(h, ch.P);
    hlo[t] = (uint32_t)h;
    idx[t] = key[t] != kEmptyKey ? atomicAdd(&a.tcount[ch.tcount_base + part[t] * ch.tstride], 1u) : 0u;
  }
#pragma unroll
  for (int t = 0; t < N; ++t) {
    if (key[t] == kEmptyKey) continue;
    if (idx[t] < ch.capt) {
      a.ptup[ch.tuple_base + (size_t)part[t] * ch.capt + idx[t]] =
          make_uint4((uint32_t)key[t], (uint32_t)(key[t] >> 32), val[t], hlo[t]);
    } else {
      const uint32_t o = atomicAdd(&a.ctl->ovf_count, 1u);
      if (o < a.ovf_cap)
        a.otup[o] = make_uint4((uint32_t)key[t], (uint32_t)(key[t] >> 32), val[t], ch.part_base + part[t]);
      else
        atomicOr(&a.ctl->err, kErrRecord);
    }
  }
}

// Switches k[t] (the chain's own indices; t < N, those with valid[t]) =
// (i, j, g) with sources e1, e2: record each reject code, mark the targets
// in the target filter and emit Algorithm 1's tuples (e3, k, INSERT),
// (e4, k, INSERT), with k made pool-wide; all N switches' atomics are in
// flight together.  Their ERASE tuples (e1, k), (e2, k) follow from
// k_sources when the filter says a target may need them.  A switch rejected
// outright has no targets.
template <int N>
__device__ __forceinline__ void build_switches(const RoundArgs &a, const ChainDesc &ch, unsigned long long round,
                                               uint32_t ell, const bool (&valid)[N], const uint32_t (&k)[N],
                                               const uint32_t (&i)[N], const unsigned long long (&e1)[N],
                                               const uint32_t (&j)[N], const unsigned long long (&e2)[N]) {
  unsigned long long key[2 * N], hash[2 * N];
  uint32_t val[2 * N];
#pragma unroll
  for (int t = 0; t < N; ++t) {
    unsigned long long e3 = kEmptyKey, e4 = kEmptyKey;
    const uint32_t kg = ch.switch_base + k[t];
    if (valid[t]) {
      const uint32_t code = is_lazy(ch, round, k[t], ell) ? kCodeLazy : tau(i[t], j[t], e1[t], e2[t], e3, e4);
      a.word[kg] = code;
      a.sw[kg] = make_uint2(kTrivial, kTrivial);
      if (code) e3 = e4 = kEmptyKey;
    }
    key[2 * t] = e3;
    key[2 * t + 1] = e4;
    val[2 * t] = kg;
    val[2 * t + 1] = kg | kTupleWhich;
  }
#pragma unroll
  for (int t = 0; t < 2 * N; ++t) {
    hash[t] = mix64(key[t]);
    if (key[t] != kEmptyKey) {
      const uint32_t fb = filter_bit(a, hash[t]);
      atomicOr(&a.tfilter[fb >> 5], 1u << (fb & 31));
    }
  }
  emit_tuples<2 * N>(a, ch, key, hash, val);
}

// ---------------------------------------------------------------- decide
constexpr int kOk = 0, kWait = 1, kBad = 2;

__device__ __forceinline__ bool decided_before(uint32_t st, uint32_t wave) {
  const uint32_t w = st >> 2;
  return w != 0 && w < wave;
}

// Algorithm 1's test of one target edge of switch k in wave `wave` >= 2,
// from its dependency entry (p, q): kBad if the edge exists when k runs,
// kOk if it certainly does not, kWait if that depends on an undecided switch.
__device__ __forceinline__ int check_target(const RoundArgs &a, uint32_t k, uint32_t d, uint32_t wave) {
  if (d == kTrivial) return kOk;
  const uint2 pq = __ldcg(&a.dep[d]);
  const uint32_t p = pq.x, q = pq.y;
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

// An illegal switch no longer counts as an inserter: where it was the
// smallest one, clear the field; the waiting inserters re-register.
__device__ __forceinline__ void drop_inserter(const RoundArgs &a, uint32_t k, uint2 s) {
  if (s.x != kTrivial && __ldcg(&a.dep[s.x].y) == k) atomicCAS(&a.dep[s.x].y, k, kQNone);
  if (s.y != kTrivial && __ldcg(&a.dep[s.y].y) == k) atomicCAS(&a.dep[s.y].y, k, kQNone);
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

// Per-chain count of accepted switches: each thread keeps a running count
// for the chain it last saw and hands it on when the chain changes; at the
// end, lanes of a warp holding the same chain add once (all lanes call).
struct ChainCount {
  uint32_t chain = kNoChain, n = 0;
};

__device__ __forceinline__ void count_accepted(const RoundArgs &a, ChainCount &cc, uint32_t chain) {
  if (chain != cc.chain) {
    if (cc.n) atomicAdd(&a.chain_accepted[cc.chain], (unsigned long long)cc.n);
    cc.chain = chain;
    cc.n = 0;
  }
  ++cc.n;
}

__device__ __forceinline__ void flush_count(const RoundArgs &a, const ChainCount &cc) {
  const unsigned same = __match_any_sync(0xffffffffu, cc.n ? cc.chain : kNoChain);
  unsigned long long n = cc.n;
  // sum n over the lanes of this group, result at its first lane
  const int lane = threadIdx.x & 31;
  unsigned long long total = 0;
  for (unsigned rest = same; rest; rest &= rest - 1) total += __shfl_sync(same, n, __ffs(rest) - 1);
  if (cc.n && (__ffs(same) - 1) == lane) atomicAdd(&a.chain_accepted[cc.chain], total);
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

__device__ __forceinline__ void clear_body(const RoundArgs &a) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (uint32_t b = tid; b < a.bucket_hw; b += nth) a.pcount[b] = 0;
  for (uint32_t p = tid; p < a.part_hw; p += nth) a.ocount[p] = 0;
  for (uint32_t p = tid; p < a.tcount_hw; p += nth) a.tcount[p] = 0;
  for (uint32_t c = tid; c < a.chain_hw; c += nth) a.chain_ell[c] = 0;
  if (tid == 0) {
    a.ctl->pending[0] = 0;
    a.ctl->pending[1] = 0;
    a.ctl->boundary = 0;
    a.ctl->waves = 0;
    a.ctl->dep_count = 0;
    a.ctl->ovf_count = 0;
    a.ctl->cur = 0;
    a.ctl->wave_next = 2;
    a.ctl->wave_blocks = 0;
  }
}

__global__ void k_clear(RoundArgs a) { clear_body(a); }

__device__ __forceinline__ void store_record(const RoundArgs &a, uint32_t b, uint32_t idx, uint32_t keybits,
                                             uint32_t pos, unsigned long long e) {
  if (idx < (1u << a.bucket_log2))
    a.prec[((size_t)b << a.bucket_log2) + idx] = make_uint4(keybits, pos, (uint32_t)e, (uint32_t)(e >> 32));
  else
    atomicOr(&a.ctl->err, kErrBucket);
}

// The positions of the chain with few buckets (a pool of one chain with at
// most kAggBuckets buckets), each CTA taking kAggThreads * kAggPairs
// consecutive pairs of slots: the CTA counts its records per bucket in
// shared memory (a record's rank among the CTA's records of its bucket comes
// with it), takes each bucket's range with one cursor atomic, then stores
// its records (keys recomputed).  With few buckets every cursor takes
// thousands of same-address atomics per round, which serialise in L2; here
// it takes one per CTA.  The order of records inside a bucket does not
// matter: the sort orders them by key and position.
constexpr int kAggThreads = 1024, kAggPairs = 2;

// The pair of slots x of the chain (its position and edge pair with the last
// round's decision applied, and the keys).
__device__ __forceinline__ void agg_pair(const RoundArgs &a, const ChainDesc &ch, unsigned long long R,
                                         unsigned long long round, uint32_t x, bool &two, uint32_t (&pos)[2],
                                         unsigned long long (&e)[2], unsigned long long (&K)[2]) {
  const uint32_t gx = (ch.slot_base >> 1) + x;  // pair index in the pool's slots
  two = 2 * x + 1 < ch.m;
  if (two) {
    const uint2 ij = __ldcs(reinterpret_cast<const uint2 *>(a.cpos) + gx);
    const ulonglong2 ee = __ldcs(reinterpret_cast<const ulonglong2 *>(a.cedge) + gx);
    e[0] = ee.x;
    e[1] = ee.y;
    apply_last(a, ch, chain_apply(ch, R), x, ij.x, ij.y, e[0], e[1]);
    pos[0] = ij.x;
    pos[1] = ij.y;
  } else {  // odd m: the chain's last slot has no partner
    pos[0] = a.cpos[2 * gx];
    e[0] = a.cedge[2 * gx];
    pos[1] = 0;
    e[1] = 0;
  }
  K[0] = perm_key(ch.seed, round, pos[0]);
  K[1] = two ? perm_key(ch.seed, round, pos[1]) : 0ull;
}

__global__ void __launch_bounds__(kAggThreads, 1) k_permute_agg(RoundArgs a) {
  __shared__ uint32_t sc[kAggBuckets];  // per bucket: the CTA's count, then its base
  const ChainDesc ch = a.chains[a.agg_chain];
  const unsigned long long R = a.ctl->pool_round;
  const unsigned long long round = chain_round(ch, R);
  const uint32_t tid = threadIdx.x, nb = 1u << ch.B, npair = (ch.m + 1) >> 1;
  const uint32_t x0 = blockIdx.x * (kAggThreads * kAggPairs) + tid;
  for (uint32_t b = tid; b < nb; b += kAggThreads) sc[b] = 0;
  __syncthreads();
  uint32_t bk[2 * kAggPairs], rk[2 * kAggPairs];
#pragma unroll
  for (int j = 0; j < kAggPairs; ++j) {
    const uint32_t x = x0 + j * kAggThreads;
    bk[2 * j] = bk[2 * j + 1] = kNoChain;
    if (x >= npair) continue;
    bool two;
    uint32_t pos[2];
    unsigned long long e[2], K[2];
    agg_pair(a, ch, R, round, x, two, pos, e, K);
    bk[2 * j] = bucket_of(K[0], ch.B);
    rk[2 * j] = atomicAdd(&sc[bk[2 * j]], 1u);
    if (two) {
      bk[2 * j + 1] = bucket_of(K[1], ch.B);
      rk[2 * j + 1] = atomicAdd(&sc[bk[2 * j + 1]], 1u);
    }
  }
  __syncthreads();
  for (uint32_t b = tid; b < nb; b += kAggThreads) {
    const uint32_t n = sc[b];
    if (n) sc[b] = atomicAdd(&a.pcount[ch.bucket_base + b], n);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kAggPairs; ++j) {
    const uint32_t x = x0 + j * kAggThreads;
    if (x >= npair) continue;
    bool two;
    uint32_t pos[2];
    unsigned long long e[2], K[2];
    agg_pair(a, ch, R, round, x, two, pos, e, K);
    store_record(a, ch.bucket_base + bk[2 * j], sc[bk[2 * j]] + rk[2 * j], mid_of(K[0], ch.B), pos[0], e[0]);
    if (two)
      store_record(a, ch.bucket_base + bk[2 * j + 1], sc[bk[2 * j + 1]] + rk[2 * j + 1], mid_of(K[1], ch.B), pos[1],
                   e[1]);
  }
}

// Exact l (Def. 2 as printed): per chain in that mode, the number of its
// switches whose laziness word passes (>= threshold); the round then runs
// the chain's first l switches.  Each CTA takes a contiguous range of
// switches and each thread keeps a running count for its current chain.
__device__ __forceinline__ void lazy_count_body(const RoundArgs &a) {
  const unsigned long long R = a.ctl->pool_round;
  const uint32_t per = (a.switch_hw + gridDim.x - 1) / gridDim.x;
  const uint32_t chunk = (per + blockDim.x - 1) / blockDim.x * blockDim.x;
  const uint32_t beg = min(blockIdx.x * chunk, a.switch_hw), end = min(beg + chunk, a.switch_hw);
  uint32_t cur = kNoChain, n = 0;
  for (uint32_t k = beg + threadIdx.x; k < end; k += blockDim.x) {
    const uint32_t c = a.owner_switch[k];
    if (c == kNoChain) continue;
    const ChainDesc ch = a.chains[c];
    if (!ch.exact_ell || ch.lazy_threshold == 0) continue;
    if (c != cur) {
      if (n) atomicAdd(&a.chain_ell[cur], n);
      cur = c;
      n = 0;
    }
    n += lazy_word(ch, chain_round(ch, R), k - ch.switch_base) >= ch.lazy_threshold ? 1u : 0u;
  }
  if (n) atomicAdd(&a.chain_ell[cur], n);
}

__global__ void k_lazy_count(RoundArgs a) { lazy_count_body(a); }

// Append every position, with its current edge, to its chain's bucket.
// Five CTAs of 256 per SM (48 registers, no spills): 3.16 ms per round on
// G(2^24) against 3.20 with six (40 registers and a few spilled) and 3.29
// with eight (32).  The round launches one pair per thread (short-lived
// CTAs): that measured 3.13 ms against 3.46 ms for a grid-stride loop over
// 8 CTAs per SM and 4.05 ms over one resident wave; the loop form serves the
// one-launch round.
__device__ __forceinline__ void permute_pair(const RoundArgs &a, uint32_t x, unsigned long long R) {
  const uint32_t s0 = 2 * x;
  const uint32_t c = a.owner_slot[s0];
  if (c == kNoChain) return;
  const ChainDesc ch = a.chains[c];
  const unsigned long long round = chain_round(ch, R);
  const uint32_t ls = s0 - ch.slot_base;
  if (ls + 1 < ch.m) {
    const uint2 ij = __ldcs(reinterpret_cast<const uint2 *>(a.cpos) + x);
    const ulonglong2 ee = __ldcs(reinterpret_cast<const ulonglong2 *>(a.cedge) + x);
    unsigned long long e1 = ee.x, e2 = ee.y;
    apply_last(a, ch, chain_apply(ch, R), ls >> 1, ij.x, ij.y, e1, e2);
    // both keys and both atomics before the two stores
    const unsigned long long K1 = perm_key(ch.seed, round, ij.x);
    const unsigned long long K2 = perm_key(ch.seed, round, ij.y);
    const uint32_t b1 = ch.bucket_base + bucket_of(K1, ch.B), b2 = ch.bucket_base + bucket_of(K2, ch.B);
    const uint32_t x1 = atomicAdd(&a.pcount[b1], 1u);
    const uint32_t x2 = atomicAdd(&a.pcount[b2], 1u);
    store_record(a, b1, x1, mid_of(K1, ch.B), ij.x, e1);
    store_record(a, b2, x2, mid_of(K2, ch.B), ij.y, e2);
  } else {  // odd m: the chain's last slot has no partner
    const uint32_t pos = a.cpos[s0];
    const unsigned long long K = perm_key(ch.seed, round, pos);
    const uint32_t b = ch.bucket_base + bucket_of(K, ch.B);
    store_record(a, b, atomicAdd(&a.pcount[b], 1u), mid_of(K, ch.B), pos, a.cedge[s0]);
  }
}

__device__ __forceinline__ void permute_body(const RoundArgs &a) {
  const unsigned long long R = a.ctl->pool_round;
  const uint32_t npair = (a.slot_hw + 1) >> 1;
  const uint32_t nth = gridDim.x * blockDim.x;
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < npair; x += nth) permute_pair(a, x, R);
}

// The CTA's place in a flat pass: CTA b takes range (b * stride) mod ctas.
__device__ __forceinline__ uint32_t scrambled_cta(uint32_t stride) {
  return (uint32_t)(((unsigned long long)blockIdx.x * stride) % gridDim.x);
}

// One pair of slots per thread, CTAs in scrambled order.
__global__ void __launch_bounds__(256, 5) k_permute(RoundArgs a) {
  const uint32_t x = scrambled_cta(a.permute_stride) * blockDim.x + threadIdx.x;
  if (x < (a.slot_hw + 1) >> 1) permute_pair(a, x, a.ctl->pool_round);
}

// Exclusive scan of n counters (n + 1 offsets) by one CTA of 1024 threads,
// in place if off == count; counts above `clamp` are clamped (their
// overflow was already reported).
__device__ __forceinline__ void cta_scan_1024(const uint32_t *count, uint32_t *off, uint32_t *copy, uint32_t n,
                                              uint32_t clamp) {
  __shared__ uint32_t part[1024];
  const uint32_t tid = threadIdx.x;
  const uint32_t per = (n + 1023) / 1024;
  const uint32_t beg = min(tid * per, n), end = min(beg + per, n);
  uint32_t sum = 0;
  for (uint32_t b = beg; b < end; ++b) sum += min(count[b], clamp);
  part[tid] = sum;
  __syncthreads();
  for (uint32_t d = 1; d < 1024; d <<= 1) {
    const uint32_t v = tid >= d ? part[tid - d] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  uint32_t run = part[tid] - sum;
  for (uint32_t b = beg; b < end; ++b) {
    const uint32_t c = min(count[b], clamp);  // read before writing: count may be off itself
    off[b] = run;
    if (copy) copy[b] = run;
    run += c;
  }
  if (tid == 1023) off[n] = part[1023];
}

// Bucket slot offsets in two steps: each CTA scans a block of 1024 bucket
// counts (clamped to the capacity; an overflow was reported) and records the
// block's sum; one CTA then scans the block sums.  A bucket's offset is
// pblk[b / 1024] + poff[b].
__global__ void __launch_bounds__(1024) k_scan_perm(RoundArgs a) {
  __shared__ uint32_t warp_tot[32];
  const uint32_t b = blockIdx.x * 1024 + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t v = b < a.bucket_hw ? min(a.pcount[b], 1u << a.bucket_log2) : 0u;
  uint32_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= (uint32_t)d) incl += u;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = warp_tot[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, t, d);
      if (lane >= (uint32_t)d) t += u;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  if (b < a.bucket_hw) a.poff[b] = incl - v + (warp ? warp_tot[warp - 1] : 0u);
  if (threadIdx.x == 1023) a.pblk[blockIdx.x] = warp_tot[31];
}

__global__ void __launch_bounds__(1024) k_scan_blocks(RoundArgs a) {
  const uint32_t nblk = (a.bucket_hw + 1023) / 1024;
  cta_scan_1024(a.pblk, a.pblk, nullptr, nblk, 0xFFFFFFFFu);
}

__device__ __forceinline__ uint32_t bucket_offset(const RoundArgs &a, uint32_t b) {
  return a.pblk[b >> 10] + a.poff[b];
}

// Overflow tuples (those that found their partition full), grouped by
// partition with exact counts.  Every kernel does nothing when there is no
// overflow, which is the normal case for a single chain.  The partition
// offsets are scanned like the bucket offsets: blocks of 1024 partitions on
// many CTAs (local offsets, and the cursors the scatter starts from), then
// the block sums on one CTA; partition p's list starts at
// oblk[p / 1024] + ooff[p].
__device__ __forceinline__ void overflow_count_body(const RoundArgs &a) {
  const uint32_t n = min(a.ctl->ovf_count, a.ovf_cap);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
    atomicAdd(&a.ocount[a.otup[t].w], 1u);
}

__global__ void k_overflow_count(RoundArgs a) { overflow_count_body(a); }

__global__ void __launch_bounds__(1024) k_overflow_scan_blocks(RoundArgs a) {
  if (a.ctl->ovf_count == 0) return;
  __shared__ uint32_t warp_tot[32];
  const uint32_t p = blockIdx.x * 1024 + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t v = p < a.part_hw ? a.ocount[p] : 0u;
  uint32_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= (uint32_t)d) incl += u;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = warp_tot[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, t, d);
      if (lane >= (uint32_t)d) t += u;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  if (p < a.part_hw) {
    const uint32_t local = incl - v + (warp ? warp_tot[warp - 1] : 0u);
    a.ooff[p] = local;
    a.ocursor[p] = local;
  }
  if (threadIdx.x == 1023) a.oblk[blockIdx.x] = warp_tot[31];
}

__global__ void __launch_bounds__(1024) k_overflow_scan_top(RoundArgs a) {
  if (a.ctl->ovf_count == 0) return;
  const uint32_t nblk = (a.part_hw + 1023) / 1024;
  cta_scan_1024(a.oblk, a.oblk, nullptr, nblk, 0xFFFFFFFFu);  // oblk[nblk] = all overflow tuples
}

// Start of partition p's overflow list (p <= part_hw; part_hw gives the end).
__device__ __forceinline__ uint32_t overflow_offset(const RoundArgs &a, uint32_t p) {
  return p < a.part_hw ? a.oblk[p >> 10] + a.ooff[p] : a.oblk[(a.part_hw + 1023) >> 10];
}

__device__ __forceinline__ void overflow_scatter_body(const RoundArgs &a) {
  const uint32_t n = min(a.ctl->ovf_count, a.ovf_cap);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const uint4 r = a.otup[t];
    const uint32_t dst = a.oblk[r.w >> 10] + atomicAdd(&a.ocursor[r.w], 1u);
    if (dst < n) a.stup[dst] = make_uint4(r.x, r.y, r.z, (uint32_t)mix64(((unsigned long long)r.y << 32) | r.x));
  }
}

__global__ void k_overflow_scatter(RoundArgs a) { overflow_scatter_body(a); }

// In-place exclusive scan of 2^kLog2 counters by a CTA of kThreads.
template <int kThreads, int kLog2>
__device__ __forceinline__ void cta_exclusive_scan(uint32_t *h, uint32_t *warp_tot) {
  constexpr int n = 1 << kLog2;
  constexpr int per = n / kThreads;
  constexpr int nwarps = kThreads / 32;
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
    uint32_t t = lane < nwarps ? warp_tot[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, t, d);
      if (lane >= d) t += v;
    }
    if (lane < nwarps) warp_tot[lane] = t;
  }
  __syncthreads();
  uint32_t run = incl - sum + (warp ? warp_tot[warp - 1] : 0);
#pragma unroll
  for (int r = 0; r < per; ++r) {
    h[tid * per + r] = run;
    run += loc[r];
  }
}

// Sum of v over the CTA's kThreads threads, returned to every thread
// (warp_tot: kThreads / 32 words of scratch).  Every thread calls it.
template <int kThreads>
__device__ __forceinline__ uint32_t cta_sum(uint32_t v, uint32_t *warp_tot) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = v;
  __syncthreads();
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) total += warp_tot[w];
  __syncthreads();
  return total;
}

__device__ __forceinline__ bool full_key_less(unsigned long long seed, unsigned long long round, uint32_t i,
                                              uint32_t j) {
  const unsigned long long ki = perm_key(seed, round, i), kj = perm_key(seed, round, j);
  return ki < kj || (ki == kj && i < j);
}

// The shared memory of one bucket's sort: the bucket's records as copied,
// the record at each slot, the sub-bucket histogram, per-warp sums, and the
// mbarrier the bulk copy completes on.
struct SortSmem {
  uint4 *srec;       // {32 key bits, position, edge lo, edge hi}, room for a bucket
  uint16_t *sidx;    // record at each slot of the bucket
  uint32_t *hist;    // one counter per sub-bucket (as many as the bucket has room for records)
  uint32_t *warp_tot;
  unsigned long long *bar;
};

// Shared memory of a sort of buckets with room for 2^log2 records (the
// sub-bucket histogram has as many counters).
constexpr size_t sort_smem_bytes(uint32_t log2) {
  return (sizeof(uint4) + sizeof(uint16_t) + sizeof(uint32_t)) * (size_t(1) << log2) + sizeof(uint32_t) * 32 + 16;
}

// Bucket b, by one CTA of kThreads threads.  The bucket's records come into
// shared memory in one bulk copy (the TMA engine, cp.async.bulk, completing
// on the mbarrier's phase `parity`); an exact sort of record indices by
// (key, position) follows: a counting sort on the top key bits, insertion
// sort inside the sub-buckets, and a full-key fix for runs of equal 32-bit
// key parts.  Then the list is written back in this round's slot order and
// the switches of all pairs of consecutive slots inside the bucket are
// built.  Returns false (with kErrCopy set) if the copy did not land in time;
// the caller must stop then.  Every thread of the CTA calls it; `parity`
// tracks the barrier's phase across the buckets a CTA sorts.
template <int kThreads, int kLog2>
__device__ __forceinline__ bool sort_bucket(const RoundArgs &a, uint32_t b, const SortSmem &sm, uint32_t &parity,
                                            bool local_offsets = false) {
  constexpr uint32_t kCap = 1u << kLog2;
  constexpr int kSubBits = kLog2;  // sub-buckets: about two per record
  uint4 *const srec = sm.srec;
  uint16_t *const sidx = sm.sidx;
  uint32_t *const hist = sm.hist;
  const int tid = threadIdx.x;
  constexpr int nsub = 1 << kSubBits;
  const uint32_t c = a.owner_bucket[b];
  if (c == kNoChain) return true;
  const uint32_t cnt = min(a.pcount[b], kCap);
  if (tid == 0 && cnt) {
    mbar_arrive_expect(sm.bar, cnt * (uint32_t)sizeof(uint4));
    bulk_copy_g2s(srec, a.prec + ((size_t)b << kLog2), cnt * (uint32_t)sizeof(uint4), sm.bar);
  }
  for (int s2 = tid; s2 < nsub; s2 += kThreads) hist[s2] = 0;
  const unsigned long long R = a.ctl->pool_round;
  const ChainDesc ch = a.chains[c];
  const unsigned long long round = chain_round(ch, R);
  const uint32_t ell = ch.exact_ell ? a.chain_ell[c] : 0u;
  // chain-local slot offset: from the scanned offsets, or summed here over
  // the chain's earlier buckets (a small chain in the one-launch round)
  uint32_t loff;
  if (local_offsets) {
    uint32_t sum = 0;
    for (uint32_t j = ch.bucket_base + tid; j < b; j += kThreads) sum += min(a.pcount[j], kCap);
    loff = cta_sum<kThreads>(sum, sm.warp_tot);
  } else {
    loff = bucket_offset(a, b) - bucket_offset(a, ch.bucket_base);
  }
  const uint32_t goff = ch.slot_base + loff;
  __syncthreads();  // the histogram is cleared
  const bool landed = cnt == 0 || mbar_wait(sm.bar, parity, kCopyWaitPolls);
  if (__syncthreads_or(!landed)) {
    // the copy did not complete in time: report it, give it a last bounded
    // wait (shared memory must not be released under a copy in flight), stop
    if (tid == 0) atomicOr(&a.ctl->err, kErrCopy);
    if (cnt) mbar_wait(sm.bar, parity, kCopyWaitPolls);
    return false;
  }
  if (cnt) parity ^= 1u;  // the barrier's next phase serves the CTA's next copy
  for (uint32_t t = tid; t < cnt; t += kThreads) atomicAdd(&hist[srec[t].x >> (32 - kSubBits)], 1u);
  __syncthreads();
  cta_exclusive_scan<kThreads, kSubBits>(hist, sm.warp_tot);
  __syncthreads();
  for (uint32_t t = tid; t < cnt; t += kThreads) sidx[atomicAdd(&hist[srec[t].x >> (32 - kSubBits)], 1u)] = t;
  __syncthreads();
  // hist[s] is now the end of sub-bucket s; sort each (a handful of items)
  // by (32 key bits, position)
  for (int s2 = tid; s2 < nsub; s2 += kThreads) {
    const uint32_t beg = s2 ? hist[s2 - 1] : 0, end = hist[s2];
    for (uint32_t x = beg + 1; x < end; ++x) {
      const uint16_t li = sidx[x];
      const unsigned long long val = ((unsigned long long)srec[li].x << 32) | srec[li].y;
      uint32_t y = x;
      for (; y > beg; --y) {
        const uint2 kp = *reinterpret_cast<const uint2 *>(&srec[sidx[y - 1]]);
        if ((((unsigned long long)kp.x << 32) | kp.y) <= val) break;
        sidx[y] = sidx[y - 1];
      }
      sidx[y] = li;
    }
  }
  __syncthreads();
  // equal 32-bit key parts: order those runs by the full key
  for (uint32_t t = tid; t + 1 < cnt; t += kThreads) {
    const uint32_t mt = srec[sidx[t]].x;
    if (srec[sidx[t + 1]].x == mt && (t == 0 || srec[sidx[t - 1]].x != mt)) {
      uint32_t e = t + 2;
      while (e < cnt && srec[sidx[e]].x == mt) ++e;
      for (uint32_t x = t + 1; x < e; ++x) {
        const uint16_t li = sidx[x];
        const uint32_t pos = srec[li].y;
        uint32_t y = x;
        while (y > t && full_key_less(ch.seed, round, pos, srec[sidx[y - 1]].y)) {
          sidx[y] = sidx[y - 1];
          --y;
        }
        sidx[y] = li;
      }
    }
  }
  __syncthreads();
  // slots of the bucket hold pi in order: write the list in slot order, a
  // pair of slots (a switch) per thread, and build the switch; a pair's first
  // slot is even in the pool (chains start on even slots), so both slots go
  // out in one 8-byte and one 16-byte store
  const uint32_t t0 = loff & 1u;
  const uint32_t npairs = cnt > t0 ? (cnt - t0) >> 1 : 0;
  for (uint32_t p = tid; p < npairs; p += kThreads) {
    const uint32_t t = t0 + 2 * p;
    const uint4 r1 = srec[sidx[t]], r2 = srec[sidx[t + 1]];
    const bool valid[1] = {true};
    const uint32_t k[1] = {(loff + t) >> 1}, i[1] = {r1.y}, j[1] = {r2.y};
    const unsigned long long e1[1] = {((unsigned long long)r1.w << 32) | r1.z};
    const unsigned long long e2[1] = {((unsigned long long)r2.w << 32) | r2.z};
    *reinterpret_cast<uint2 *>(&a.cpos[goff + t]) = make_uint2(r1.y, r2.y);
    *reinterpret_cast<ulonglong2 *>(&a.cedge[goff + t]) = make_ulonglong2(e1[0], e2[0]);
    build_switches<1>(a, ch, round, ell, valid, k, i, e1, j, e2);
  }
  // the slots in no pair of this bucket: the first (its pair started in the
  // bucket before) and the last (its pair ends in the next bucket, or m is odd)
  if (tid < 2 && cnt > 0) {
    const uint32_t t = tid == 0 ? 0u : cnt - 1;
    const bool alone = tid == 0 ? t0 == 1 : ((cnt - t0) & 1u) && cnt - 1 >= t0 && !(t0 == 1 && cnt == 1);
    if (alone) {
      const uint4 r = srec[sidx[t]];
      a.cpos[goff + t] = r.y;
      a.cedge[goff + t] = ((unsigned long long)r.w << 32) | r.z;
    }
  }
  if (tid == 0 && t0 == 1 && cnt > 0) {
    // this bucket's first slot is the second of a pair started in an
    // earlier bucket: k_boundary builds that switch from the list
    const uint32_t idx = atomicAdd(&a.ctl->boundary, 1u);
    a.bnd[idx] = goff - 1;  // the pair's first slot
  }
  __syncthreads();  // the CTA's shared memory may take the next bucket's copy
  return true;
}

// One CTA per bucket (the round's launch over all buckets): buckets with
// room for 2^kLog2 records, CTAs of 2^(kLog2 - 3) threads, kMin of them
// per SM.  Seven CTAs of 128 threads (70 registers) sorted G(2^24)'s
// buckets in 3.85 ms per round, against 3.98 with six (80 registers), 4.02-
// 4.07 with eight (63) and 5.37 with nine (56).  The larger buckets run four
// CTAs of 256 threads (63 registers; three at 80 took 4.90 against 4.51 ms on
// the 4096-chain ensemble).
template <int kLog2, int kMin>
__global__ void __launch_bounds__(1 << (kLog2 - 3), kMin) k_sortpair(RoundArgs a) {
  constexpr int kThreads = 1 << (kLog2 - 3);
  __shared__ __align__(128) uint4 srec[1 << kLog2];
  __shared__ uint16_t sidx[1 << kLog2];
  __shared__ uint32_t hist[1 << kLog2];
  __shared__ uint32_t warp_tot[kThreads / 32];
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const SortSmem sm{srec, sidx, hist, warp_tot, &bar};
  uint32_t parity = 0;
  if (sort_bucket<kThreads, kLog2>(a, blockIdx.x, sm, parity) && threadIdx.x == 0) mbar_inval(&bar);
}

__device__ __forceinline__ void boundary_body(const RoundArgs &a) {
  const uint32_t n = a.ctl->boundary;
  const unsigned long long R = a.ctl->pool_round;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const uint32_t g = a.bnd[idx];  // first slot of the pair
    const uint32_t c = g < a.slot_hw ? a.owner_slot[g] : kNoChain;
    if (c == kNoChain) {  // cannot happen unless a bucket overflowed (reported)
      atomicOr(&a.ctl->err, kErrRecord);
      continue;
    }
    const ChainDesc ch = a.chains[c];
    const uint32_t k = (g - ch.slot_base) >> 1;
    if (k >= ch.L) {
      atomicOr(&a.ctl->err, kErrRecord);
      continue;
    }
    // both slots were written by the sort kernel (the list in this round's slot order)
    const bool valid[1] = {true};
    const uint32_t kk[1] = {k}, i[1] = {a.cpos[g]}, j[1] = {a.cpos[g + 1]};
    const unsigned long long e1[1] = {a.cedge[g]}, e2[1] = {a.cedge[g + 1]};
    build_switches<1>(a, ch, chain_round(ch, R), ch.exact_ell ? a.chain_ell[c] : 0u, valid, kk, i, e1, j, e2);
  }
}

__global__ void k_boundary(RoundArgs a) { boundary_body(a); }

// The chain of a thread's current pair, kept while its consecutive pairs
// stay in it: pairs [lo, hi) are chain c's.
struct PairChain {
  uint32_t c = kNoChain, lo = 1, hi = 0;
};

// Make pc the chain of pair x; false if no chain owns it.
__device__ __forceinline__ bool pair_chain(const RoundArgs &a, uint32_t x, PairChain &pc) {
  if (x >= pc.lo && x < pc.hi) return true;
  pc.c = a.owner_slot[2 * x];
  if (pc.c == kNoChain) {
    pc.lo = 1;
    pc.hi = 0;
    return false;
  }
  pc.lo = a.chains[pc.c].slot_base >> 1;
  pc.hi = pc.lo + ((a.chains[pc.c].m + 1) >> 1);
  return true;
}

// One pair of slots: its two sources, the ERASE value they carry, and
// where their tuples go (each key's partition cursor and storage, from its
// chain).  A key that needs no tuple becomes kEmptyKey.
struct SourcePair {
  unsigned long long key[2], hash[2];
  uint32_t val, cursor[2], capt, part[2];
  size_t base[2];
};

__device__ __forceinline__ void load_source_pair(const RoundArgs &a, uint32_t x, bool owned, uint32_t c,
                                                 ulonglong2 ee, SourcePair &sp) {
  sp.key[0] = ee.x;
  sp.key[1] = ee.y;
  sp.val = kTupleSource | kKeepK;
  if (!owned) {
    sp.key[0] = sp.key[1] = kEmptyKey;
    return;
  }
  const ChainDesc &ch = a.chains[c];
  const uint32_t ls = 2 * x - ch.slot_base;
  if (ls + 1 < ch.m) {
    const uint32_t kg = ch.switch_base + (ls >> 1);
    if ((__ldcs(&a.word[kg]) & kCodeMask) == 0) sp.val = kTupleSource | kg;
  } else {
    sp.key[1] = kEmptyKey;  // odd m: the unpaired last slot
  }
  sp.capt = ch.capt;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    sp.hash[t] = mix64(sp.key[t]);
    const uint32_t p = partition_of(sp.hash[t], ch.P);
    sp.cursor[t] = ch.tcount_base + p * ch.tstride;
    sp.base[t] = ch.tuple_base + (size_t)p * ch.capt;
    sp.part[t] = ch.part_base + p;
  }
}

// The sources of every switch (Algorithm 1's ERASE tuples) from the list in
// this round's slot order, two pairs per thread (x and x + 256): all loads
// first (list entries, reject words, filter words), then the cursor atomics
// of all four keys, then their stores.  Only an edge id that is some
// switch's target needs a tuple (the grouping only asks whether targets
// exist and who erases them), so a source whose filter bit is clear is
// dropped; a set bit can be a collision, which only adds a tuple nobody
// needs.  The unpaired last slot of an odd list is a source no switch
// erases, and so are the sources of a switch rejected outright.
__device__ __forceinline__ void source_pairs(const RoundArgs &a, uint32_t x, uint32_t y, uint32_t end) {
  PairChain pc;
  const ulonglong2 ex = __ldcs(reinterpret_cast<const ulonglong2 *>(a.cedge) + x);
  ulonglong2 ey = make_ulonglong2(kEmptyKey, kEmptyKey);
  if (y < end) ey = __ldcs(reinterpret_cast<const ulonglong2 *>(a.cedge) + y);
  SourcePair sp[2];
  const bool ox = pair_chain(a, x, pc);
  load_source_pair(a, x, ox, pc.c, ex, sp[0]);
  const bool oy = y < end && pair_chain(a, y, pc);
  load_source_pair(a, y, oy, pc.c, ey, sp[1]);
  uint32_t w[2][2];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int t = 0; t < 2; ++t)
      w[q][t] = sp[q].key[t] == kEmptyKey ? 0u : __ldcg(&a.tfilter[filter_bit(a, sp[q].hash[t]) >> 5]);
  uint32_t idx[2][2];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (!((w[q][t] >> (filter_bit(a, sp[q].hash[t]) & 31)) & 1u)) sp[q].key[t] = kEmptyKey;
      idx[q][t] = sp[q].key[t] != kEmptyKey ? atomicAdd(&a.tcount[sp[q].cursor[t]], 1u) : 0u;
    }
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const unsigned long long k = sp[q].key[t];
      if (k == kEmptyKey) continue;
      if (idx[q][t] < sp[q].capt) {
        a.ptup[sp[q].base[t] + idx[q][t]] = make_uint4((uint32_t)k, (uint32_t)(k >> 32), sp[q].val,
                                                       (uint32_t)sp[q].hash[t]);
      } else {
        const uint32_t o = atomicAdd(&a.ctl->ovf_count, 1u);
        if (o < a.ovf_cap)
          a.otup[o] = make_uint4((uint32_t)k, (uint32_t)(k >> 32), sp[q].val, sp[q].part[t]);
        else
          atomicOr(&a.ctl->err, kErrRecord);
      }
    }
}

// One launch of short-lived CTAs, two pairs per thread (measured faster than
// a grid-stride loop over a resident grid).
__global__ void __launch_bounds__(256, 4) k_sources(RoundArgs a) {
  const uint32_t end = a.slot_hw >> 1;
  const uint32_t x = scrambled_cta(a.sources_stride) * 2 * blockDim.x + threadIdx.x;
  if (x < end) source_pairs(a, x, x + blockDim.x, end);
}

// Grouping of one tuple partition by edge id (Algorithm 1's table T for the
// partition's edge ids) in a shared-memory table of S slots: slot[s] =
// {key lo, key hi, p, q} with p the eraser (from the source tuple) and q
// the smallest inserter, and aux[s] = 1 once a second inserter arrives.
// Then wave 1 for every target: present when k runs (p >= k), dependent on
// an undecided switch (p < k, or an earlier inserter q < k), or free.  Edge
// ids with a dependency get an entry {p, q} for the later waves, whose index
// replaces aux[s].  Slots are probed from the low bits of the id's hash,
// which the tuple carries.
struct GroupSmem {
  uint4 *slot;
  uint32_t *aux;
};

__device__ __forceinline__ GroupSmem group_smem(uint32_t S) {
  extern __shared__ uint4 group_dyn[];
  GroupSmem g;
  g.slot = group_dyn;
  g.aux = reinterpret_cast<uint32_t *>(group_dyn + S);
  return g;
}

__device__ __forceinline__ unsigned long long *slot_key(const GroupSmem &g, uint32_t s) {
  return reinterpret_cast<unsigned long long *>(&g.slot[s]);
}

__device__ __forceinline__ void group_reset_slot(const GroupSmem &g, uint32_t s) {
  g.slot[s] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, kPNone, kQNone);
  g.aux[s] = 0;
}

constexpr uint32_t kClaimed = 0x80000000u;  // slot result: this thread took the slot

// Insert one tuple; returns its slot (| kClaimed if this thread took the
// empty slot), or S if the table is full.
__device__ __forceinline__ uint32_t group_insert(const GroupSmem &g, uint32_t S, unsigned long long key, uint32_t h,
                                                 uint32_t v) {
  uint32_t s = h & (S - 1), n = 0, claimed = 0;
  for (; n < S; ++n) {
    const unsigned long long cur = *slot_key(g, s);
    if (cur == key) break;
    if (cur == kEmptyKey) {
      const unsigned long long prev = atomicCAS(slot_key(g, s), kEmptyKey, key);
      if (prev == kEmptyKey) {
        claimed = kClaimed;
        break;
      }
      if (prev == key) break;
    }
    s = (s + 1) & (S - 1);
  }
  if (n == S) return S;
  if (v & kTupleSource) {
    const uint32_t kk = v & kTupleK;
    g.slot[s].z = kk == kKeepK ? kPKeep : kk;  // one source per edge id (Obs. 2)
  } else if (atomicMin(&g.slot[s].w, v & kTupleK) != kQNone) {
    g.aux[s] = 1;  // a second inserter
  }
  return s | claimed;
}

// One dependency entry per edge id that some target depends on: an id
// inserted more than once, or inserted while in E at the round start.
// aux[s] is replaced by the entry index (kTrivial if none).
__device__ __forceinline__ void group_alloc(const RoundArgs &a, const GroupSmem &g, uint32_t s) {
  const uint32_t p = g.slot[s].z, q = g.slot[s].w;
  const bool need = q != kQNone && (g.aux[s] != 0 || p != kPNone);
  uint32_t idx = kTrivial;
  if (need) {
    idx = atomicAdd(&a.ctl->dep_count, 1u);
    if (idx < a.dep_cap) {
      a.dep[idx] = make_uint2(p, q);
    } else {
      idx = kTrivial;
      atomicOr(&a.ctl->err, kErrRecord);
    }
  }
  g.aux[s] = idx;
}

// Wave 1 for target tuple v in slot s.
__device__ __forceinline__ void group_decide(const RoundArgs &a, const GroupSmem &g, uint32_t s, uint32_t v) {
  const uint32_t k = v & kTupleK;
  const uint32_t p = g.slot[s].z, q = g.slot[s].w;
  if (p != kPNone && p >= k) atomicOr(&a.word[k], kFlagBad);       // present when k runs
  else if (p != kPNone || q != k) atomicOr(&a.word[k], kFlagDep);  // erased or inserted earlier, maybe
  const uint32_t d = g.aux[s];
  if (d != kTrivial) {
    if (v & kTupleWhich) a.sw[k].y = d;
    else a.sw[k].x = d;
  }
}

// Tuples a thread holds in registers on the fast path: 2 in the grouping
// kernel's 1024-thread CTAs (measured 7% faster than 4 in 512-thread CTAs:
// fewer probe loops in a row per thread before each barrier), 4 in the
// one-launch round's 512-thread CTAs; both take partitions of up to 2048
// tuples on the fast path.
constexpr int kGroupR = 2;

// Persistent CTAs over the partitions.  Fast path: the partition's tuples
// stay in registers, and each thread later visits and clears the slots it
// claimed.  Partitions with more tuples than fit, or more distinct ids than
// slots, take the sub-pass path: the ids whose hash bits 16.. select them,
// split further until each sub-pass fits.
// Bring the own tuples of partition `part` (if it exists and is owned) into
// L2 with one bulk prefetch (the TMA engine), so that the CTA finds them
// there when it gets to that partition.
__device__ __forceinline__ void prefetch_partition(const RoundArgs &a, uint32_t part) {
  if (part >= a.part_hw) return;
  const uint32_t c = a.owner_part[part];
  if (c == kNoChain) return;
  const ChainDesc &cd = a.chains[c];
  const uint32_t n = min(a.tcount[cd.tcount_base + (part - cd.part_base) * cd.tstride], cd.capt);
  if (n) bulk_prefetch_l2(a.ptup + cd.tuple_base + (size_t)(part - cd.part_base) * cd.capt, n * (uint32_t)sizeof(uint4));
}

template <int T, int R>
__device__ __forceinline__ void group_body(const RoundArgs &a) {
  const uint32_t S = 1u << a.group_log2;
  const GroupSmem g = group_smem(S);
  __shared__ uint32_t stk_sub[64], stk_n[64];
  __shared__ int stk_top;
  __shared__ uint32_t overflow;
  const int tid = threadIdx.x;
  const bool ovf = a.ctl->ovf_count != 0;
  for (uint32_t s = tid; s < S; s += T) group_reset_slot(g, s);
  if (tid == 0) overflow = 0;
  __syncthreads();
  for (uint32_t part = blockIdx.x; part < a.part_hw; part += gridDim.x) {
    const uint32_t c = a.owner_part[part];
    if (c == kNoChain) continue;
    if (tid == 0) prefetch_partition(a, part + gridDim.x);
    const uint32_t pbase = a.chains[c].part_base, tbase = a.chains[c].tuple_base, capt = a.chains[c].capt;
    // the partition's tuples: its own region, then its overflow tuples
    const uint4 *prim = a.ptup + tbase + (size_t)(part - pbase) * capt;
    const ChainDesc &cd = a.chains[c];
    const uint32_t nprim = min(a.tcount[cd.tcount_base + (part - pbase) * cd.tstride], capt);
    const uint32_t obeg = ovf ? overflow_offset(a, part) : 0, oend = ovf ? overflow_offset(a, part + 1) : 0;
    const uint32_t ntup = nprim + (oend - obeg);
    if (ntup <= (uint32_t)(R * T)) {
      uint4 r[R];
      uint32_t slot[R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const uint32_t t = tid + j * T;
        r[j] = make_uint4(0, 0, 0, 0);
        if (t < ntup) r[j] = t < nprim ? __ldcs(&prim[t]) : a.stup[obeg + (t - nprim)];
      }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const uint32_t t = tid + j * T;
        slot[j] = S;
        if (t < ntup) {
          slot[j] = group_insert(g, S, ((unsigned long long)r[j].y << 32) | r[j].x, r[j].w, r[j].z);
          if (slot[j] == S) overflow = 1;
        }
      }
      __syncthreads();
      const bool full = overflow != 0;
      if (!full) {
#pragma unroll
        for (int j = 0; j < R; ++j)
          if (slot[j] != S && (slot[j] & kClaimed)) group_alloc(a, g, slot[j] & ~kClaimed);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < R; ++j)
          if (slot[j] != S && !(r[j].z & kTupleSource)) group_decide(a, g, slot[j] & ~kClaimed, r[j].z);
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (slot[j] != S && (slot[j] & kClaimed)) group_reset_slot(g, slot[j] & ~kClaimed);
      if (tid == 0) overflow = 0;
      __syncthreads();
      if (!full) continue;
    }
    // sub-pass path
    if (tid == 0) {
      atomicAdd(&a.st->subpass_partitions, 1ull);
      stk_top = 1;
      stk_sub[0] = 0;
      stk_n[0] = 1;
    }
    __syncthreads();
    while (stk_top > 0) {
      const uint32_t sub = stk_sub[stk_top - 1], ns = stk_n[stk_top - 1];
      __syncthreads();
      if (tid == 0) {
        --stk_top;
        overflow = 0;
      }
      for (uint32_t s = tid; s < S; s += T) group_reset_slot(g, s);
      __syncthreads();
      for (uint32_t t = tid; t < ntup; t += T) {
        const uint4 r = t < nprim ? prim[t] : a.stup[obeg + (t - nprim)];
        if (ns > 1 && ((r.w >> 16) & (ns - 1)) != sub) continue;
        if (group_insert(g, S, ((unsigned long long)r.y << 32) | r.x, r.w, r.z) == S) overflow = 1;
      }
      __syncthreads();
      if (overflow) {
        if (tid == 0) {
          if (ns >= (1u << 16) || stk_top + 2 > 64) {
            atomicOr(&a.ctl->err, kErrGroup);
          } else {
            stk_sub[stk_top] = sub + ns;
            stk_n[stk_top] = 2 * ns;
            stk_sub[stk_top + 1] = sub;
            stk_n[stk_top + 1] = 2 * ns;
            stk_top += 2;
          }
        }
        __syncthreads();
        continue;
      }
      for (uint32_t s = tid; s < S; s += T)
        if (*slot_key(g, s) != kEmptyKey) group_alloc(a, g, s);
      __syncthreads();
      for (uint32_t t = tid; t < ntup; t += T) {
        const uint4 r = t < nprim ? prim[t] : a.stup[obeg + (t - nprim)];
        if (r.z & kTupleSource) continue;
        if (ns > 1 && ((r.w >> 16) & (ns - 1)) != sub) continue;
        const unsigned long long key = ((unsigned long long)r.y << 32) | r.x;
        uint32_t s = r.w & (S - 1);
        for (uint32_t n = 0; n < S && *slot_key(g, s) != key; ++n) s = (s + 1) & (S - 1);
        group_decide(a, g, s, r.z);
      }
      __syncthreads();
    }
    // leave the table empty for the next partition
    for (uint32_t s = tid; s < S; s += T) group_reset_slot(g, s);
    if (tid == 0) overflow = 0;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kGroupThreads, 2) k_group(RoundArgs a) { group_body<kGroupThreads, kGroupR>(a); }

// Each CTA takes a contiguous range of switches, so that a thread's running
// per-chain count changes chain only at chain boundaries.
__device__ __forceinline__ void wave1_body(const RoundArgs &a) {
  Tally t;
  ChainCount cc;
  const uint32_t per = (a.switch_hw + gridDim.x - 1) / gridDim.x;
  const uint32_t chunk = (per + blockDim.x - 1) / blockDim.x * blockDim.x;
  const uint32_t beg = min(blockIdx.x * chunk, a.switch_hw), end = min(beg + chunk, a.switch_hw);
  for (uint32_t base = beg; base < end; base += blockDim.x) {
    const uint32_t k = base + threadIdx.x;
    bool wait = false;
    uint32_t c = kNoChain;
    if (k < a.switch_hw) c = a.owner_switch[k];
    if (c != kNoChain) {
      const uint32_t w = __ldcs(&a.word[k]);
      const uint32_t code = w & kCodeMask;
      uint32_t state = kLegal;
      if (code) {
        state = kIllegal;
        if (code == kCodeLazy) ++t.lazy;
        else if (code == kCodeLoop) ++t.rej_loop;
        else ++t.rej_exists;
      } else if (w & kFlagBad) {
        state = kIllegal;
        ++t.rej_exists;
        drop_inserter(a, k, a.sw[k]);
      } else if (w & kFlagDep) {
        state = kUndecided;
        wait = true;
      } else {
        ++t.accepted;
        count_accepted(a, cc, c);
      }
      a.status[k] = state == kUndecided ? 0u : ((1u << 2) | state);
    }
    append_if(wait, k, a.list0, &a.ctl->pending[0]);
  }
  flush_tally(a, t);
  flush_count(a, cc);
}

__global__ void k_wave1(RoundArgs a) { wave1_body(a); }

__device__ __forceinline__ uint32_t wave_cap(const RoundArgs &a) {
  return a.max_waves ? a.max_waves : kDefaultWaveCap;
}

// One wave after the first, on the whole GPU.  Registration: every
// undecided switch becomes an inserter of its targets again (the q fields
// of illegal minima were cleared); also empties the list of the next wave.
// Nothing to do once no switch is undecided, or past the wave cap (k_tail
// reports that).
__global__ void k_wave_register(RoundArgs a) {
  const uint32_t cur = a.ctl->cur, wave = a.ctl->wave_next;
  const uint32_t n = a.ctl->pending[cur];
  if (n == 0 || wave > wave_cap(a)) return;
  const uint32_t *in = cur ? a.list1 : a.list0;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const uint32_t k = in[idx];
    const uint2 s = __ldcg(&a.sw[k]);
    if (s.x != kTrivial) atomicMin(&a.dep[s.x].y, k);
    if (s.y != kTrivial) atomicMin(&a.dep[s.y].y, k);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctl->pending[cur ^ 1] = 0;
    if (wave < kWaveHist) a.st->last_pending[wave] = n;
  }
}

// Decision of the same wave: legal, illegal (dropping it as an inserter),
// or undecided again (appended to the next wave's list).  The last CTA to
// finish moves the wave number on and switches lists.
__global__ void k_wave_decide(RoundArgs a) {
  __shared__ bool last;
  const uint32_t cur = a.ctl->cur, wave = a.ctl->wave_next;
  const uint32_t n = a.ctl->pending[cur];
  if (n == 0 || wave > wave_cap(a)) return;
  Tally t;
  ChainCount cc;
  const uint32_t *in = cur ? a.list1 : a.list0;
  uint32_t *out = cur ? a.list0 : a.list1;
  for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const uint32_t idx = base + threadIdx.x;
    bool wait = false;
    uint32_t k = 0;
    if (idx < n) {
      k = in[idx];
      const uint2 s = __ldcg(&a.sw[k]);
      const int r3 = check_target(a, k, s.x, wave);
      const int r4 = check_target(a, k, s.y, wave);
      if (r3 == kBad || r4 == kBad) {
        a.status[k] = (wave << 2) | kIllegal;
        drop_inserter(a, k, s);
        ++t.rej_exists;
      } else if (r3 == kWait || r4 == kWait) {
        wait = true;
      } else {
        a.status[k] = (wave << 2) | kLegal;
        ++t.accepted;
        count_accepted(a, cc, a.owner_switch[k]);
      }
    }
    append_if(wait, k, out, &a.ctl->pending[cur ^ 1]);
  }
  flush_tally(a, t);
  flush_count(a, cc);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&a.ctl->wave_blocks, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    a.ctl->wave_blocks = 0;
    a.ctl->cur = cur ^ 1;
    a.ctl->wave_next = wave + 1;
  }
}

// Waves 2, 3, ... on one CTA: undecided switches re-register as inserters
// (the q fields of illegal minima were cleared), then decide.  The kernel
// also closes the pool round (the round counter every chain derives its own
// round number from).
__global__ void __launch_bounds__(1024) k_tail(RoundArgs a) {
  __shared__ uint32_t s_n;
  Tally t;
  ChainCount cc;
  uint32_t cur = a.ctl->cur, wave = a.ctl->wave_next, prev_n = a.switch_hw + 1;
  volatile uint32_t *pend = a.ctl->pending;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_n = pend[cur];
    __syncthreads();
    const uint32_t n = s_n;
    if (n == 0) break;
    if (wave > wave_cap(a)) {
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
      const uint2 s = __ldcg(&a.sw[k]);
      if (s.x != kTrivial) atomicMin(&a.dep[s.x].y, k);
      if (s.y != kTrivial) atomicMin(&a.dep[s.y].y, k);
    }
    if (threadIdx.x == 0) {
      pend[cur ^ 1] = 0;
      if (wave < kWaveHist) a.st->last_pending[wave] = n;
    }
    __syncthreads();
    for (uint32_t base = 0; base < n; base += blockDim.x) {
      const uint32_t idx = base + threadIdx.x;
      bool wait = false;
      uint32_t k = 0;
      if (idx < n) {
        k = in[idx];
        const uint2 s = __ldcg(&a.sw[k]);
        const int r3 = check_target(a, k, s.x, wave);
        const int r4 = check_target(a, k, s.y, wave);
        if (r3 == kBad || r4 == kBad) {
          a.status[k] = (wave << 2) | kIllegal;
          drop_inserter(a, k, s);
          ++t.rej_exists;
        } else if (r3 == kWait || r4 == kWait) {
          wait = true;
        } else {
          a.status[k] = (wave << 2) | kLegal;
          ++t.accepted;
          count_accepted(a, cc, a.owner_switch[k]);
        }
      }
      append_if(wait, k, out, (uint32_t *)&pend[cur ^ 1]);
    }
    cur ^= 1;
    ++wave;
  }
  flush_tally(a, t);
  flush_count(a, cc);
  if (threadIdx.x == 0) {
    const uint32_t waves = a.any_work ? wave - 1 : 0;
    a.ctl->waves = waves;
    if (a.any_work) {
      a.st->waves_total += waves;
      if (waves > a.st->waves_max) a.st->waves_max = waves;
      a.st->wave_hist[waves < kWaveHist ? waves : kWaveHist - 1] += 1;
    }
    a.st->last_pending[1] = a.switch_hw;
    a.st->overflow_tuples += a.ctl->ovf_count;
    for (uint32_t w = wave; w < kWaveHist; ++w) a.st->last_pending[w] = 0;
    a.ctl->pool_round += 1;
  }
}

// ---------------------------------------------------------------- one-launch round

// Grid-wide barrier of a cooperative launch (every CTA resident).  Arrivals
// are counted on one monotonic counter: the CTA's thread 0 adds one with
// release-acquire semantics and polls (acquire) until every CTA has arrived
// at this barrier, i.e. the count has reached `target`, which every thread
// advances by the CTA count per barrier.  With the CTA barriers on both
// sides, every write before the barrier is visible after it.  The wait is
// bounded (kGridWaitPolls): a CTA that gives up sets kErrGridSync and
// returns false, and its caller leaves the kernel; the other CTAs see the
// error bit while they wait and leave too.
__device__ __forceinline__ bool grid_sync(Counters *ctl, unsigned long long &target) {
  __shared__ uint32_t ok;
  target += gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long v;
    asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], 1;" : "=l"(v) : "l"(&ctl->gbar_arrived) : "memory");
    ++v;
    uint32_t it = 0;
    while (v < target && it < kGridWaitPolls) {
      if (*(volatile uint32_t *)&ctl->err & kErrGridSync) break;
      __nanosleep(20);
      asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(&ctl->gbar_arrived) : "memory");
      ++it;
    }
    ok = v >= target;
    if (!ok) atomicOr(&ctl->err, kErrGridSync);
  }
  __syncthreads();
  return ok != 0;
}

// Exclusive scan of n counters (each clamped to `clamp`) by the calling CTA:
// off[b] (and copy[b], if given) receives the sum of the counters before b.
// Returns the total.  Every thread of the CTA calls it.
__device__ __forceinline__ uint32_t cta_scan_full(const uint32_t *count, uint32_t *off, uint32_t *copy, uint32_t n,
                                                  uint32_t clamp) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t total;
  const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t per = (n + nt - 1) / nt;
  const uint32_t beg = min(tid * per, n), end = min(beg + per, n);
  uint32_t sum = 0;
  for (uint32_t b = beg; b < end; ++b) sum += min(count[b], clamp);
  uint32_t incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= (uint32_t)d) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < nt / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, t, d);
      if (lane >= (uint32_t)d) t += v;
    }
    if (lane < nt / 32) wsum[lane] = t;
    if (lane == 31) total = t;
  }
  __syncthreads();
  uint32_t run = incl - sum + (warp ? wsum[warp - 1] : 0);
  for (uint32_t b = beg; b < end; ++b) {
    const uint32_t c = min(count[b], clamp);
    off[b] = run;
    if (copy) copy[b] = run;
    run += c;
  }
  const uint32_t tot = total;
  __syncthreads();
  return tot;
}

// End of a pool round (the work of k_tail after its waves): wave telemetry,
// statistics, and the pool's round counter.  One thread.
__device__ __forceinline__ void close_round(const RoundArgs &a, uint32_t wave) {
  const uint32_t waves = a.any_work ? wave - 1 : 0;
  a.ctl->waves = waves;
  if (a.any_work) {
    a.st->waves_total += waves;
    if (waves > a.st->waves_max) a.st->waves_max = waves;
    a.st->wave_hist[waves < kWaveHist ? waves : kWaveHist - 1] += 1;
  }
  a.st->last_pending[1] = a.switch_hw;
  a.st->overflow_tuples += a.ctl->ovf_count;
  for (uint32_t w = wave; w < kWaveHist; ++w) a.st->last_pending[w] = 0;
  a.ctl->pool_round += 1;
}

// The whole round of a pool in one cooperative launch of kFusedThreads-thread
// CTAs: the same stages as the multi-kernel round, in the same order, each
// spread over the launch's CTAs, with a grid barrier where the multi-kernel
// round has a kernel boundary.  The offset scans run on CTA 0 (the pools this
// launch is for have few buckets and partitions), and the waves after the
// first repeat register / decide until no switch is undecided.  The shared
// memory holds the sort's arrays and, later, the grouping table.
__global__ void __launch_bounds__(kFusedThreads, 1) k_round_fused(RoundArgs a) {
  extern __shared__ __align__(128) uint4 fused_dyn[];
  const uint32_t tid = threadIdx.x;
  const uint32_t gtid = blockIdx.x * blockDim.x + tid, nth = gridDim.x * blockDim.x;
  Counters *const ctl = a.ctl;
  // an earlier round of this call gave up at a barrier, which may have left
  // the barrier's counter behind: run nothing (every CTA reads the same
  // value, since no CTA can set the bit before all have passed the first
  // barrier below)
  if (*(volatile uint32_t *)&ctl->err & kErrGridSync) return;
  // the barrier count this launch starts from: earlier launches (all of this
  // CTA count) left it at a multiple of the CTA count, and fewer than that
  // many arrivals of this launch can precede this read
  __shared__ unsigned long long start_count;
  if (tid == 0) {
    const unsigned long long v = *(volatile unsigned long long *)&ctl->gbar_arrived;
    start_count = v / gridDim.x * gridDim.x;
  }
  __syncthreads();
  unsigned long long target = start_count;
  clear_body(a);
  for (uint32_t w = gtid; w <= (a.tfilter_mask >> 5); w += nth) a.tfilter[w] = 0;
  if (!grid_sync(ctl, target)) return;
  uint32_t wave = 2;
  if (a.any_work) {
    if (a.any_exact) {
      lazy_count_body(a);
      if (!grid_sync(ctl, target)) return;
    }
    permute_body(a);
    if (!grid_sync(ctl, target)) return;
    if (!a.fused_local_offsets) {
      if (blockIdx.x == 0) {  // bucket offsets: full offsets in poff, zero block offsets
        cta_scan_full(a.pcount, a.poff, nullptr, a.bucket_hw, 1u << a.bucket_log2);
        for (uint32_t j = tid; j <= (a.bucket_hw + 1023) / 1024; j += blockDim.x) a.pblk[j] = 0;
      }
      if (!grid_sync(ctl, target)) return;
    }
    {
      // laid out for the pool's bucket room (the region has room for the largest)
      unsigned char *base = reinterpret_cast<unsigned char *>(fused_dyn);
      const size_t room = size_t(1) << a.bucket_log2;
      SortSmem sm;
      sm.srec = reinterpret_cast<uint4 *>(base);
      sm.sidx = reinterpret_cast<uint16_t *>(base + sizeof(uint4) * room);
      sm.hist = reinterpret_cast<uint32_t *>(base + (sizeof(uint4) + sizeof(uint16_t)) * room);
      sm.warp_tot = sm.hist + room;
      sm.bar = reinterpret_cast<unsigned long long *>(sm.warp_tot + 32);
      if (tid == 0) mbar_init(sm.bar, 1);
      __syncthreads();
      uint32_t parity = 0;
      const bool local = a.fused_local_offsets != 0;
      for (uint32_t b = blockIdx.x; b < a.bucket_hw; b += gridDim.x)
        if (!(a.bucket_log2 == kBucketLog2Small
                  ? sort_bucket<kFusedThreads, kBucketLog2Small>(a, b, sm, parity, local)
                  : sort_bucket<kFusedThreads, kBucketLog2Large>(a, b, sm, parity, local)))
          return;
      __syncthreads();
      if (tid == 0) mbar_inval(sm.bar);  // the grouping table takes these bytes next
    }
    if (!grid_sync(ctl, target)) return;
    boundary_body(a);
    if (!grid_sync(ctl, target)) return;
    const uint32_t npair = a.slot_hw >> 1;
    for (uint32_t base = blockIdx.x * 2 * blockDim.x; base < npair; base += 2 * nth) {
      const uint32_t x = base + tid;
      if (x < npair) source_pairs(a, x, x + blockDim.x, npair);
    }
    if (!grid_sync(ctl, target)) return;
    if (*(volatile uint32_t *)&ctl->ovf_count) {
      overflow_count_body(a);
      if (!grid_sync(ctl, target)) return;
      if (blockIdx.x == 0) {  // overflow offsets: full offsets in ooff, zero block offsets, the total last
        const uint32_t tot = cta_scan_full(a.ocount, a.ooff, a.ocursor, a.part_hw, 0xFFFFFFFFu);
        const uint32_t nblk = (a.part_hw + 1023) >> 10;
        for (uint32_t j = tid; j < nblk; j += blockDim.x) a.oblk[j] = 0;
        if (tid == 0) a.oblk[nblk] = tot;
      }
      if (!grid_sync(ctl, target)) return;
      overflow_scatter_body(a);
      if (!grid_sync(ctl, target)) return;
    }
    group_body<kFusedThreads, 2048 / kFusedThreads>(a);
    if (!grid_sync(ctl, target)) return;
    wave1_body(a);
    if (!grid_sync(ctl, target)) return;
    // waves 2, 3, ...: undecided switches re-register as inserters, then decide
    Tally t;
    ChainCount cc;
    uint32_t cur = 0, prev_n = a.switch_hw + 1;
    volatile uint32_t *pend = ctl->pending;
    for (;;) {
      const uint32_t n = pend[cur];  // the same for every thread: read after a barrier
      if (n == 0) break;
      if (wave > wave_cap(a)) {
        if (gtid == 0) atomicOr(&ctl->err, kErrWaveCap);
        break;
      }
      if (n >= prev_n) {  // no switch was decided in the last wave: impossible
        if (gtid == 0) atomicOr(&ctl->err, kErrNoProgress);
        break;
      }
      prev_n = n;
      const uint32_t *in = cur ? a.list1 : a.list0;
      uint32_t *out = cur ? a.list0 : a.list1;
      for (uint32_t idx = gtid; idx < n; idx += nth) {
        const uint32_t k = in[idx];
        const uint2 sv = __ldcg(&a.sw[k]);
        if (sv.x != kTrivial) atomicMin(&a.dep[sv.x].y, k);
        if (sv.y != kTrivial) atomicMin(&a.dep[sv.y].y, k);
      }
      if (gtid == 0) {
        pend[cur ^ 1] = 0;
        if (wave < kWaveHist) a.st->last_pending[wave] = n;
      }
      if (!grid_sync(ctl, target)) return;
      for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += nth) {
        const uint32_t idx = base + tid;
        bool wait = false;
        uint32_t k = 0;
        if (idx < n) {
          k = in[idx];
          const uint2 sv = __ldcg(&a.sw[k]);
          const int r3 = check_target(a, k, sv.x, wave);
          const int r4 = check_target(a, k, sv.y, wave);
          if (r3 == kBad || r4 == kBad) {
            a.status[k] = (wave << 2) | kIllegal;
            drop_inserter(a, k, sv);
            ++t.rej_exists;
          } else if (r3 == kWait || r4 == kWait) {
            wait = true;
          } else {
            a.status[k] = (wave << 2) | kLegal;
            ++t.accepted;
            count_accepted(a, cc, a.owner_switch[k]);
          }
        }
        append_if(wait, k, out, (uint32_t *)&pend[cur ^ 1]);
      }
      if (!grid_sync(ctl, target)) return;
      cur ^= 1;
      ++wave;
    }
    flush_tally(a, t);
    flush_count(a, cc);
  }
  if (gtid == 0) close_round(a, wave);
}

// ---------------------------------------------------------------- state in / out

__global__ void k_load_chain(RoundArgs a, ChainDesc ch, const unsigned long long *E) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ch.m; s += gridDim.x * blockDim.x) {
    a.cpos[ch.slot_base + s] = s;
    a.cedge[ch.slot_base + s] = E[s];
  }
}

__global__ void k_store_chain(RoundArgs a, ChainDesc ch, unsigned long long *E) {
  const bool apply = chain_apply(ch, a.ctl->pool_round);
  const uint32_t npair = (ch.m + 1) >> 1;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < npair; k += gridDim.x * blockDim.x) {
    const uint32_t s0 = ch.slot_base + 2 * k;
    if (2 * k + 1 < ch.m) {
      const uint32_t i = a.cpos[s0], j = a.cpos[s0 + 1];
      unsigned long long e1 = a.cedge[s0], e2 = a.cedge[s0 + 1];
      apply_last(a, ch, apply, k, i, j, e1, e2);
      E[i] = e1;
      E[j] = e2;
    } else {
      E[a.cpos[s0]] = a.cedge[s0];
    }
  }
}

// ParES: the lists of the chains with a job, by position, with the last
// round's legal switches applied; and back into their slots (slot s holds
// position s, nothing pending).
__global__ void k_es_store(RoundArgs a, const EsJob *jobs, const uint32_t *job_of) {
  const unsigned long long R = a.ctl->pool_round;
  const uint32_t npair = (a.slot_hw + 1) >> 1;
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < npair; x += gridDim.x * blockDim.x) {
    const uint32_t s0 = 2 * x;
    const uint32_t c = a.owner_slot[s0];
    if (c == kNoChain || job_of[c] == kNoChain) continue;
    const ChainDesc ch = a.chains[c];
    unsigned long long *E = jobs[job_of[c]].E;
    const uint32_t ls = s0 - ch.slot_base;
    if (ls + 1 < ch.m) {
      const uint32_t i = a.cpos[s0], j = a.cpos[s0 + 1];
      unsigned long long e1 = a.cedge[s0], e2 = a.cedge[s0 + 1];
      apply_last(a, ch, chain_apply(ch, R), ls >> 1, i, j, e1, e2);
      E[i] = e1;
      E[j] = e2;
    } else {
      E[a.cpos[s0]] = a.cedge[s0];
    }
  }
}

__global__ void k_es_load(RoundArgs a, const EsJob *jobs, const uint32_t *job_of) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < a.slot_hw; s += gridDim.x * blockDim.x) {
    const uint32_t c = a.owner_slot[s];
    if (c == kNoChain || job_of[c] == kNoChain) continue;
    const ChainDesc ch = a.chains[c];
    const uint32_t ls = s - ch.slot_base;
    a.cpos[s] = ls;
    a.cedge[s] = jobs[job_of[c]].E[ls];
    if ((ls & 1u) == 0 && (ls >> 1) < ch.L) a.status[ch.switch_base + (ls >> 1)] = 0;  // nothing pending
  }
}

__global__ void k_fill_u32(uint32_t *p, uint32_t n, uint32_t v) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
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

__global__ void k_fill_u64(unsigned long long *p, unsigned long long n, unsigned long long v) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_duplicates(const unsigned long long *E, uint32_t m, unsigned long long *set, unsigned long long cap,
                             uint32_t *flags) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const unsigned long long key = E[i];
    unsigned long long s = __umul64hi(mix64(key), cap);
    bool placed = false;
    for (unsigned long long n = 0; n < cap && !placed; ++n) {
      const unsigned long long prev = atomicCAS(&set[s], kEmptyKey, key);
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

// Degree fingerprint term of one endpoint: the list's fingerprint is the sum
// (mod 2^64) over its edges of both endpoints' terms, a function of the
// multiset of endpoints, i.e. of the degree sequence, which a switch keeps.
__device__ __forceinline__ unsigned long long endpoint_term(uint32_t v) {
  return mix64(0x9E3779B97F4A7C15ull + v);
}

// Debug check of a position-order list: every entry canonical and
// loop-free (u < v) and in range (v < n, if n), and its degree fingerprint.
__global__ void k_list_check(const unsigned long long *E, uint32_t m, unsigned long long n, uint32_t *flags,
                             unsigned long long *fp) {
  uint32_t f = 0;
  unsigned long long sum = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const unsigned long long e = E[i];
    const uint32_t u = (uint32_t)(e >> 32), v = (uint32_t)e;
    if (!(u < v)) f |= kFlagLoop;
    if (n && v >= n) f |= kFlagRange;
    sum += endpoint_term(u) + endpoint_term(v);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off);
  if ((threadIdx.x & 31) == 0 && sum) atomicAdd(fp, sum);
  if (f) atomicOr(flags, f);
}

inline int grid_for(unsigned long long work, int threads, int num_sms, int per_sm) {
  unsigned long long g = (work + threads - 1) / threads;
  const unsigned long long lim = (unsigned long long)num_sms * per_sm;
  if (g > lim) g = lim;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

size_t group_smem_bytes(uint32_t group_log2) { return (size_t)kGroupSlotBytes << group_log2; }

cudaError_t prepare_kernels(uint32_t group_log2, int num_sms, LaunchShapes *shapes) {
  // opt in to the largest table any pool may use, so that pools with
  // different table sizes never lower each other's limit
  cudaError_t e = cudaFuncSetAttribute(k_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)group_smem_bytes(kMaxGroupLog2));
  if (e != cudaSuccess) return e;
  auto resident = [num_sms](const void *fn, int threads, size_t smem, uint32_t *grid) {
    int per_sm = 0;
    const cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    *grid = (uint32_t)(num_sms * (per_sm > 0 ? per_sm : 1));
    return r;
  };
  e = resident((const void *)k_group, kGroupThreads, group_smem_bytes(group_log2), &shapes->group);
  return e;
}



size_t fused_smem_bytes(uint32_t group_log2) {
  return std::max(sort_smem_bytes(kBucketLog2Large), group_smem_bytes(group_log2));
}

cudaError_t prepare_fused(uint32_t group_log2, int num_sms, uint32_t *max_ctas) {
  cudaError_t e = cudaFuncSetAttribute(k_round_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fused_smem_bytes(kMaxGroupLog2));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_round_fused, kFusedThreads,
                                                    fused_smem_bytes(group_log2));
  *max_ctas = (uint32_t)(num_sms * (per_sm > 0 ? per_sm : 0));
  return e;
}

cudaError_t launch_round_fused(const RoundArgs &a, cudaStream_t s, uint32_t ctas) {
  RoundArgs arg = a;
  void *params[] = {&arg};
  return cudaLaunchCooperativeKernel((const void *)k_round_fused, dim3(ctas), dim3(kFusedThreads), params,
                                     fused_smem_bytes(a.group_log2), s);
}

cudaError_t launch_round(const RoundArgs &a, cudaStream_t s, int num_sms, cudaEvent_t *ev, uint32_t *launches) {
  // ev (optional) receives kNumStages + 1 stage boundaries; stages that do
  // not run (no chain with two edges) still get both events (zero duration)
  auto mark = [&](int stage) {
    if (ev) cudaEventRecord(ev[stage], s);
  };
  uint32_t n = 0;
  const bool work = a.any_work != 0;
  mark(kStageClear);
  if (work) cudaMemsetAsync(a.tfilter, 0, 4ull * ((a.tfilter_mask >> 5) + 1), s);
  k_clear<<<grid_for(max(max(a.bucket_hw, a.part_hw), a.tcount_hw), 256, num_sms, 4), 256, 0, s>>>(a);
  ++n;
  if (work && a.any_exact) { k_lazy_count<<<grid_for(a.switch_hw, 256, num_sms, 8), 256, 0, s>>>(a); ++n; }
  mark(kStagePermute);
  if (work && a.agg_chain != kNoChain) {
    k_permute_agg<<<(a.agg_pairs + kAggThreads * kAggPairs - 1) / (kAggThreads * kAggPairs), kAggThreads, 0, s>>>(a);
    ++n;
  } else if (work) {
    k_permute<<<a.permute_ctas, 256, 0, s>>>(a);
    ++n;
  }
  mark(kStageScanPerm);
  if (work) {
    k_scan_perm<<<a.bucket_hw ? (a.bucket_hw + 1023) / 1024 : 1, 1024, 0, s>>>(a);
    k_scan_blocks<<<1, 1024, 0, s>>>(a);
    n += 2;
  }
  mark(kStageSortPair);
  if (work) {
    if (a.bucket_log2 == kBucketLog2Small)
      k_sortpair<kBucketLog2Small, 7><<<a.bucket_hw, 1 << (kBucketLog2Small - 3), 0, s>>>(a);
    else
      k_sortpair<kBucketLog2Large, 4><<<a.bucket_hw, 1 << (kBucketLog2Large - 3), 0, s>>>(a);
    ++n;
  }
  mark(kStageBoundary);
  if (work) { k_boundary<<<grid_for(a.bucket_hw, 256, num_sms, 2), 256, 0, s>>>(a); ++n; }
  mark(kStageSources);
  if (work) { k_sources<<<a.sources_ctas, 256, 0, s>>>(a); ++n; }
  mark(kStageOverflow);
  if (work) {
    const int g = grid_for(a.ovf_cap, 256, num_sms, 2);
    k_overflow_count<<<g, 256, 0, s>>>(a);
    k_overflow_scan_blocks<<<(a.part_hw + 1023) / 1024 ? (a.part_hw + 1023) / 1024 : 1, 1024, 0, s>>>(a);
    k_overflow_scan_top<<<1, 1024, 0, s>>>(a);
    k_overflow_scatter<<<g, 256, 0, s>>>(a);
    n += 4;
  }
  mark(kStageGroup);
  if (work) {
    const uint32_t ctas = a.group_grid ? a.group_grid : (uint32_t)num_sms;
    k_group<<<ctas < a.part_hw ? ctas : a.part_hw, kGroupThreads, group_smem_bytes(a.group_log2), s>>>(a);
    ++n;
  }
  mark(kStageWave1);
  if (work) { k_wave1<<<grid_for(a.switch_hw, 256, num_sms, 16), 256, 0, s>>>(a); ++n; }
  mark(kStageWaves);
  if (work) {
    for (uint32_t w = 0; w < a.wave_kernels && w < kMaxWaveKernels; ++w) {
      k_wave_register<<<num_sms * 4, 256, 0, s>>>(a);
      k_wave_decide<<<num_sms * 4, 256, 0, s>>>(a);
      n += 2;
    }
  }
  mark(kStageTail);
  k_tail<<<1, 1024, 0, s>>>(a);
  ++n;
  mark(kNumStages);
  if (launches) *launches += n;
  return cudaGetLastError();
}

cudaError_t launch_load_chain(const RoundArgs &a, const ChainDesc &ch, const unsigned long long *E, cudaStream_t s,
                              int num_sms) {
  if (ch.m == 0) return cudaSuccess;
  k_load_chain<<<grid_for(ch.m, 256, num_sms, 8), 256, 0, s>>>(a, ch, E);
  return cudaGetLastError();
}

cudaError_t launch_store_chain(const RoundArgs &a, const ChainDesc &ch, unsigned long long *E, cudaStream_t s,
                               int num_sms) {
  if (ch.m == 0) return cudaSuccess;
  k_store_chain<<<grid_for((ch.m + 1) / 2, 256, num_sms, 8), 256, 0, s>>>(a, ch, E);
  return cudaGetLastError();
}

cudaError_t launch_es_store(const RoundArgs &a, const EsJob *jobs, const uint32_t *job_of, cudaStream_t s,
                            int num_sms) {
  if (a.slot_hw == 0) return cudaSuccess;
  k_es_store<<<grid_for((a.slot_hw + 1) / 2, 256, num_sms, 8), 256, 0, s>>>(a, jobs, job_of);
  return cudaGetLastError();
}

cudaError_t launch_es_load(const RoundArgs &a, const EsJob *jobs, const uint32_t *job_of, cudaStream_t s,
                           int num_sms) {
  if (a.slot_hw == 0) return cudaSuccess;
  k_es_load<<<grid_for(a.slot_hw, 256, num_sms, 8), 256, 0, s>>>(a, jobs, job_of);
  return cudaGetLastError();
}

cudaError_t launch_fill_u32(uint32_t *p, uint32_t n, uint32_t v, cudaStream_t s, int num_sms) {
  if (n == 0) return cudaSuccess;
  k_fill_u32<<<grid_for(n, 256, num_sms, 8), 256, 0, s>>>(p, n, v);
  return cudaGetLastError();
}

cudaError_t launch_canonicalise(unsigned long long *E, uint32_t m, unsigned long long n_bound, uint32_t *flags,
                                uint32_t *max_id, cudaStream_t s, int num_sms) {
  k_canonicalise<<<grid_for(m, 256, num_sms, 8), 256, 0, s>>>(E, m, n_bound, flags, max_id);
  return cudaGetLastError();
}

cudaError_t launch_list_check(const unsigned long long *E, uint32_t m, unsigned long long n, uint32_t *flags,
                              unsigned long long *fp, cudaStream_t s, int num_sms) {
  if (m == 0) return cudaSuccess;
  k_list_check<<<grid_for(m, 256, num_sms, 8), 256, 0, s>>>(E, m, n, flags, fp);
  return cudaGetLastError();
}

cudaError_t launch_duplicate_check(const unsigned long long *E, uint32_t m, unsigned long long *set,
                                   unsigned long long cap, uint32_t *flags, cudaStream_t s, int num_sms) {
  k_fill_u64<<<grid_for(cap, 256, num_sms, 8), 256, 0, s>>>(set, cap, kEmptyKey);
  k_duplicates<<<grid_for(m, 256, num_sms, 8), 256, 0, s>>>(E, m, set, cap, flags);
  return cudaGetLastError();
}

}  // namespace gesmc
