// Resident rounds: global switches (Def. 2, performed as Algorithm 1's
// decide / delay waves) of small chains, one CTA per chain, the chain's list
// in shared memory from the first round of a call to the last.
//
// The paper notes that small graphs are the weak case of a parallel global
// switch (too little work per round to pay for its synchronisation) and that
// dedicated base cases would help.  On the GPU a round of the general path
// is a dozen dependent stages spread over the device; for a chain of about
// 10^4 edges their barriers or launches cost more than the work.  Here one
// CTA holds the whole chain: E as one 32-bit word per edge (two 16-bit node
// ids), the permutation, the switch statuses and a hash table of target
// edge ids, all in shared memory, so a round's stages are separated by
// __syncthreads only and nothing goes to global memory between rounds.
//
// Per round (round number r of the chain):
//   1. keys K(i) = Philox4x64-10((i >> 2, r, 0, 0); (seed, 0))[i & 3], the
//      same keys as the general path; a counting sort of the positions into
//      about m/2 buckets by the keys' top bits, then each position's rank in
//      its bucket in (K, i) order: the argsort pi.
//   2. switch k = (pi(2k), pi(2k+1), [pi(2k) < pi(2k+1)]): the outright
//      rejects (laziness, a loop, a shared node) are ILLEGAL before the first
//      wave; every other switch enters its two targets into the table
//      (ordered linear probing), then registers as an inserter (the entry
//      keeps the smallest inserter q) and keeps its targets' slots.
//   3. an edge of E that is some switch's target records its eraser p, the
//      switch whose slot holds it (the unpaired slot of an odd m erases
//      nothing: the edge stays, p = "never").
//   4. Jacobi waves: an undecided switch k decides from the statuses of
//      earlier waves only (a status word carries its wave): ILLEGAL if a
//      target is still there when k runs (erased by a later switch or never,
//      or its eraser failed, or an earlier inserter succeeded), UNDECIDED if
//      that depends on a switch not yet decided, else LEGAL.  Where a switch
//      turned illegal in the last wave, the smallest inserters of the ids
//      with two inserters or more are recomputed from the switches that are
//      not illegal (an id with one inserter is looked at by that one only).
//   5. the legal switches write their targets to their two positions.
// After the last round of the launch the list goes back to the chain's slots
// in position order with nothing pending, as the general path would leave
// it after store and reload.
#include "device_util.cuh"
#include "gesmc_internal.cuh"
#include "resident.cuh"

namespace gesmc {
namespace {

constexpr uint32_t kEmpty32 = 0xFFFFFFFFu;  // no edge packs to this (low id < high id)
constexpr uint32_t kP16None = 0xFFFFu;      // the id is not in E at the round's start
constexpr uint32_t kP16Keep = 0xFFFEu;      // in E, erased by no switch
constexpr uint32_t kQ16None = 0xFFFFu;      // no inserter that is not illegal

struct ResidentJob {
  const uint32_t *jobs;
  uint32_t rounds;
  uint32_t *round_waves;
  uint32_t *last_pending;
  uint32_t final;
  uint32_t wave_cap;
  // permutations sorted beforehand (null: each CTA sorts its own): round t
  // of job j at pbuf + (t * njobs + j) * pstride, its l (exact laziness) at
  // ebuf[t * njobs + j]; job_base = index of jobs[0] among all jobs
  uint16_t *pbuf;
  uint32_t *ebuf;
  uint32_t pstride, njobs, job_base;
};

// Byte offsets of a chain's pieces of shared memory (all grow with m).
struct ResLayout {
  uint32_t scat, perm, status, region, multi, nb_log2, slog2, bytes;
};

__host__ __device__ inline uint32_t ceil_log2(uint32_t x) {
  uint32_t b = 0;
  while ((1u << b) < x) ++b;
  return b;
}

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline ResLayout res_layout(uint32_t m) {
  ResLayout l;
  const uint32_t lg = ceil_log2(m);
  l.nb_log2 = lg > 6 ? lg - 1 : 5;             // about two keys per bucket, at least 32 buckets
  l.slog2 = lg + 1 < 6 ? 6 : (lg + 1 > 14 ? 14 : lg + 1);  // >= 2m slots, at most 2^14 (m targets at most)
  l.scat = align16(4 * m);                     // E: u32 per position
  l.perm = l.scat + align16(2 * m);            // positions by bucket (u16 per slot), later the
                                               // targets' table slots (u32 per switch)
  l.status = l.perm + align16(2 * m);          // pi: u16 per slot
  l.region = l.status + align16(2 * (m / 2));  // status: u16 per switch
  // the sort's keys (u64 per position) and bucket counts, then the table
  // (u32 key + u32 {p, q} per slot) in the same bytes
  const uint32_t sort_bytes = align16(8 * m) + 4 * (1u << l.nb_log2);
  const uint32_t table_bytes = 8 * (1u << l.slog2);
  l.multi = l.region + (sort_bytes > table_bytes ? sort_bytes : table_bytes);
  l.bytes = l.multi + align16((1u << l.slog2) / 8);  // one bit per table slot: two inserters or more
  return l;
}

// Canonical 32-bit id of the edge {a, b}: smaller node in the high half.
__device__ __forceinline__ uint32_t pack16(uint32_t a, uint32_t b) {
  return a < b ? (a << 16) | b : (b << 16) | a;
}

// tau of Def. 1 on packed edges (the same rules as tau_g): targets e3, e4
// and the outright-reject code (a loop, or sources sharing a node).
__device__ __forceinline__ uint32_t tau16(uint32_t g, uint32_t e1, uint32_t e2, uint32_t &e3, uint32_t &e4) {
  const uint32_t u = e1 >> 16, v = e1 & 0xFFFFu, x = e2 >> 16, y = e2 & 0xFFFFu;
  const uint32_t a3 = u, b3 = g ? y : x, a4 = v, b4 = g ? x : y;
  e3 = pack16(a3, b3);
  e4 = pack16(a4, b4);
  if (a3 == b3 || a4 == b4) return kCodeLoop;
  if (u == x || u == y || v == x || v == y) return kCodeShared;
  return 0;
}

__device__ __forceinline__ uint32_t home_slot(uint32_t e, uint32_t slog2) { return (e * 0x9E3779B1u) >> (32 - slog2); }

// Ordered linear probing: id e goes in by atomicMin from its home slot on;
// a slot keeps the smaller id and the larger one moves on to the next slot,
// until an id lands in an empty slot or meets its own copy.  False if the
// table is full.  A slot's id only ever decreases, and an id passes a slot
// only while the slot holds a smaller id, so every slot between an id's home
// and its final slot holds a smaller id: a search for e from its home can
// stop at the first slot whose id is >= e.
__device__ __forceinline__ bool tab_insert(uint32_t *tkey, uint32_t slog2, uint32_t e) {
  const uint32_t mask = (1u << slog2) - 1;
  uint32_t s = home_slot(e, slog2);
  for (uint32_t n = 0; n <= mask; ++n) {
    const uint32_t old = atomicMin(&tkey[s], e);
    if (old == kEmpty32 || old == e) return true;
    if (old > e) e = old;  // e took the slot; the displaced id moves on
    s = (s + 1) & mask;
  }
  return false;
}

// Slot of id e, or 2^slog2 if absent (no insertions run meanwhile).
__device__ __forceinline__ uint32_t tab_find(const uint32_t *tkey, uint32_t slog2, uint32_t e) {
  const uint32_t mask = (1u << slog2) - 1;
  uint32_t s = home_slot(e, slog2);
  for (uint32_t n = 0; n <= mask; ++n) {
    const uint32_t cur = tkey[s];
    if (cur >= e) return cur == e ? s : mask + 1;  // (the empty mark is the largest word)
    s = (s + 1) & mask;
  }
  return mask + 1;
}

// q of an entry (low 16 bits of {p, q}) lowered to k if k is smaller: one
// atomicMin of the whole word, since p (the high half) does not change while
// inserters register (all p are "none" at the first registration, and fixed
// by step 3 before any re-registration).
__device__ __forceinline__ uint32_t tab_qmin(uint32_t *tpq, uint32_t s, uint32_t k) {
  return atomicMin(&tpq[s], (tpq[s] & 0xFFFF0000u) | k);
}

__device__ __forceinline__ bool is_multi(const uint32_t *multi, uint32_t s) { return (multi[s >> 5] >> (s & 31)) & 1u; }

__device__ __forceinline__ bool decided_before(uint32_t st, uint32_t wave) {
  return (st & 3u) != kUndecided && (st >> 2) < wave;
}

// Exclusive scan of v[0 .. n) in place; ends with a barrier.
template <int T>
__device__ void block_exclusive_scan(uint32_t *v, uint32_t n, uint32_t *warp_sums) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
  const uint32_t per = (n + T - 1) / T;
  const uint32_t lo = min(tid * per, n), hi = min(lo + per, n);
  uint32_t sum = 0;
  for (uint32_t i = lo; i < hi; ++i) sum += v[i];
  uint32_t x = sum;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if ((int)lane >= off) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const uint32_t w0 = lane < (uint32_t)(T / 32) ? warp_sums[lane] : 0u;
    uint32_t w = w0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
      if ((int)lane >= off) w += y;
    }
    if (lane < (uint32_t)(T / 32)) warp_sums[lane] = w - w0;
  }
  __syncthreads();
  uint32_t run = warp_sums[wid] + x - sum;
  for (uint32_t i = lo; i < hi; ++i) {
    const uint32_t c = v[i];
    v[i] = run;
    run += c;
  }
  __syncthreads();
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  return x;
}

// pi of round `round` of chain ch into perm (shared or global memory): keys
// K(i) = Philox4x64-10((i >> 2, round, 0, 0); (seed, 0))[i & 3] and bucket
// counts (two Philox blocks per thread at a time, independent so that they
// overlap), a scan, the positions scattered by bucket, then each position's
// rank in its bucket in (K, i) order.  Returns l (exact laziness; L
// otherwise).  Every thread of the CTA calls it; it ends with a barrier.
template <int T>
__device__ __forceinline__ uint32_t sort_round(const ChainDesc &ch, unsigned long long round, uint32_t m, uint32_t L,
                                               uint32_t nb_log2, unsigned long long *keys, uint32_t *cnt,
                                               uint16_t *scat, uint16_t *perm, uint32_t *s_warp, uint32_t *s_ell) {
  const uint32_t tid = threadIdx.x, nb = 1u << nb_log2, shift = 64 - nb_log2;
  const bool exact = ch.exact_ell && ch.lazy_threshold;
  for (uint32_t b = tid; b < nb; b += T) cnt[b] = 0;
  if (tid == 0) *s_ell = 0;
  __syncthreads();
  const uint32_t nq = (m + 3) / 4;
  for (uint32_t q = tid; q < nq; q += 2 * T) {
    if (q + T < nq) {
      const U64x4 w0 = philox(q, round, 0, 0, ch.seed, 0);
      const U64x4 w1 = philox(q + T, round, 0, 0, ch.seed, 0);
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) {
        const uint32_t x0 = 4 * q + u, x1 = 4 * (q + T) + u;
        keys[x0] = w0.w[u];
        atomicAdd(&cnt[(uint32_t)(w0.w[u] >> shift)], 1u);
        if (x1 < m) {
          keys[x1] = w1.w[u];
          atomicAdd(&cnt[(uint32_t)(w1.w[u] >> shift)], 1u);
        }
      }
    } else {
      const U64x4 w0 = philox(q, round, 0, 0, ch.seed, 0);
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) {
        const uint32_t x0 = 4 * q + u;
        if (x0 < m) {
          keys[x0] = w0.w[u];
          atomicAdd(&cnt[(uint32_t)(w0.w[u] >> shift)], 1u);
        }
      }
    }
  }
  if (exact) {
    uint32_t n = 0;
    const uint32_t nl = (L + 3) / 4;
    for (uint32_t q = tid; q < nl; q += 2 * T) {
      const U64x4 w0 = philox(q, round, 1, 0, ch.seed, 0);
      const U64x4 w1 = philox(q + T, round, 1, 0, ch.seed, 0);
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) {
        n += (4 * q + u < L && w0.w[u] >= ch.lazy_threshold) ? 1u : 0u;
        n += (4 * (q + T) + u < L && w1.w[u] >= ch.lazy_threshold) ? 1u : 0u;
      }
    }
    n = warp_sum(n);
    if ((tid & 31u) == 0 && n) atomicAdd(s_ell, n);
  }
  __syncthreads();
  const uint32_t ell = exact ? *s_ell : L;
  block_exclusive_scan<T>(cnt, nb, s_warp);
  for (uint32_t x = tid; x < m; x += T) scat[atomicAdd(&cnt[(uint32_t)(keys[x] >> shift)], 1u)] = (uint16_t)x;
  __syncthreads();
  // cnt[b] is now the end of bucket b; each position's place in its bucket
  // is the number of the bucket's positions before it in (K, i) order
  for (uint32_t y = tid; y < m; y += T) {
    const uint32_t x = scat[y];
    const unsigned long long kx = keys[x];
    const uint32_t b = (uint32_t)(kx >> shift);
    const uint32_t lo = b ? cnt[b - 1] : 0u, hi = cnt[b];
    uint32_t r = 0;
    for (uint32_t z = lo; z < hi; ++z) {
      const uint32_t u = scat[z];
      const unsigned long long ku = keys[u];
      r += (ku < kx || (ku == kx && u < x)) ? 1u : 0u;
    }
    perm[lo + r] = (uint16_t)x;
  }
  __syncthreads();
  return ell;
}

template <int T>
__global__ void __launch_bounds__(T, 1024 / T) k_round_resident(RoundArgs a, ResidentJob job) {
  extern __shared__ __align__(16) unsigned char res_dyn[];
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_ell;
  __shared__ uint32_t s_wave[3][3];  // per wave (mod 3): undecided, decided, turned illegal on an id
                                     // with two inserters or more
  const uint32_t tid = threadIdx.x;
  const uint32_t c = job.jobs[blockIdx.x];
  const ChainDesc ch = a.chains[c];
  const uint32_t m = ch.m, L = ch.L;
  if (m < 2 || m > kResidentMaxEdges) return;  // the host sends only chains that qualify
  const ResLayout lay = res_layout(m);
  uint32_t *const E = reinterpret_cast<uint32_t *>(res_dyn);
  uint16_t *const scat = reinterpret_cast<uint16_t *>(res_dyn + lay.scat);   // positions by bucket
  uint32_t *const tslot = reinterpret_cast<uint32_t *>(res_dyn + lay.scat);  // later: the targets' slots
  uint16_t *const perm = reinterpret_cast<uint16_t *>(res_dyn + lay.perm);   // pi
  uint16_t *const status = reinterpret_cast<uint16_t *>(res_dyn + lay.status);
  unsigned long long *const keys = reinterpret_cast<unsigned long long *>(res_dyn + lay.region);
  uint32_t *const cnt = reinterpret_cast<uint32_t *>(res_dyn + lay.region + align16(8 * m));
  uint32_t *const tkey = reinterpret_cast<uint32_t *>(res_dyn + lay.region);
  const uint32_t nb_log2 = lay.nb_log2, slog2 = lay.slog2, S = 1u << slog2;
  uint32_t *const tpq = tkey + S;
  uint32_t *const multi = reinterpret_cast<uint32_t *>(res_dyn + lay.multi);
  const unsigned long long R0 = *(volatile unsigned long long *)&a.ctl->pool_round;

  // the list by position, with the last round's decision of each pair of
  // slots applied (Def. 1's rewiring of a legal switch)
  bool bad = false;
  const bool apply = R0 > ch.added;
  for (uint32_t s = tid; s < m; s += T) {
    const uint32_t pos = a.cpos[ch.slot_base + s];
    unsigned long long e = a.cedge[ch.slot_base + s];
    const uint32_t k = s >> 1;
    if (apply && k < L && (a.status[ch.switch_base + k] & 3u) == kLegal) {
      const uint32_t s0 = ch.slot_base + 2 * k;
      unsigned long long e3, e4;
      tau_g(a.cpos[s0] < a.cpos[s0 + 1] ? 1u : 0u, a.cedge[s0], a.cedge[s0 + 1], e3, e4);
      e = (s & 1u) ? e4 : e3;
    }
    const uint32_t lo = (uint32_t)(e >> 32), hi = (uint32_t)e;
    if (pos >= m || lo >= hi || hi >= kResidentMaxNodes) {
      bad = true;
      continue;
    }
    E[pos] = (lo << 16) | hi;
  }
  if (__syncthreads_or(bad)) {
    if (tid == 0) atomicOr(&a.ctl->err, kErrRecord);
    return;
  }

  uint32_t acc = 0, rloop = 0, rexist = 0, rlazy = 0;  // this thread's tallies
  const bool exact = ch.exact_ell && ch.lazy_threshold;
  const bool per_switch = ch.lazy_threshold && !ch.exact_ell;
  uint32_t err = 0;
  for (uint32_t t = 0; t < job.rounds && !err; ++t) {
    const unsigned long long round = ch.start_round + (R0 + t - ch.join);
    // 1. pi of this round (sorted here, or beforehand on other SMs) and l
    uint32_t ell;
    if (job.pbuf) {
      const size_t jg = (size_t)t * job.njobs + job.job_base + blockIdx.x;
      const uint16_t *src = job.pbuf + jg * job.pstride;
      for (uint32_t y = tid; y < m; y += T) perm[y] = __ldcg(&src[y]);
      ell = exact ? __ldcg(&job.ebuf[jg]) : L;
      __syncthreads();
    } else {
      ell = sort_round<T>(ch, round, m, L, nb_log2, keys, cnt, scat, perm, s_warp, &s_ell);
    }

    // 2. switches: outright rejects, targets into the table (keys are dead)
    for (uint32_t s = tid; s < S; s += T) {
      tkey[s] = kEmpty32;
      tpq[s] = 0xFFFFFFFFu;
    }
    for (uint32_t w = tid; w < S / 32; w += T) multi[w] = 0;
    __syncthreads();
    bool full = false;
    for (uint32_t k = tid; k < L; k += T) {
      const uint32_t i = perm[2 * k], j = perm[2 * k + 1];
      const bool lazy =
          exact ? k >= ell
                : (per_switch && word_of(philox(k >> 2, round, 1, 0, ch.seed, 0), k & 3) < ch.lazy_threshold);
      uint32_t e3 = 0, e4 = 0;
      const uint32_t code = lazy ? kCodeLazy : tau16(i < j ? 1u : 0u, E[i], E[j], e3, e4);
      if (code) {
        status[k] = (uint16_t)kIllegal;  // known before the first wave (wave field 0)
        if (code == kCodeLazy) ++rlazy;
        else if (code == kCodeLoop) ++rloop;
        else ++rexist;
        continue;
      }
      status[k] = (uint16_t)kUndecided;
      if (!tab_insert(tkey, slog2, e3) || !tab_insert(tkey, slog2, e4)) full = true;
    }
    if (__syncthreads_or(full)) {
      err = kErrTableFull;
      break;
    }
    // every switch that is not known to fail registers as an inserter of its
    // targets (smallest q per id) and keeps its targets' slots
    bool lost = false;  // a target not found (never, by construction)
    for (uint32_t k = tid; k < L; k += T) {
      if (status[k] != kUndecided) continue;
      const uint32_t i = perm[2 * k], j = perm[2 * k + 1];
      uint32_t e3, e4;
      tau16(i < j ? 1u : 0u, E[i], E[j], e3, e4);
      const uint32_t s3 = tab_find(tkey, slog2, e3), s4 = tab_find(tkey, slog2, e4);
      if (s3 >= S || s4 >= S) {
        lost = true;
        continue;
      }
      tslot[k] = s3 | (s4 << 16);
      // a slot whose q was already set has a second inserter
      if ((tab_qmin(tpq, s3, k) & 0xFFFFu) != kQ16None) atomicOr(&multi[s3 >> 5], 1u << (s3 & 31));
      if ((tab_qmin(tpq, s4, k) & 0xFFFFu) != kQ16None) atomicOr(&multi[s4 >> 5], 1u << (s4 & 31));
    }
    if (__syncthreads_or(lost)) {
      err = kErrTableFull;
      break;
    }

    // 3. erasers of the edges that are targets
    for (uint32_t s = tid; s < m; s += T) {
      const uint32_t slot = tab_find(tkey, slog2, E[perm[s]]);
      if (slot < S) {
        const uint32_t p = (s >> 1) < L ? (s >> 1) : kP16Keep;
        atomicAnd(&tpq[slot], (p << 16) | 0xFFFFu);
      }
    }
    if (tid < 9) s_wave[tid / 3][tid % 3] = 0;
    __syncthreads();

    // 4. waves
    uint32_t wave = 1, entering = L;
    bool requeue = false;
    for (;;) {
      if (job.final && t + 1 == job.rounds && tid == 0 && wave >= 2 && wave < kWaveHist)
        atomicAdd(&job.last_pending[wave], entering);
      if (tid < 3) s_wave[(wave + 1) % 3][tid] = 0;  // read two waves ago, written next wave
      if (requeue) {
        // q of every id with two inserters or more goes back to "none", and
        // the inserters that are not illegal register again; an id with one
        // inserter keeps it as q, since only that inserter looks at the id's q
        // (the switches known to fail before the first wave never registered)
        for (uint32_t k = tid; k < L; k += T) {
          if (status[k] == (uint16_t)kIllegal) continue;
          const uint32_t ts = tslot[k], s3 = ts & 0xFFFFu, s4 = ts >> 16;
          if (is_multi(multi, s3)) atomicOr(&tpq[s3], 0xFFFFu);
          if (is_multi(multi, s4)) atomicOr(&tpq[s4], 0xFFFFu);
        }
        __syncthreads();
        for (uint32_t k = tid; k < L; k += T) {
          if ((status[k] & 3u) == kIllegal) continue;
          const uint32_t ts = tslot[k], s3 = ts & 0xFFFFu, s4 = ts >> 16;
          if (is_multi(multi, s3)) tab_qmin(tpq, s3, k);
          if (is_multi(multi, s4)) tab_qmin(tpq, s4, k);
        }
        __syncthreads();
      }
      uint32_t und = 0, dec = 0, ill = 0;
      for (uint32_t k = tid; k < L; k += T) {
        if (status[k] != kUndecided) continue;
        const uint32_t ts = tslot[k];
        bool illegal = false, wait = false;
#pragma unroll
        for (int x = 0; x < 2; ++x) {
          const uint32_t pq = tpq[x ? ts >> 16 : ts & 0xFFFFu];
          const uint32_t p = pq >> 16, q = pq & 0xFFFFu;
          if (p != kP16None) {      // the target is in E when the round starts
            if (p > k) {
              illegal = true;       // erased after k, or never
            } else {
              const uint32_t sp = status[p];
              if (!decided_before(sp, wave)) wait = true;
              else if ((sp & 3u) == kIllegal) illegal = true;  // its eraser failed
            }
          }
          if (q != kQ16None && q < k) {  // an earlier switch may insert it first
            const uint32_t sq = status[q];
            if (!decided_before(sq, wave)) wait = true;
            else if ((sq & 3u) == kLegal) illegal = true;
          }
        }
        if (!illegal && wait) {
          ++und;
          continue;
        }
        status[k] = (uint16_t)((wave << 2) | (illegal ? kIllegal : kLegal));
        ++dec;
        ill += (illegal && (is_multi(multi, ts & 0xFFFFu) || is_multi(multi, ts >> 16))) ? 1u : 0u;
      }
      und = warp_sum(und);
      dec = warp_sum(dec);
      ill = warp_sum(ill);
      uint32_t *const ws = s_wave[wave % 3];
      if ((tid & 31u) == 0) {
        if (und) atomicAdd(&ws[0], und);
        if (dec) atomicAdd(&ws[1], dec);
        if (ill) atomicAdd(&ws[2], ill);
      }
      __syncthreads();
      const uint32_t U = ws[0], D = ws[1], I = ws[2];
      if (U == 0) break;
      if (D == 0) {             // impossible for a valid round: the smallest undecided switch decides
        err = kErrNoProgress;
        break;
      }
      if (wave >= job.wave_cap) {
        err = kErrWaveCap;
        break;
      }
      ++wave;
      entering = U;
      requeue = I != 0;
    }
    if (err) break;
    if (tid == 0) atomicMax(&job.round_waves[t], wave);

    // 5. legal switches rewrite their positions
    for (uint32_t k = tid; k < L; k += T) {
      const uint32_t st = status[k];
      if ((st & 3u) == kLegal) {
        const uint32_t i = perm[2 * k], j = perm[2 * k + 1];
        uint32_t e3, e4;
        tau16(i < j ? 1u : 0u, E[i], E[j], e3, e4);
        E[i] = e3;
        E[j] = e4;
        ++acc;
      } else if ((st >> 2) != 0) {
        ++rexist;               // illegal by a wave: a target was in E when it ran
      }
    }
    __syncthreads();
  }
  if (err) {
    if (tid == 0) atomicOr(&a.ctl->err, err);
    return;
  }
  // the list back to the chain's slots, by position, nothing pending
  for (uint32_t x = tid; x < m; x += T) {
    const uint32_t e = E[x];
    a.cpos[ch.slot_base + x] = x;
    a.cedge[ch.slot_base + x] = ((unsigned long long)(e >> 16) << 32) | (e & 0xFFFFu);
  }
  for (uint32_t k = tid; k < L; k += T) a.status[ch.switch_base + k] = 0u;
  acc = warp_sum(acc);
  rloop = warp_sum(rloop);
  rexist = warp_sum(rexist);
  rlazy = warp_sum(rlazy);
  if ((tid & 31u) == 0) {
    if (acc) {
      atomicAdd(&a.st->accepted, (unsigned long long)acc);
      atomicAdd(&a.chain_accepted[c], (unsigned long long)acc);
    }
    if (rloop) atomicAdd(&a.st->rej_loop, (unsigned long long)rloop);
    if (rexist) atomicAdd(&a.st->rej_exists, (unsigned long long)rexist);
    if (rlazy) atomicAdd(&a.st->lazy, (unsigned long long)rlazy);
  }
}

// The permutations of all rounds of a launch, one CTA per (chain, round),
// ahead of the resident kernel, for pools of few chains: the keys and the
// sort depend only on the chain's seed, round number and m, never on its
// list, so other SMs sort them while the chain's own CTA would otherwise
// sit in the sort phases of each round.
template <int T>
__global__ void __launch_bounds__(T, 1024 / T) k_resident_perm(RoundArgs a, ResidentJob job) {
  extern __shared__ __align__(16) unsigned char res_dyn[];
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_ell;
  const ChainDesc ch = a.chains[job.jobs[blockIdx.x]];
  const uint32_t m = ch.m;
  if (m < 2 || m > kResidentMaxEdges) return;
  const ResLayout lay = res_layout(m);
  unsigned long long *const keys = reinterpret_cast<unsigned long long *>(res_dyn);
  uint32_t *const cnt = reinterpret_cast<uint32_t *>(res_dyn + align16(8 * m));
  uint16_t *const scat = reinterpret_cast<uint16_t *>(res_dyn + align16(8 * m) + 4 * (1u << lay.nb_log2));
  const unsigned long long R0 = *(volatile unsigned long long *)&a.ctl->pool_round;
  const uint32_t t = blockIdx.y;
  const size_t jg = (size_t)t * job.njobs + job.job_base + blockIdx.x;
  const uint32_t ell = sort_round<T>(ch, ch.start_round + (R0 + t - ch.join), m, ch.L, lay.nb_log2, keys, cnt, scat,
                                     job.pbuf + jg * job.pstride, s_warp, &s_ell);
  if (threadIdx.x == 0) job.ebuf[jg] = ell;
}

__host__ __device__ inline uint32_t perm_smem_bytes(uint32_t m) {
  const ResLayout l = res_layout(m < 2 ? 2 : m);
  return align16(8 * m) + 4 * (1u << l.nb_log2) + align16(2 * m);
}

// The launch's rounds into the statistics (each round's wave count is the
// largest over its chains, as in the general path) and the pool round on.
__global__ void k_resident_fold(RoundArgs a, ResidentJob job) {
  __shared__ unsigned long long hist[kWaveHist];
  __shared__ unsigned long long total, most;
  const uint32_t tid = threadIdx.x;
  for (uint32_t i = tid; i < kWaveHist; i += blockDim.x) hist[i] = 0;
  if (tid == 0) total = most = 0;
  __syncthreads();
  for (uint32_t t = tid; t < job.rounds; t += blockDim.x) {
    const uint32_t w = job.round_waves[t];
    atomicAdd(&hist[w < kWaveHist ? w : kWaveHist - 1], 1ull);
    atomicAdd(&total, (unsigned long long)w);
    atomicMax(&most, (unsigned long long)w);
  }
  __syncthreads();
  if (a.any_work) {
    for (uint32_t i = tid; i < kWaveHist; i += blockDim.x)
      if (hist[i]) a.st->wave_hist[i] += hist[i];
  }
  if (tid == 0) {
    if (a.any_work) {
      a.st->waves_total += total;
      if (most > a.st->waves_max) a.st->waves_max = most;
    }
    if (job.final) {
      a.ctl->waves = (a.any_work && job.rounds) ? job.round_waves[job.rounds - 1] : 0u;
      a.st->last_pending[1] = a.switch_hw;
      for (uint32_t w = 2; w < kWaveHist; ++w) a.st->last_pending[w] = job.last_pending[w];
    }
    a.ctl->pool_round += job.rounds;
  }
}

// The most edges a chain of each class has (CTAs of 1024, 512, 256 and 128
// threads).
constexpr uint32_t kClassMaxEdges[kResidentClasses] = {kResidentMaxEdges, 4096, 2048, 1024};

template <int T>
cudaError_t launch_class(const RoundArgs &a, const ResidentJob &j, uint32_t n, uint32_t max_m, cudaStream_t s) {
  if (j.pbuf) k_resident_perm<T><<<dim3(n, j.rounds), T, perm_smem_bytes(max_m), s>>>(a, j);
  k_round_resident<T><<<n, T, res_layout(max_m < 2 ? 2 : max_m).bytes, s>>>(a, j);
  return cudaGetLastError();
}

}  // namespace

uint32_t resident_class(uint32_t m) {
  uint32_t c = 0;
  while (c + 1 < kResidentClasses && m <= kClassMaxEdges[c + 1]) ++c;
  return c;
}

size_t resident_smem_bytes(uint32_t m) { return res_layout(m).bytes; }

cudaError_t prepare_resident() {
  cudaError_t e = cudaFuncSetAttribute(k_round_resident<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)resident_smem_bytes(kClassMaxEdges[0]));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_round_resident<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)resident_smem_bytes(kClassMaxEdges[1]));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_round_resident<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)resident_smem_bytes(kClassMaxEdges[2]));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_round_resident<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)resident_smem_bytes(kClassMaxEdges[3]));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_resident_perm<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)perm_smem_bytes(kClassMaxEdges[0]));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_resident_perm<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)perm_smem_bytes(kClassMaxEdges[1]));
  return e;
}

cudaError_t launch_round_resident(const RoundArgs &a, const uint32_t *jobs, const uint32_t (&count)[kResidentClasses],
                                  const uint32_t (&max_m)[kResidentClasses], uint32_t rounds, uint32_t *round_waves,
                                  uint32_t *last_pending, bool final, uint16_t *pbuf, uint32_t *ebuf, uint32_t pstride,
                                  cudaStream_t s, uint32_t *launches) {
  ResidentJob j;
  j.rounds = rounds;
  j.pbuf = pbuf;
  j.ebuf = ebuf;
  j.pstride = pstride;
  j.njobs = 0;
  for (uint32_t c = 0; c < kResidentClasses; ++c) j.njobs += count[c];
  j.round_waves = round_waves;
  j.last_pending = last_pending;
  j.final = final ? 1u : 0u;
  // status words hold the wave in 14 bits; a round needs at most L + 1 <= 6145 waves
  const uint32_t cap = a.max_waves ? a.max_waves : kDefaultWaveCap;
  j.wave_cap = cap < 16383u ? cap : 16383u;
  uint32_t off = 0;
  for (uint32_t c = 0; c < kResidentClasses; ++c) {
    if (!count[c]) continue;
    j.jobs = jobs + off;
    j.job_base = off;
    off += count[c];
    cudaError_t e = cudaSuccess;
    switch (c) {
      case 0: e = launch_class<1024>(a, j, count[c], max_m[c], s); break;
      case 1: e = launch_class<512>(a, j, count[c], max_m[c], s); break;
      case 2: e = launch_class<256>(a, j, count[c], max_m[c], s); break;
      default: e = launch_class<128>(a, j, count[c], max_m[c], s); break;
    }
    if (e != cudaSuccess) return e;
    *launches += pbuf ? 2 : 1;
  }
  j.jobs = jobs;
  k_resident_fold<<<1, 256, 0, s>>>(a, j);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace gesmc
