// ParES (Algorithm 2 of arXiv 2111.03005): exact parallel ES-MC on one GB300.
//
// ES-MC runs independent edge switches sigma_k = (i, j, g) one after
// another (Def. 1's chain).  Algorithm 2 cuts the sequence into supersteps:
// maximal runs of consecutive switches of which no two share a source
// position, found with a first-touch table (each switch of a window writes
// its index into the entries of its two positions with a minimum, and the
// first switch that finds a smaller index there starts the next superstep;
// the table is a shared-memory hash table keyed by position).  A
// superstep has no source dependencies, so ParallelSuperstep (Algorithm 1)
// performs it with the sequential outcome: each target edge exists when its
// switch runs iff it was in E at the superstep's start and its eraser (the
// switch whose source it is) is not an earlier legal switch, or an earlier
// legal switch inserts it.
//
// Supersteps of ES-MC hold about sqrt(m) switches (the birthday bound), so
// one CTA runs all supersteps of one chain: the switches of a superstep, the
// table of its erasers and the lists of its inserters live in shared memory,
// the waves of Algorithm 1 are separated by __syncthreads, and the list E
// (position order) and the edge set H (open addressing over canonical ids,
// tombstones on erase) live in HBM.  Many chains run as many CTAs of one
// launch.  A superstep is also cut at the window size (32 to 1024 switches,
// by the chain's size); any cut into consecutive runs without source
// dependencies gives the sequential result.  When tombstones pile up, the
// set is rebuilt from the list between supersteps: in place by the CTA for
// the smaller windows, on the whole GPU between launches for the largest.
#include "device_util.cuh"
#include "gesmc_internal.cuh"

namespace gesmc {
namespace {

constexpr uint32_t kNil = 0xFFFFFFFFu;
constexpr uint32_t kNoTouch = 0xFFFFFFFFu;
constexpr uint8_t kEsUndecided = 0, kEsLegal = 1, kEsIllegal = 2;
// Window sizes by chain size (supersteps hold about 0.63 sqrt(m) switches:
// 450 at 2^19, 160 at 2^16, 57 at 2^13): chains of at least 2^19 edges run
// windows of 1024 switches, chains of at least 2^16 windows of 256 on CTAs of
// 256 threads (six per SM), chains of at least 2^13 windows of 128, smaller
// ones windows of 32 on one warp each (up to 32 per SM), whose barriers cost
// next to nothing.
constexpr uint32_t kEsBigChain = 1u << 19;
constexpr uint32_t kEsMidChain = 1u << 16;
constexpr uint32_t kEsSmallChain = 1u << 13;

__device__ __forceinline__ uint32_t hash32(unsigned long long key) { return (uint32_t)mix64(key); }

// ---------------------------------------------------------------- the edge set H
// Open addressing with linear probing from h & mask (h = hash32(key)).
// Insert a key that is not in the set into the first empty or tombstone
// slot of its probe sequence.  Returns 0 (empty slot taken), 1 (tombstone
// reused) or -1 (table full).
__device__ __forceinline__ int hset_insert(unsigned long long *H, uint32_t mask, unsigned long long key, uint32_t h) {
  uint32_t s = h & mask;
  for (uint32_t n = 0; n <= mask; ++n) {
    const unsigned long long cur = __ldcg(&H[s]);
    if (cur == kEmptyKey || cur == kTombKey) {
      if (atomicCAS(&H[s], cur, key) == cur) return cur == kTombKey ? 1 : 0;
      continue;  // taken meanwhile: look at the same slot again
    }
    s = (s + 1) & mask;
  }
  return -1;
}

// Two keys at once: both probe chains advance together, so that their loads
// are in flight together (one HBM latency per step for the pair).
// Presence: the first slots' loads are passed in (issued by the caller
// before other work), bit w of the result says key w is in the set.
__device__ __forceinline__ uint32_t hset_contains2(const unsigned long long *H, uint32_t mask,
                                                   const unsigned long long (&key)[2], const uint32_t (&h)[2],
                                                   unsigned long long (&cur)[2]) {
  uint32_t s[2] = {h[0] & mask, h[1] & mask}, found = 0, done = 0;
  for (uint32_t n = 0; n <= mask; ++n) {
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      if ((done >> w) & 1u) continue;
      if (cur[w] == key[w]) {
        found |= 1u << w;
        done |= 1u << w;
      } else if (cur[w] == kEmptyKey) {
        done |= 1u << w;
      } else {
        s[w] = (s[w] + 1) & mask;
      }
    }
    if (done == 3u) break;
#pragma unroll
    for (int w = 0; w < 2; ++w)
      if (!((done >> w) & 1u)) cur[w] = __ldcg(&H[s[w]]);
  }
  return found;
}

__device__ __forceinline__ void hset_erase2(unsigned long long *H, uint32_t mask, const unsigned long long (&key)[2],
                                            const uint32_t (&h)[2]) {
  uint32_t s[2] = {h[0] & mask, h[1] & mask}, done = 0;
  for (uint32_t n = 0; n <= mask && done != 3u; ++n) {
    unsigned long long cur[2];
#pragma unroll
    for (int w = 0; w < 2; ++w)
      if (!((done >> w) & 1u)) cur[w] = __ldcg(&H[s[w]]);
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      if ((done >> w) & 1u) continue;
      if (cur[w] == key[w]) {
        H[s[w]] = kTombKey;
        done |= 1u << w;
      } else if (cur[w] == kEmptyKey) {
        done |= 1u << w;
      } else {
        s[w] = (s[w] + 1) & mask;
      }
    }
  }
}

// Insert two keys that are not in the set, each into the first empty or
// tombstone slot of its probe sequence.  r[w] = 0 (empty slot taken), 1
// (tombstone reused) or -1 (table full).
__device__ __forceinline__ void hset_insert2(unsigned long long *H, uint32_t mask, const unsigned long long (&key)[2],
                                             const uint32_t (&h)[2], int (&r)[2]) {
  uint32_t s[2] = {h[0] & mask, h[1] & mask}, done = 0;
  uint32_t left[2] = {mask + 1, mask + 1};  // probes each key may still take
  r[0] = r[1] = -1;
  while (done != 3u) {
    unsigned long long cur[2];
#pragma unroll
    for (int w = 0; w < 2; ++w)
      if (!((done >> w) & 1u)) cur[w] = __ldcg(&H[s[w]]);
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      if ((done >> w) & 1u) continue;
      if (left[w] == 0) {  // every slot looked at: table full
        done |= 1u << w;
        continue;
      }
      --left[w];
      if (cur[w] == kEmptyKey || cur[w] == kTombKey) {
        if (atomicCAS(&H[s[w]], cur[w], key[w]) == cur[w]) {
          r[w] = cur[w] == kTombKey ? 1 : 0;
          done |= 1u << w;
        }
        // taken meanwhile: look at the same slot again
      } else {
        s[w] = (s[w] + 1) & mask;
      }
    }
  }
}

// ---------------------------------------------------------------- shared memory
// Per CTA, for windows of B switches (one per thread) and tables of S = 4B
// slots: a region that holds the first-touch table while the window is cut
// (position keys and minima, u32) and the erasers' and inserters' key tables
// afterwards (u64), then the erasers' switches, the inserters' list heads and
// links, and every switch's state.  Everything else a switch needs (its
// positions, edges, hashes, outcome) stays in its thread's registers.
template <int B>
struct EsShape {
  static constexpr int kSlots = 4 * B;
  static constexpr int kSlotsLog2 = B == 1024 ? 12 : B == 256 ? 10 : B == 128 ? 9 : B == 32 ? 7 : -1;
  static constexpr size_t kRegion = 16ull * kSlots;
  static constexpr size_t kBytes = kRegion + 4ull * (2 * kSlots + 2 * B) + B;
  static_assert(kSlotsLog2 > 0, "window of 32, 128, 256 or 1024 switches");
};

template <int B>
struct EsSmem {
  unsigned long long *skey, *ikey;  // key tables (after the cut)
  uint32_t *pkey, *pmin;            // first-touch table (until the cut); the same bytes
  uint32_t *sval, *ihead, *tnext;
  uint8_t *st;
};

template <int B>
__device__ __forceinline__ EsSmem<B> es_smem() {
  extern __shared__ unsigned long long es_dyn[];
  constexpr int S = EsShape<B>::kSlots;
  EsSmem<B> m;
  m.skey = es_dyn;
  m.ikey = es_dyn + S;
  m.pkey = reinterpret_cast<uint32_t *>(es_dyn);
  m.pmin = m.pkey + S;
  uint32_t *q = reinterpret_cast<uint32_t *>(es_dyn + 2 * S);
  m.sval = q;
  m.ihead = q + S;
  m.tnext = q + 2 * S;
  m.st = reinterpret_cast<uint8_t *>(q + 2 * S + 2 * B);
  return m;
}

// Sources of the superstep's switches (key -> switch) and its targets (key
// -> list of (switch, which) entries through next[]); h = hash32(key).
template <int S>
__device__ __forceinline__ uint32_t table_slot(unsigned long long *keys, unsigned long long key, uint32_t h,
                                               bool claim) {
  uint32_t s = h & (S - 1);
  for (int n = 0; n < S; ++n) {
    const unsigned long long cur = keys[s];
    if (cur == key) return s;
    if (cur == kEmptyKey) {
      if (!claim) return kNil;
      const unsigned long long prev = atomicCAS(&keys[s], kEmptyKey, key);
      if (prev == kEmptyKey || prev == key) return s;
    }
    s = (s + 1) & (S - 1);
  }
  return kNil;
}

// First touches of a window (Algorithm 2's insert_if_min): position ->
// smallest switch of the window that has it as a source position.  At most
// 2B positions in S = 4B slots; a position is below 2^31, so never kNil.
template <int S, int LOG2>
__device__ __forceinline__ void touch_first(uint32_t *pkey, uint32_t *pmin, uint32_t pos, uint32_t x) {
  uint32_t s = (pos * 0x9E3779B1u) >> (32 - LOG2);
  for (int n = 0; n < S; ++n) {
    uint32_t cur = pkey[s];
    if (cur == kNil) {
      cur = atomicCAS(&pkey[s], kNil, pos);
      if (cur == kNil) cur = pos;
    }
    if (cur == pos) {
      atomicMin(&pmin[s], x);
      return;
    }
    s = (s + 1) & (S - 1);
  }
}

template <int S, int LOG2>
__device__ __forceinline__ uint32_t first_touch(const uint32_t *pkey, const uint32_t *pmin, uint32_t pos) {
  uint32_t s = (pos * 0x9E3779B1u) >> (32 - LOG2);
  for (int n = 0; n < S; ++n) {
    const uint32_t cur = pkey[s];
    if (cur == pos) return pmin[s];
    if (cur == kNil) break;
    s = (s + 1) & (S - 1);
  }
  return kNoTouch;
}

// The region as the first-touch table / as the key tables (with the list heads).
template <int B>
__device__ __forceinline__ void clear_touch(const EsSmem<B> &sm) {
  for (uint32_t t = threadIdx.x; t < (uint32_t)EsShape<B>::kSlots; t += B) {
    sm.pkey[t] = kNil;
    sm.pmin[t] = kNoTouch;
  }
}

template <int B>
__device__ __forceinline__ void clear_tables(const EsSmem<B> &sm) {
  for (uint32_t t = threadIdx.x; t < (uint32_t)EsShape<B>::kSlots; t += B) {
    sm.skey[t] = kEmptyKey;
    sm.ikey[t] = kEmptyKey;
    sm.ihead[t] = kNil;
  }
}

// ---------------------------------------------------------------- kernels
// H <- empty, for every job (blockIdx.y = job).
__global__ void k_es_clear(const EsJob *jobs, uint32_t job_off, bool only_stopped) {
  const EsJob jb = jobs[job_off + blockIdx.y];
  if (jb.m < 2 || (only_stopped && !jb.stopped)) return;  // no list, no set; or a set that needs no rebuild
  const unsigned long long cap = 1ull << jb.hlog2;
  const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s < cap; s += nth)
    jb.H[s] = kEmptyKey;
}

// H <- the entries of E.
__global__ void k_es_fill(const EsJob *jobs, uint32_t job_off, uint32_t *err, bool only_stopped) {
  const EsJob jb = jobs[job_off + blockIdx.y];
  if (jb.m < 2 || (only_stopped && !jb.stopped)) return;
  const uint32_t mask = (uint32_t)((1ull << jb.hlog2) - 1);
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < jb.m; s += gridDim.x * blockDim.x) {
    const unsigned long long e = jb.E[s];
    if (hset_insert(jb.H, mask, e, hash32(e)) < 0) atomicOr(err, kErrTableFull);
  }
}

// One CTA per job: switches k0 .. k0 + count - 1 of the job's chain, in
// windows of B switches (thread x holds switch x of the window).
// A CTA of the largest variant does not rebuild its chain's edge set itself
// (one SM reinserting millions of ids): it stops after the superstep that
// passes the tombstone limit (an eighth of the slots: rebuilds are cheap on
// the whole GPU, and fewer tombstones keep the probe chains short), records
// how far it got in jobs_out (k0, count advanced, stopped = 1, *nstop
// counted), and the host rebuilds the set on the whole GPU and launches the
// variant again; a finished job is left with count = 0, which a launch
// again skips.  The smaller variants rebuild in place at a quarter.
template <int B, bool kStopToRebuild>
__device__ __forceinline__ void es_run_body(const EsJob *jobs, uint32_t job_off, StatsDev *stats,
                                            unsigned long long *chain_acc, uint32_t *err, EsJob *jobs_out,
                                            uint32_t *nstop) {
  constexpr int S = EsShape<B>::kSlots, LOG2 = EsShape<B>::kSlotsLog2;
  const EsJob jb = jobs[job_off + blockIdx.x];
  const EsSmem<B> sm = es_smem<B>();
  __shared__ uint32_t s_cut, s_tombs;
  const uint32_t x = threadIdx.x;
  uint32_t acc = 0, rej_loop = 0, rej_exists = 0;
  if (jb.m < 2) {  // no pair of positions: every requested switch is skipped
    if (x == 0 && jb.count) atomicAdd(&stats->lazy, jb.count);
    return;
  }
  bool stop = false;
  const uint32_t mask = (uint32_t)((1ull << jb.hlog2) - 1);
  if (x == 0) s_tombs = 0;  // the set was built from the list just before
  clear_touch(sm);
  __syncthreads();
  unsigned long long done = 0;  // switches run before a stop (largest variant)
  for (unsigned long long s = 0; s < jb.count;) {
    const uint32_t win = (uint32_t)min((unsigned long long)B, jb.count - s);
    // sample the window and mark first touches (Algorithm 2's insert_if_min)
    if (x == 0) s_cut = win;
    uint32_t i = 0, j = 0, g = 0;
    if (x < win) {
      const U64x4 w = philox(jb.k0 + s + x, 0, 2, 0, jb.seed, 0);
      i = (uint32_t)__umul64hi(w.w[0], (unsigned long long)jb.m);
      const uint32_t jj = (uint32_t)__umul64hi(w.w[1], (unsigned long long)(jb.m - 1));
      j = jj + (jj >= i ? 1u : 0u);
      g = (uint32_t)(w.w[2] >> 63);
      touch_first<S, LOG2>(sm.pkey, sm.pmin, i, x);
      touch_first<S, LOG2>(sm.pkey, sm.pmin, j, x);
    }
    __syncthreads();
    // the superstep ends before the first switch that shares a position with an earlier one
    if (x < win && (first_touch<S, LOG2>(sm.pkey, sm.pmin, i) < x || first_touch<S, LOG2>(sm.pkey, sm.pmin, j) < x))
      atomicMin(&s_cut, x);
    __syncthreads();
    const uint32_t n = s_cut;
    clear_tables(sm);  // the region becomes the key tables (the cut has read it)
    // sources, targets and the outright rules
    unsigned long long e1 = 0, e2 = 0, e3 = 0, e4 = 0;
    uint32_t h1 = 0, h2 = 0, h3 = 0, h4 = 0, code = 1;
    if (x < n) {
      e1 = __ldcg(&jb.E[i]);
      e2 = __ldcg(&jb.E[j]);
      code = tau_g(g, e1, e2, e3, e4);
      sm.st[x] = code ? kEsIllegal : kEsUndecided;
      if (code == kCodeLoop) ++rej_loop;
      else if (code) ++rej_exists;  // shared node: the targets re-create the sources
      if (!code) {
        h1 = hash32(e1);
        h2 = hash32(e2);
        h3 = hash32(e3);
        h4 = hash32(e4);
      }
    }
    __syncthreads();
    // erasers and inserters of the superstep; presence of the targets in E at its start (the first
    // probes of the edge set are issued before the shared-memory tables are filled, so that they overlap)
    uint32_t pres = 0;
    if (x < n && code == 0) {
      unsigned long long cur[2] = {__ldcg(&jb.H[h3 & mask]), __ldcg(&jb.H[h4 & mask])};
      uint32_t t = table_slot<S>(sm.skey, e1, h1, true);
      if (t != kNil) sm.sval[t] = x;
      t = table_slot<S>(sm.skey, e2, h2, true);
      if (t != kNil) sm.sval[t] = x;
      const unsigned long long tk[2] = {e3, e4};
      const uint32_t th[2] = {h3, h4};
      t = table_slot<S>(sm.ikey, e3, h3, true);
      if (t != kNil) sm.tnext[2 * x] = atomicExch(&sm.ihead[t], 2 * x);
      else atomicOr(err, kErrTableFull);
      t = table_slot<S>(sm.ikey, e4, h4, true);
      if (t != kNil) sm.tnext[2 * x + 1] = atomicExch(&sm.ihead[t], 2 * x + 1);
      else atomicOr(err, kErrTableFull);
      pres = hset_contains2(jb.H, mask, tk, th, cur);
    }
    __syncthreads();
    // waves (Algorithm 1): a switch decided in wave w only uses decisions of earlier waves
    uint8_t dec = x < n ? sm.st[x] : kEsIllegal;
    for (uint32_t wave = 1;; ++wave) {
      if (dec == kEsUndecided) {
        bool bad = false, wait = false;
        for (uint32_t w = 0; w < 2 && !bad; ++w) {
          const unsigned long long e = w ? e4 : e3;
          const uint32_t h = w ? h4 : h3;
          if ((pres >> w) & 1u) {  // in E at the start: present unless an earlier legal switch erased it
            const uint32_t t = table_slot<S>(sm.skey, e, h, false);
            const uint32_t p = t == kNil ? kNil : sm.sval[t];
            if (p == kNil || p >= x || sm.st[p] == kEsIllegal) bad = true;
            else if (sm.st[p] == kEsUndecided) wait = true;
          }
          if (bad) break;
          const uint32_t t = table_slot<S>(sm.ikey, e, h, false);
          for (uint32_t q = t == kNil ? kNil : sm.ihead[t]; q != kNil; q = sm.tnext[q]) {
            const uint32_t k = q >> 1;  // an earlier switch that inserts e
            if (k >= x) continue;
            if (sm.st[k] == kEsLegal) {
              bad = true;
              break;
            }
            if (sm.st[k] == kEsUndecided) wait = true;
          }
        }
        dec = bad ? kEsIllegal : (wait ? kEsUndecided : kEsLegal);
      }
      __syncthreads();  // every read of this wave's states is done
      if (x < n) sm.st[x] = dec;
      const int left = __syncthreads_count(dec == kEsUndecided);
      if (left == 0) break;
      if (wave > (uint32_t)B) {  // every wave decides the smallest undecided switch: cannot happen
        if (x == 0) atomicOr(err, kErrNoProgress);
        return;
      }
    }
    // apply: rewire, then erase the sources before inserting the targets
    clear_touch(sm);  // the region becomes the next window's first-touch table (no table is read any more)
    const bool legal = dec == kEsLegal;
    if (legal) {
      jb.E[i] = e3;
      jb.E[j] = e4;
      const unsigned long long sk[2] = {e1, e2};
      const uint32_t shh[2] = {h1, h2};
      hset_erase2(jb.H, mask, sk, shh);
      atomicAdd(&s_tombs, 2u);
      ++acc;
    } else if (x < n && code == 0) {
      ++rej_exists;
    }
    __syncthreads();
    if (legal) {
      const unsigned long long tk[2] = {e3, e4};
      const uint32_t th[2] = {h3, h4};
      int r[2];
      hset_insert2(jb.H, mask, tk, th, r);
      if (r[0] < 0 || r[1] < 0) atomicOr(err, kErrTableFull);
      const uint32_t reused = (r[0] > 0 ? 1u : 0u) + (r[1] > 0 ? 1u : 0u);
      if (reused) atomicSub(&s_tombs, reused);
    }
    __syncthreads();
    if constexpr (kStopToRebuild) {
      s += n;
      if (s_tombs > (mask >> 3)) {  // a rebuild on the whole GPU is cheap: keep the probe chains short
        stop = s < jb.count;        // the same in every thread; a finished job needs no rebuild
        done = s;
        if (stop) break;
      }
    } else {
      if (s_tombs > (mask >> 2)) {  // rebuild the set from the list on this CTA
        for (uint32_t t = x; t <= mask; t += B) jb.H[t] = kEmptyKey;
        __syncthreads();
        for (uint32_t t = x; t < jb.m; t += B) {
          const unsigned long long e = __ldcg(&jb.E[t]);
          if (hset_insert(jb.H, mask, e, hash32(e)) < 0) atomicOr(err, kErrTableFull);
        }
        if (x == 0) s_tombs = 0;
        __syncthreads();
      }
      s += n;
    }
  }
  if constexpr (kStopToRebuild) {
    if (!stop) done = jb.count;
    if (x == 0) {  // progress of the job (the host launches it again while stopped)
      EsJob &out = jobs_out[job_off + blockIdx.x];
      out.k0 = jb.k0 + done;
      out.count = jb.count - done;
      out.stopped = stop ? 1u : 0u;
      if (stop) atomicAdd(nstop, 1u);
    }
  }
  // counts of this job
  const unsigned a32 = __reduce_add_sync(0xffffffffu, acc);
  const unsigned l32 = __reduce_add_sync(0xffffffffu, rej_loop);
  const unsigned r32 = __reduce_add_sync(0xffffffffu, rej_exists);
  if ((x & 31) == 0) {
    if (a32) {
      atomicAdd(&stats->accepted, (unsigned long long)a32);
      atomicAdd(&chain_acc[jb.chain], (unsigned long long)a32);
    }
    if (l32) atomicAdd(&stats->rej_loop, (unsigned long long)l32);
    if (r32) atomicAdd(&stats->rej_exists, (unsigned long long)r32);
  }
}

// Windows of 32, 128 and 256 switches (the set rebuilt in place).
template <int B, int MIN_BLOCKS>
__global__ void __launch_bounds__(B, MIN_BLOCKS) k_es_run(const EsJob *jobs, uint32_t job_off, StatsDev *stats,
                                                          unsigned long long *chain_acc, uint32_t *err) {
  es_run_body<B, false>(jobs, job_off, stats, chain_acc, err, nullptr, nullptr);
}

// Windows of 1024 switches (chains of at least 2^19 edges: the set rebuilt
// on the whole GPU between launches).
__global__ void __launch_bounds__(1024, 1) k_es_run_big(EsJob *jobs, uint32_t job_off, StatsDev *stats,
                                                        unsigned long long *chain_acc, uint32_t *err,
                                                        uint32_t *nstop) {
  es_run_body<1024, true>(jobs, job_off, stats, chain_acc, err, jobs, nstop);
}

}  // namespace

uint32_t es_window(uint32_t m) {
  return m >= kEsBigChain ? 1024u : m >= kEsMidChain ? 256u : m >= kEsSmallChain ? 128u : 32u;
}

cudaError_t prepare_es_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_es_run_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)EsShape<1024>::kBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_es_run<256, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)EsShape<256>::kBytes);
}

cudaError_t launch_es_set(const EsJob *jobs, uint32_t njobs, uint32_t *err, cudaStream_t s, int num_sms,
                          bool only_stopped) {
  for (uint32_t off = 0; off < njobs; off += 65535u) {
    const uint32_t nj = njobs - off < 65535u ? njobs - off : 65535u;
    const uint32_t gx = (uint32_t)((num_sms * 8 + nj - 1) / nj);
    const dim3 grid(gx < 1 ? 1 : gx, nj);
    k_es_clear<<<grid, 256, 0, s>>>(jobs, off, only_stopped);
    k_es_fill<<<grid, 256, 0, s>>>(jobs, off, err, only_stopped);
  }
  return cudaGetLastError();
}

cudaError_t launch_es_run(EsJob *jobs, const uint32_t (&group)[4], StatsDev *stats,
                          unsigned long long *chain_acc, uint32_t *err, uint32_t *nstop, cudaStream_t s,
                          cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join, uint32_t *launches) {
  // group[w] jobs with windows of 1024, 256, 128 and 32 switches, in that
  // order; the two small-window groups run on s2 (after s, and joined back
  // into s) when there is one, beside the others
  uint32_t beg[5] = {0, 0, 0, 0, 0};
  for (int w = 0; w < 4; ++w) beg[w + 1] = beg[w] + group[w];
  uint32_t n = 0;
  const bool side = s2 && fork && join && beg[2] > 0 && beg[4] > beg[2];
  cudaStream_t ss = side ? s2 : s;
  if (side && (cudaEventRecord(fork, s) != cudaSuccess || cudaStreamWaitEvent(s2, fork, 0) != cudaSuccess))
    return cudaGetLastError();
  auto run = [&](int w, cudaStream_t st) {
    for (uint32_t off = beg[w]; off < beg[w + 1]; off += 65535u, ++n) {
      const uint32_t nj = beg[w + 1] - off < 65535u ? beg[w + 1] - off : 65535u;
      if (w == 0) k_es_run_big<<<nj, 1024, EsShape<1024>::kBytes, st>>>(jobs, off, stats, chain_acc, err, nstop);
      else if (w == 1) k_es_run<256, 6><<<nj, 256, EsShape<256>::kBytes, st>>>(jobs, off, stats, chain_acc, err);
      else if (w == 2) k_es_run<128, 12><<<nj, 128, EsShape<128>::kBytes, st>>>(jobs, off, stats, chain_acc, err);
      else k_es_run<32, 32><<<nj, 32, EsShape<32>::kBytes, st>>>(jobs, off, stats, chain_acc, err);
    }
  };
  run(3, ss);
  run(2, ss);
  run(0, s);
  run(1, s);
  if (side && (cudaEventRecord(join, s2) != cudaSuccess || cudaStreamWaitEvent(s, join, 0) != cudaSuccess))
    return cudaGetLastError();
  if (launches) *launches = n;
  return cudaGetLastError();
}

}  // namespace gesmc
