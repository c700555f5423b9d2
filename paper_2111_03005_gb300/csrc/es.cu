// ParES (Algorithm 2 of arXiv 2111.03005): exact parallel ES-MC on one GB300.
//
// ES-MC runs independent edge switches sigma_k = (i, j, g) one after
// another (Def. 1's chain).  Algorithm 2 cuts the sequence into supersteps:
// maximal runs of consecutive switches of which no two share a source
// position, found with a first-touch table (each switch writes its index
// into the entries of its two positions with a minimum, and the first
// switch that finds a smaller index there starts the next superstep).  A
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
// launch.  A superstep is also cut at kEsBatch switches; any cut into
// consecutive runs without source dependencies gives the sequential result.
// When tombstones pass a quarter of the set's slots, the CTA rebuilds the set
// from the list between supersteps.
#include "device_util.cuh"
#include "gesmc_internal.cuh"

namespace gesmc {
namespace {

constexpr int kEsThreads = 1024;
constexpr int kEsBatch = kEsThreads;  // one switch per thread
constexpr int kEsSlots = 4096;        // shared-memory table slots (>= 2 x 2 x kEsBatch keys at load <= 1/2)
constexpr uint32_t kNil = 0xFFFFFFFFu;
constexpr uint32_t kNoTouch = 0xFFFFFFFFu;
constexpr uint8_t kEsUndecided = 0, kEsLegal = 1, kEsIllegal = 2;

// ---------------------------------------------------------------- the edge set H
__device__ __forceinline__ bool hset_contains(const unsigned long long *H, uint32_t mask, unsigned long long key) {
  uint32_t s = (uint32_t)mix64(key) & mask;
  for (uint32_t n = 0; n <= mask; ++n) {
    const unsigned long long cur = __ldcg(&H[s]);
    if (cur == key) return true;
    if (cur == kEmptyKey) return false;
    s = (s + 1) & mask;
  }
  return false;
}

__device__ __forceinline__ void hset_erase(unsigned long long *H, uint32_t mask, unsigned long long key) {
  uint32_t s = (uint32_t)mix64(key) & mask;
  for (uint32_t n = 0; n <= mask; ++n) {
    const unsigned long long cur = __ldcg(&H[s]);
    if (cur == key) {
      H[s] = kTombKey;
      return;
    }
    if (cur == kEmptyKey) return;
    s = (s + 1) & mask;
  }
}

// Insert a key that is not in the set into the first empty or tombstone
// slot of its probe sequence.  Returns 0 (empty slot taken), 1 (tombstone
// reused) or -1 (table full).
__device__ __forceinline__ int hset_insert(unsigned long long *H, uint32_t mask, unsigned long long key) {
  uint32_t s = (uint32_t)mix64(key) & mask;
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

// ---------------------------------------------------------------- shared-memory tables
// Sources of the superstep's switches (key -> switch) and its targets (key
// -> list of (switch, which) entries through next[]).
__device__ __forceinline__ uint32_t table_slot(unsigned long long *keys, unsigned long long key, bool claim) {
  uint32_t s = (uint32_t)mix64(key) & (kEsSlots - 1);
  for (int n = 0; n < kEsSlots; ++n) {
    const unsigned long long cur = keys[s];
    if (cur == key) return s;
    if (cur == kEmptyKey) {
      if (!claim) return kNil;
      const unsigned long long prev = atomicCAS(&keys[s], kEmptyKey, key);
      if (prev == kEmptyKey || prev == key) return s;
    }
    s = (s + 1) & (kEsSlots - 1);
  }
  return kNil;
}

struct EsSmem {
  uint32_t *si, *sj;
  unsigned long long *e1, *e2, *e3, *e4;
  unsigned long long *skey, *ikey;
  uint32_t *sval, *ihead, *tnext;
  uint8_t *code, *st, *nx, *pres, *gb;
};

__device__ __forceinline__ EsSmem es_smem() {
  extern __shared__ unsigned long long es_dyn[];
  EsSmem m;
  unsigned long long *p = es_dyn;
  m.e1 = p;
  m.e2 = p + kEsBatch;
  m.e3 = p + 2 * kEsBatch;
  m.e4 = p + 3 * kEsBatch;
  m.skey = p + 4 * kEsBatch;
  m.ikey = m.skey + kEsSlots;
  uint32_t *q = reinterpret_cast<uint32_t *>(m.ikey + kEsSlots);
  m.si = q;
  m.sj = q + kEsBatch;
  m.sval = q + 2 * kEsBatch;
  m.ihead = m.sval + kEsSlots;
  m.tnext = m.ihead + kEsSlots;
  uint8_t *b = reinterpret_cast<uint8_t *>(m.tnext + 2 * kEsBatch);
  m.code = b;
  m.st = b + kEsBatch;
  m.nx = b + 2 * kEsBatch;
  m.pres = b + 3 * kEsBatch;
  m.gb = b + 4 * kEsBatch;
  return m;
}

constexpr size_t kEsSmemBytes = 8ull * (4 * kEsBatch + 2 * kEsSlots) + 4ull * (2 * kEsBatch + 2 * kEsSlots + 2 * kEsBatch) +
                                5ull * kEsBatch;

// ---------------------------------------------------------------- kernels
// H <- empty, first <- untouched, for every job (blockIdx.y = job).
__global__ void k_es_clear(const EsJob *jobs, uint32_t job_off) {
  const EsJob jb = jobs[job_off + blockIdx.y];
  if (jb.m < 2) return;  // no list, no set
  const unsigned long long cap = 1ull << jb.hlog2;
  const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s < cap; s += nth)
    jb.H[s] = kEmptyKey;
  for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s < jb.m; s += nth)
    jb.first[s] = kNoTouch;
}

// H <- the entries of E.
__global__ void k_es_fill(const EsJob *jobs, uint32_t job_off, uint32_t *err) {
  const EsJob jb = jobs[job_off + blockIdx.y];
  if (jb.m < 2) return;
  const uint32_t mask = (uint32_t)((1ull << jb.hlog2) - 1);
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < jb.m; s += gridDim.x * blockDim.x)
    if (hset_insert(jb.H, mask, jb.E[s]) < 0) atomicOr(err, kErrTableFull);
}

// One CTA per job: switches k0 .. k0 + count - 1 of the job's chain.
__global__ void __launch_bounds__(kEsThreads) k_es_run(const EsJob *jobs, uint32_t job_off, StatsDev *stats,
                                                       unsigned long long *chain_acc, uint32_t *err) {
  const EsJob jb = jobs[job_off + blockIdx.x];
  const EsSmem sm = es_smem();
  __shared__ uint32_t s_cut, s_tombs;
  const uint32_t x = threadIdx.x;
  uint32_t acc = 0, rej_loop = 0, rej_exists = 0;
  if (jb.m < 2) {  // no pair of positions: every requested switch is skipped
    if (x == 0 && jb.count) atomicAdd(&stats->lazy, jb.count);
    return;
  }
  const uint32_t mask = (uint32_t)((1ull << jb.hlog2) - 1);
  if (x == 0) s_tombs = 0;  // the set was built from the list just before
  for (unsigned long long s = 0; s < jb.count;) {
    const uint32_t win = (uint32_t)min((unsigned long long)kEsBatch, jb.count - s);
    // sample the window and mark first touches (Algorithm 2's insert_if_min)
    if (x == 0) s_cut = win;
    if (x < win) {
      const U64x4 w = philox(jb.k0 + s + x, 0, 2, 0, jb.seed, 0);
      const uint32_t i = (uint32_t)__umul64hi(w.w[0], (unsigned long long)jb.m);
      const uint32_t jj = (uint32_t)__umul64hi(w.w[1], (unsigned long long)(jb.m - 1));
      const uint32_t j = jj + (jj >= i ? 1u : 0u);
      sm.si[x] = i;
      sm.sj[x] = j;
      sm.gb[x] = (uint8_t)(w.w[2] >> 63);
      atomicMin(&jb.first[i], x);
      atomicMin(&jb.first[j], x);
    }
    for (uint32_t t = x; t < kEsSlots; t += kEsThreads) {
      sm.skey[t] = kEmptyKey;
      sm.ikey[t] = kEmptyKey;
      sm.ihead[t] = kNil;
    }
    __syncthreads();
    // the superstep ends before the first switch that shares a position with an earlier one
    if (x < win && (__ldcg(&jb.first[sm.si[x]]) < x || __ldcg(&jb.first[sm.sj[x]]) < x)) atomicMin(&s_cut, x);
    __syncthreads();
    const uint32_t n = s_cut;
    if (x < win) {
      atomicExch(&jb.first[sm.si[x]], kNoTouch);  // at L2, like the minima of the next window
      atomicExch(&jb.first[sm.sj[x]], kNoTouch);
    }
    // sources, targets and the outright rules
    if (x < n) {
      const unsigned long long e1 = __ldcg(&jb.E[sm.si[x]]), e2 = __ldcg(&jb.E[sm.sj[x]]);
      unsigned long long e3, e4;
      const uint32_t code = tau_g(sm.gb[x], e1, e2, e3, e4);
      sm.e1[x] = e1;
      sm.e2[x] = e2;
      sm.e3[x] = e3;
      sm.e4[x] = e4;
      sm.code[x] = (uint8_t)code;
      sm.st[x] = code ? kEsIllegal : kEsUndecided;
      if (code == kCodeLoop) ++rej_loop;
      else if (code) ++rej_exists;  // shared node: the targets re-create the sources
    }
    __syncthreads();
    // erasers and inserters of the superstep; presence of the targets in E at its start
    if (x < n && sm.code[x] == 0) {
      uint32_t t = table_slot(sm.skey, sm.e1[x], true);
      if (t != kNil) sm.sval[t] = x;
      t = table_slot(sm.skey, sm.e2[x], true);
      if (t != kNil) sm.sval[t] = x;
      uint8_t pres = 0;
      for (uint32_t w = 0; w < 2; ++w) {
        const unsigned long long e = w ? sm.e4[x] : sm.e3[x];
        if (hset_contains(jb.H, mask, e)) pres |= (uint8_t)(1u << w);
        t = table_slot(sm.ikey, e, true);
        if (t != kNil) sm.tnext[2 * x + w] = atomicExch(&sm.ihead[t], 2 * x + w);
        else atomicOr(err, kErrTableFull);
      }
      sm.pres[x] = pres;
    }
    __syncthreads();
    // waves (Algorithm 1): a switch decided in wave w only uses decisions of earlier waves
    for (uint32_t wave = 1;; ++wave) {
      uint8_t dec = x < n ? sm.st[x] : kEsIllegal;
      if (x < n && dec == kEsUndecided) {
        bool bad = false, wait = false;
        for (uint32_t w = 0; w < 2 && !bad; ++w) {
          const unsigned long long e = w ? sm.e4[x] : sm.e3[x];
          if ((sm.pres[x] >> w) & 1u) {  // in E at the start: present unless an earlier legal switch erased it
            const uint32_t t = table_slot(sm.skey, e, false);
            const uint32_t p = t == kNil ? kNil : sm.sval[t];
            if (p == kNil || p >= x || sm.st[p] == kEsIllegal) bad = true;
            else if (sm.st[p] == kEsUndecided) wait = true;
          }
          if (bad) break;
          const uint32_t t = table_slot(sm.ikey, e, false);
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
      if (x < n) sm.nx[x] = dec;
      __syncthreads();
      if (x < n) sm.st[x] = sm.nx[x];
      const int left = __syncthreads_count(x < n && sm.st[x] == kEsUndecided);
      if (left == 0) break;
      if (wave > kEsBatch) {  // every wave decides the smallest undecided switch: cannot happen
        if (x == 0) atomicOr(err, kErrNoProgress);
        return;
      }
    }
    // apply: rewire, then erase the sources before inserting the targets
    const bool legal = x < n && sm.st[x] == kEsLegal;
    if (legal) {
      jb.E[sm.si[x]] = sm.e3[x];
      jb.E[sm.sj[x]] = sm.e4[x];
      hset_erase(jb.H, mask, sm.e1[x]);
      hset_erase(jb.H, mask, sm.e2[x]);
      atomicAdd(&s_tombs, 2u);
      ++acc;
    } else if (x < n && sm.code[x] == 0) {
      ++rej_exists;
    }
    __syncthreads();
    if (legal) {
      const int r3 = hset_insert(jb.H, mask, sm.e3[x]), r4 = hset_insert(jb.H, mask, sm.e4[x]);
      if (r3 < 0 || r4 < 0) atomicOr(err, kErrTableFull);
      const uint32_t reused = (r3 > 0 ? 1u : 0u) + (r4 > 0 ? 1u : 0u);
      if (reused) atomicSub(&s_tombs, reused);
    }
    __syncthreads();
    if (s_tombs > (mask >> 2)) {  // rebuild the set from the list
      for (uint32_t t = x; t <= mask; t += kEsThreads) jb.H[t] = kEmptyKey;
      __syncthreads();
      for (uint32_t t = x; t < jb.m; t += kEsThreads)
        if (hset_insert(jb.H, mask, __ldcg(&jb.E[t])) < 0) atomicOr(err, kErrTableFull);
      if (x == 0) s_tombs = 0;
      __syncthreads();
    }
    s += n;
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

}  // namespace

size_t es_smem_bytes() { return kEsSmemBytes; }

cudaError_t prepare_es_kernels() {
  return cudaFuncSetAttribute(k_es_run, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEsSmemBytes);
}

cudaError_t launch_es_set(const EsJob *jobs, uint32_t njobs, uint32_t *err, cudaStream_t s, int num_sms) {
  for (uint32_t off = 0; off < njobs; off += 65535u) {
    const uint32_t nj = njobs - off < 65535u ? njobs - off : 65535u;
    const uint32_t gx = (uint32_t)((num_sms * 8 + nj - 1) / nj);
    const dim3 grid(gx < 1 ? 1 : gx, nj);
    k_es_clear<<<grid, 256, 0, s>>>(jobs, off);
    k_es_fill<<<grid, 256, 0, s>>>(jobs, off, err);
  }
  return cudaGetLastError();
}

cudaError_t launch_es_run(const EsJob *jobs, uint32_t njobs, StatsDev *stats, unsigned long long *chain_acc,
                          uint32_t *err, cudaStream_t s) {
  for (uint32_t off = 0; off < njobs; off += 65535u) {
    const uint32_t nj = njobs - off < 65535u ? njobs - off : 65535u;
    k_es_run<<<nj, kEsThreads, kEsSmemBytes, s>>>(jobs, off, stats, chain_acc, err);
  }
  return cudaGetLastError();
}

}  // namespace gesmc
