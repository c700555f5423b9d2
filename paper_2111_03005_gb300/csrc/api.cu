// C ABI of libgesmc (declared in include/gesmc.h): pools of chains, the
// single-chain handle built on a one-chain pool, the allocation-free entry
// point, and the round loop of Algorithm 3 (ParGlobalES) of arXiv 2111.03005.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <iterator>
#include <map>
#include <mutex>
#include <numeric>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gesmc.h"
#include "gesmc_internal.cuh"
#include "resident.cuh"

using namespace gesmc;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Largest m: switch indices must fit the 30 bits a tuple gives them
// (pool-wide), so a pool's edges are bounded the same way.
constexpr uint64_t kMaxEdges = (1ull << 31) - 1;

// Shape of one chain in the index spaces.
struct ChainShape {
  uint32_t m, L, B, nb, P, np, capt;
  uint32_t slots() const { return (m + 1) & ~1u; }  // slot ranges start on even slots
  uint64_t tuples() const { return (uint64_t)np * capt; }
  uint32_t tstride() const { return P <= kSpreadLog2 ? kSpreadStride : 1u; }
  uint64_t tcounts() const { return (uint64_t)np * tstride(); }
};

bool chain_shape(uint64_t m, uint32_t tuple_log2, uint32_t bucket_log2, ChainShape *s) {
  if (m > kMaxEdges) return false;
  s->m = (uint32_t)m;
  s->L = (uint32_t)(m / 2);
  uint32_t B = 0;  // permutation buckets of about 2^(bucket_log2 - 1) positions
  while ((m >> B) > (1ull << (bucket_log2 - 1))) ++B;
  s->B = B;
  s->nb = 1u << B;
  const uint64_t ntuple = 4ull * s->L + 1;
  uint32_t P = 0;  // tuple partitions of about 2^tuple_log2 tuples
  while ((ntuple >> P) > (1ull << tuple_log2)) ++P;
  s->P = P;
  s->np = 1u << P;
  // room for the mean at four tuples per switch (the target filter lets
  // about 2.4 through) plus a margin; a partition that fills anyway spills
  // to the overflow list, which has room for every tuple
  s->capt = (uint32_t)((ntuple >> P) + 64);
  return true;
}

// Capacities of a pool's index spaces for at most M edges in at most C
// chains; each bound holds for any split of the edges into chains.
struct Capacity {
  uint64_t slots, switches, buckets, parts, tuples, ovf, dep, tcounts;
  uint32_t bucket_log2;  // room for 2^bucket_log2 records per permutation bucket
};

Capacity pool_capacity(uint64_t M, uint64_t C, uint32_t tuple_log2) {
  Capacity c;
  c.bucket_log2 = bucket_log2(M);
  ChainShape one;
  if (C == 1 && chain_shape(M, tuple_log2, c.bucket_log2, &one)) {
    // one chain: its own shape, which also covers any smaller chain (every
    // piece of a shape grows with m)
    c.slots = one.slots();
    c.switches = one.L + 1;
    c.buckets = one.nb;
    c.parts = one.np;
    c.tuples = one.tuples();
    c.ovf = 4ull * one.L + 1;
    c.dep = M + 1;
    c.tcounts = one.tcounts();
    return c;
  }
  c.slots = M + C;
  c.switches = M / 2 + C;
  c.buckets = 2 * (M >> (c.bucket_log2 - 1)) + 2 * C;
  const uint64_t ntuple = 2 * M + C;  // bounds the sum over chains of 4L + 1
  c.parts = 2 * (ntuple >> tuple_log2) + 4 * C;
  c.tuples = ntuple + 64 * c.parts;  // bounds the sum over chains of np * capt
  c.ovf = ntuple;
  c.dep = M + 1;
  c.tcounts = kSpreadStride * c.parts;  // bounds the sum over chains of np * stride
  return c;
}

// Every index space is addressed with 32-bit indices (chain ranges,
// partition cursors, tuple positions).
bool capacity_fits(const Capacity &c) {
  const uint64_t lim = 0xFFFFFFFFull;
  return c.slots < lim && c.switches < lim && c.buckets < lim && c.parts < lim && c.tuples < lim && c.ovf < lim &&
         c.dep < lim && c.tcounts < lim;
}

// Bits of the target filter for at most M edges: about four per edge (so
// that a source passes by a collision with probability about 1/5), a power
// of two between 2^12 and 2^28.  At most 32 MB: with 64 MB the filter's
// reductions missed L2 often enough that a round of G(2^24) took 0.6%
// longer, although fewer sources passed (a 16 MB filter let so many through
// that it took 17% longer).
uint64_t filter_bits(uint64_t M) {
  uint64_t b = 1ull << 12;
  while (b < 4 * M && b < (1ull << 28)) b <<= 1;
  return b;
}

// Offsets of the pieces of a pool's single device allocation.
struct Layout {
  size_t chains, chain_acc, chain_ell, es_jobs, es_job_of, tfilter, owner_slot, owner_switch, owner_bucket, owner_part, cpos, cedge, prec, pcount, poff, pblk,
      bnd, word, sw, status, list0, list1, ptup, otup, stup, tcount, ocount, ooff, oblk, ocursor, dep,
      E, ctl, st, scratch, total;
};

Layout pool_layout(const Capacity &c, uint64_t M, uint64_t C) {
  Layout l;
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o = align_up(o + (bytes ? bytes : 1));
    return at;
  };
  l.chains = take(sizeof(ChainDesc) * C);
  l.chain_acc = take(8 * C);
  l.chain_ell = take(4 * C);
  l.es_jobs = take(sizeof(EsJob) * C);
  l.es_job_of = take(4 * C);
  l.owner_slot = take(4 * c.slots);
  l.owner_switch = take(4 * c.switches);
  l.owner_bucket = take(4 * c.buckets);
  l.owner_part = take(4 * c.parts);
  l.cpos = take(4 * c.slots);
  l.cedge = take(8 * c.slots);
  // the permutation records are dead once the sort has read them, so the
  // overflow tuples sorted by partition (written after the sort, read by the
  // grouping) share their bytes; so does ParES's edge set, between rounds
  l.prec = take(std::max<uint64_t>((16ull << c.bucket_log2) * c.buckets, 16ull * c.ovf));
  l.stup = l.prec;
  l.pcount = take(4 * c.buckets);
  l.poff = take(4 * (c.buckets + 1));
  l.pblk = take(4 * (c.buckets / 1024 + 2));
  l.bnd = take(4 * (c.buckets + 1));
  l.word = take(4 * c.switches);
  l.sw = take(8 * c.switches);
  l.status = take(4 * c.switches);
  l.list0 = take(4 * c.switches);
  l.list1 = take(4 * c.switches);
  l.ptup = take(16 * c.tuples);
  l.otup = take(16 * c.ovf);
  l.tcount = take(4 * c.tcounts);
  l.ocount = take(4 * c.parts);
  l.ooff = take(4 * (c.parts + 1));
  l.oblk = take(4 * (c.parts / 1024 + 2));
  l.ocursor = take(4 * c.parts);
  l.dep = take(8 * c.dep);
  l.tfilter = take(filter_bits(M) / 8);
  l.E = take(8 * M);
  l.ctl = take(sizeof(Counters));
  l.st = take(sizeof(StatsDev));
  l.scratch = take(64);
  l.total = o;
  return l;
}

template <class T>
T *at(void *base, size_t off) {
  return reinterpret_cast<T *>(static_cast<char *>(base) + off);
}

// First-fit allocator of ranges of one index space.
class RangeSet {
 public:
  void reset(uint64_t capacity) {
    cap_ = capacity;
    free_.clear();
    if (capacity) free_[0] = capacity;
  }
  bool alloc(uint64_t len, uint64_t *start) {
    if (len == 0) {
      *start = 0;
      return true;
    }
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= len) {
        *start = it->first;
        const uint64_t rest = it->second - len, next = it->first + len;
        free_.erase(it);
        if (rest) free_[next] = rest;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t start, uint64_t len) {
    if (len == 0) return;
    auto it = free_.emplace(start, len).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  // Smallest index above every allocated range.
  uint64_t high_water() const {
    if (free_.empty()) return cap_;
    auto last = std::prev(free_.end());
    return last->first + last->second == cap_ ? last->first : cap_;
  }

 private:
  uint64_t cap_ = 0;
  std::map<uint64_t, uint64_t> free_;
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

struct HostChain {
  bool live = false;
  ChainDesc d;
  ChainShape shape;
  uint64_t n = 0;
  uint64_t es_next = 0;  // ES-MC switches run (numbering of the next one)
  unsigned long long fp = 0;  // degree fingerprint of the starting list (gesmc_verify)
};

// A chain the resident rounds take: few enough edges for one CTA's shared
// memory and node ids that fit 16 bits (chains with m < 2 have no rounds to run).
bool resident_fits(uint64_t m, uint64_t n) { return m < 2 || (m <= kResidentMaxEdges && n <= kResidentMaxNodes); }

int map_device_errors(uint32_t err) {
  if (err & kErrTableFull) return GESMC_E_TABLE_FULL;
  if (err & kErrWaveCap) return GESMC_E_WAVE_CAP;
  if (err & (kErrBucket | kErrNoProgress | kErrRecord | kErrGroup | kErrCopy | kErrGridSync)) return GESMC_E_INTERNAL;
  return GESMC_OK;
}

}  // namespace

// A pool: device state for up to max_chains chains with max_edges edges in
// total, and the host bookkeeping of its index spaces.
struct gesmc_pool_ctx {
  int device = 0;
  int num_sms = 1;
  cudaStream_t stream = nullptr;
  gesmc_alloc_fn alloc = nullptr;
  gesmc_free_fn free_fn = nullptr;
  void *alloc_ctx = nullptr;
  bool owns_memory = true;
  void *base = nullptr;
  uint64_t max_edges = 0;
  uint32_t max_chains = 0;
  uint32_t tuple_log2 = kDefaultTupleLog2;
  Capacity cap;
  Layout lay;
  RangeSet slots, switches, buckets, parts, tuples, tcounts;
  std::vector<HostChain> chains;
  uint32_t live_chains = 0, working_chains = 0;
  uint64_t live_edges = 0;
  uint64_t pool_round = 0;  // rounds completed (host copy of the device counter)
  uint64_t rounds = 0, switches_run = 0, launches = 0;
  int broken = 0;
  RoundArgs args;
  uint64_t args_version = 1;  // bumped whenever args change (invalidates the graph)
  uint32_t wave_kernels = 0;  // whole-GPU wave kernel pairs per round (grows with the waves seen)
  // captured round (CUDA graph), replayed on gstream
  bool use_graphs = true;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t gexec = nullptr;
  uint64_t graph_version = 0;
  uint32_t graph_launches = 0;
  // one-launch rounds (k_round_fused) with this many CTAs; 0: the kernels of
  // a round one after another (replayed from the captured graph)
  uint32_t fused_ctas = 0;
  uint32_t fused_max = 0;  // CTAs of the one-launch round the device holds at once
  // the one-launch round captured in a graph of its own (replayed per round),
  // for these args and CTA count; direct launches if capture is refused
  cudaGraphExec_t fused_exec = nullptr;
  uint64_t fused_version = 0;
  uint32_t fused_exec_ctas = 0;
  bool fused_graph_refused = false;
  // resident rounds (GESMC_ROUND_RESIDENT): one CTA per chain, the list in
  // shared memory for all rounds of a call; the chain list for the kernel
  // (in es_job_of) is rebuilt when the chains change (res_version)
  bool resident = false;
  uint64_t res_version = 0;
  uint32_t res_count[kResidentClasses] = {}, res_max_m[kResidentClasses] = {};  // chains and largest m per class
  bool verify_rounds = false;  // GESMC_FLAG_VERIFY_ROUNDS
  int profiling = 0;
  std::vector<cudaEvent_t> events;
  double stage_ms[kNumStages] = {};
  uint64_t stage_rounds = 0;
};

struct gesmc_ctx {
  gesmc_pool_t pool = nullptr;
  uint32_t chain = 0;
};

namespace {

void *dev_alloc(gesmc_pool_t p, size_t bytes) {
  if (p->alloc) return p->alloc(bytes, (void *)p->stream, p->alloc_ctx);
  void *ptr = nullptr;
  if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return ptr;
}

void dev_free(gesmc_pool_t p, void *ptr) {
  if (!ptr || !p->owns_memory) return;
  if (p->free_fn) p->free_fn(ptr, p->alloc_ctx);
  else cudaFree(ptr);
}

// A stride coprime with n near n times the golden ratio's fraction (1 if n
// is tiny): CTA b of a flat pass of n CTAs takes range (b * stride) mod n.
uint32_t coprime_stride(uint32_t n) {
  if (n <= 2) return 1;
  uint64_t s = (uint64_t)(n * 0.6180339887498949) | 1u;
  while (std::gcd<uint64_t, uint64_t>(s, n) != 1) s += 2;
  return (uint32_t)(s % n);
}

void refresh_args(gesmc_pool_t p) {
  ++p->args_version;
  RoundArgs &a = p->args;
  a.slot_hw = (uint32_t)p->slots.high_water();
  a.switch_hw = (uint32_t)p->switches.high_water();
  a.bucket_hw = (uint32_t)p->buckets.high_water();
  a.part_hw = (uint32_t)p->parts.high_water();
  a.tcount_hw = (uint32_t)p->tcounts.high_water();
  a.any_work = p->working_chains > 0;
  a.wave_kernels = p->wave_kernels;
  a.chain_hw = 0;
  a.any_exact = 0;
  for (uint32_t c = 0; c < p->max_chains; ++c) {
    const HostChain &hc = p->chains[c];
    if (!hc.live) continue;
    a.chain_hw = c + 1;
    if (hc.d.exact_ell && hc.d.lazy_threshold != 0 && hc.d.L > 0) a.any_exact = 1;
  }
  // flat pair passes: one pair per thread (k_permute), two (k_sources); a
  // pool of several chains spreads its resident CTAs over all of them
  const uint32_t npair = a.slot_hw / 2;
  a.permute_ctas = std::max<uint32_t>(1, (npair + 255) / 256);
  a.sources_ctas = std::max<uint32_t>(1, (npair + 511) / 512);
  const bool spread = p->live_chains > 1;
  uint32_t most_buckets = 0;
  for (const HostChain &hc : p->chains)
    if (hc.live) most_buckets = std::max(most_buckets, hc.shape.nb);
  a.fused_local_offsets = most_buckets <= kLocalOffsetBuckets ? 1u : 0u;
  a.permute_stride = spread ? coprime_stride(a.permute_ctas) : 1;
  a.sources_stride = spread ? coprime_stride(a.sources_ctas) : 1;
  a.agg_chain = kNoChain;
  a.agg_pairs = 0;
  if (p->live_chains == 1)
    for (uint32_t c = 0; c < p->max_chains; ++c)
      if (p->chains[c].live && p->chains[c].shape.m >= 2 && p->chains[c].shape.nb <= kAggBuckets) {
        a.agg_chain = c;
        a.agg_pairs = (p->chains[c].shape.m + 1) / 2;
      }
}

// Point the round arguments at the pieces of the pool's memory.
void pool_bind(gesmc_pool_t p) {
  void *b = p->base;
  const Layout &l = p->lay;
  RoundArgs &a = p->args;
  std::memset(&a, 0, sizeof(a));
  a.chains = at<ChainDesc>(b, l.chains);
  a.chain_accepted = at<unsigned long long>(b, l.chain_acc);
  a.chain_ell = at<uint32_t>(b, l.chain_ell);
  a.owner_slot = at<uint32_t>(b, l.owner_slot);
  a.owner_switch = at<uint32_t>(b, l.owner_switch);
  a.owner_bucket = at<uint32_t>(b, l.owner_bucket);
  a.owner_part = at<uint32_t>(b, l.owner_part);
  a.cpos = at<uint32_t>(b, l.cpos);
  a.cedge = at<unsigned long long>(b, l.cedge);
  a.prec = at<uint4>(b, l.prec);
  a.pcount = at<uint32_t>(b, l.pcount);
  a.poff = at<uint32_t>(b, l.poff);
  a.pblk = at<uint32_t>(b, l.pblk);
  a.bnd = at<uint32_t>(b, l.bnd);
  a.word = at<uint32_t>(b, l.word);
  a.tfilter = at<uint32_t>(b, l.tfilter);
  a.tfilter_mask = (uint32_t)(filter_bits(p->max_edges) - 1);
  a.sw = at<uint2>(b, l.sw);
  a.status = at<uint32_t>(b, l.status);
  a.list0 = at<uint32_t>(b, l.list0);
  a.list1 = at<uint32_t>(b, l.list1);
  a.ptup = at<uint4>(b, l.ptup);
  a.otup = at<uint4>(b, l.otup);
  a.stup = at<uint4>(b, l.stup);
  a.tcount = at<uint32_t>(b, l.tcount);
  a.ocount = at<uint32_t>(b, l.ocount);
  a.ooff = at<uint32_t>(b, l.ooff);
  a.oblk = at<uint32_t>(b, l.oblk);
  a.ocursor = at<uint32_t>(b, l.ocursor);
  a.dep = at<uint2>(b, l.dep);
  a.ctl = at<Counters>(b, l.ctl);
  a.st = at<StatsDev>(b, l.st);
  a.ovf_cap = (uint32_t)p->cap.ovf;
  a.dep_cap = (uint32_t)p->cap.dep;
  a.bucket_log2 = p->cap.bucket_log2;
}

bool valid_opts(const gesmc_pool_opts &o) {
  if (o.max_edges > kMaxEdges || o.max_chains == 0 || o.max_chains > (1u << 20)) return false;
  if (o.tuple_log2 && (o.tuple_log2 < 8 || o.tuple_log2 > 16)) return false;
  if (o.group_log2 && (o.group_log2 < 10 || o.group_log2 > (uint32_t)kMaxGroupLog2)) return false;
  if ((o.alloc == nullptr) != (o.free == nullptr)) return false;
  return true;
}

// Host state and device memory (owner maps, counters) of an empty pool whose
// memory is bound at p->base.
int pool_init(gesmc_pool_t p, const gesmc_pool_opts &o) {
  p->slots.reset(p->cap.slots);
  p->switches.reset(p->cap.switches);
  p->buckets.reset(p->cap.buckets);
  p->parts.reset(p->cap.parts);
  p->tuples.reset(p->cap.tuples);
  p->tcounts.reset(p->cap.tcounts);
  p->chains.assign(p->max_chains, HostChain());
  pool_bind(p);
  RoundArgs &a = p->args;
  if (o.flags & GESMC_FLAG_TINY_OVERFLOW) {
    a.ovf_cap = std::min<uint32_t>(a.ovf_cap, 16u);
    a.dep_cap = std::min<uint32_t>(a.dep_cap, 16u);
  }
  a.max_waves = o.max_waves;
  a.group_log2 = o.group_log2 ? o.group_log2 : kDefaultGroupLog2;
  LaunchShapes shapes;
  if (prepare_kernels(a.group_log2, p->num_sms, &shapes) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  a.group_grid = shapes.group;
  if (prepare_es_kernels() != cudaSuccess || prepare_resident() != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  if (prepare_fused(a.group_log2, p->num_sms, &p->fused_max) != cudaSuccess) {
    cudaGetLastError();  // the one-launch round is then unavailable; the multi-kernel round still works
    p->fused_max = 0;
  }
  cudaStream_t s = p->stream;
  const int sms = p->num_sms;
  bool ok = launch_fill_u32(const_cast<uint32_t *>(a.owner_slot), (uint32_t)p->cap.slots, kNoChain, s, sms) ==
            cudaSuccess;
  ok &= launch_fill_u32(const_cast<uint32_t *>(a.owner_switch), (uint32_t)p->cap.switches, kNoChain, s, sms) ==
        cudaSuccess;
  ok &= launch_fill_u32(const_cast<uint32_t *>(a.owner_bucket), (uint32_t)p->cap.buckets, kNoChain, s, sms) ==
        cudaSuccess;
  ok &= launch_fill_u32(const_cast<uint32_t *>(a.owner_part), (uint32_t)p->cap.parts, kNoChain, s, sms) ==
        cudaSuccess;
  ok &= cudaMemsetAsync(a.ctl, 0, sizeof(Counters), s) == cudaSuccess;
  ok &= cudaMemsetAsync(a.st, 0, sizeof(StatsDev), s) == cudaSuccess;
  ok &= cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  refresh_args(p);
  return GESMC_OK;
}

// Validate and canonicalise the list at E (device, m edges) in place: loops,
// ids >= n_bound, repeated edges, in that precedence.  *n_out receives
// n_bound, or largest id + 1 if n_bound is 0.  Synchronises the stream.
int validate_list(gesmc_pool_t p, unsigned long long *E, uint64_t m, uint64_t n_bound, uint64_t *n_out) {
  cudaStream_t s = p->stream;
  uint32_t *flags = at<uint32_t>(p->base, p->lay.scratch);
  uint32_t host_flags[2] = {0, 0};
  bool ok = cudaMemsetAsync(flags, 0, 8, s) == cudaSuccess;
  if (ok && m > 0) ok &= launch_canonicalise(E, (uint32_t)m, n_bound, flags, flags + 1, s, p->num_sms) == cudaSuccess;
  ok &= cudaMemcpyAsync(host_flags, flags, 8, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  ok &= cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  if (host_flags[0] & kFlagLoop) return GESMC_E_LOOP;
  if (host_flags[0] & kFlagRange) return GESMC_E_RANGE;
  *n_out = n_bound ? n_bound : (m ? (uint64_t)host_flags[1] + 1 : 0);
  if (m == 0) return GESMC_OK;
  // between rounds the overflow-tuple array is free: it holds the set
  ok &= launch_duplicate_check(E, (uint32_t)m, reinterpret_cast<unsigned long long *>(p->args.otup), 2 * p->cap.ovf,
                               flags, s, p->num_sms) == cudaSuccess;
  ok &= cudaMemcpyAsync(host_flags, flags, 4, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  ok &= cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  if (host_flags[0] & kFlagMulti) return GESMC_E_MULTI;
  if (host_flags[0] & kFlagTableFull) return GESMC_E_INTERNAL;
  return GESMC_OK;
}

// Debug check of a device list: invariant flags (loop / not canonical,
// range, repeated edge) and the degree fingerprint.  set: scratch of `cap`
// u64 slots (cap >= 2m); words: 4 device words of scratch.  Synchronises s.
int list_check(const unsigned long long *E, uint64_t m, uint64_t n, unsigned long long *set, uint64_t cap,
               uint32_t *words, cudaStream_t s, int num_sms, uint32_t *flags_out, unsigned long long *fp_out) {
  unsigned long long *fp = reinterpret_cast<unsigned long long *>(words + 2);
  uint32_t host[4] = {0, 0, 0, 0};
  bool ok = cudaMemsetAsync(words, 0, 16, s) == cudaSuccess;
  ok &= launch_list_check(E, (uint32_t)m, n, words, fp, s, num_sms) == cudaSuccess;
  if (m > 0 && set) ok &= launch_duplicate_check(E, (uint32_t)m, set, cap, words, s, num_sms) == cudaSuccess;
  ok &= cudaMemcpyAsync(host, words, 16, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  ok &= cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  *flags_out = host[0];
  std::memcpy(fp_out, host + 2, 8);
  return GESMC_OK;
}

// The chain's list by position (into the pool's staging buffer) against its
// invariants and its starting degree fingerprint.
int verify_chain(gesmc_pool_t p, uint32_t chain) {
  const HostChain &hc = p->chains[chain];
  const uint64_t m = hc.shape.m;
  unsigned long long *E = at<unsigned long long>(p->base, p->lay.E);
  uint32_t *words = at<uint32_t>(p->base, p->lay.scratch) + 4;
  if (m > 0 && launch_store_chain(p->args, hc.d, E, p->stream, p->num_sms) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  uint32_t flags = 0;
  unsigned long long fp = 0;
  // between rounds the overflow-tuple array is free: it holds the set
  const int rc = list_check(E, m, hc.n, reinterpret_cast<unsigned long long *>(p->args.otup), 2 * p->cap.ovf, words,
                            p->stream, p->num_sms, &flags, &fp);
  if (rc != GESMC_OK) return rc;
  return flags == 0 && fp == hc.fp ? GESMC_OK : GESMC_E_INVARIANT;
}

void release_ranges(gesmc_pool_t p, const HostChain &hc) {
  p->slots.release(hc.d.slot_base, hc.shape.slots());
  p->switches.release(hc.d.switch_base, hc.shape.L);
  p->buckets.release(hc.d.bucket_base, hc.shape.nb);
  p->parts.release(hc.d.part_base, hc.shape.np);
  p->tuples.release(hc.d.tuple_base, hc.shape.tuples());
  p->tcounts.release(hc.d.tcount_base, hc.shape.tcounts());
}

// Ranges for a chain of this shape, all or none.
bool alloc_ranges(gesmc_pool_t p, HostChain &hc) {
  uint64_t sb = 0, wb = 0, bb = 0, pb = 0, tb = 0;
  const ChainShape &sh = hc.shape;
  if (!p->slots.alloc(sh.slots(), &sb)) return false;
  if (!p->switches.alloc(sh.L, &wb)) {
    p->slots.release(sb, sh.slots());
    return false;
  }
  if (!p->buckets.alloc(sh.nb, &bb)) {
    p->slots.release(sb, sh.slots());
    p->switches.release(wb, sh.L);
    return false;
  }
  if (!p->parts.alloc(sh.np, &pb)) {
    p->slots.release(sb, sh.slots());
    p->switches.release(wb, sh.L);
    p->buckets.release(bb, sh.nb);
    return false;
  }
  if (!p->tuples.alloc(sh.tuples(), &tb)) {
    p->slots.release(sb, sh.slots());
    p->switches.release(wb, sh.L);
    p->buckets.release(bb, sh.nb);
    p->parts.release(pb, sh.np);
    return false;
  }
  uint64_t cb = 0;
  if (!p->tcounts.alloc(sh.tcounts(), &cb)) {
    p->slots.release(sb, sh.slots());
    p->switches.release(wb, sh.L);
    p->buckets.release(bb, sh.nb);
    p->parts.release(pb, sh.np);
    p->tuples.release(tb, sh.tuples());
    return false;
  }
  hc.d.slot_base = (uint32_t)sb;
  hc.d.switch_base = (uint32_t)wb;
  hc.d.bucket_base = (uint32_t)bb;
  hc.d.part_base = (uint32_t)pb;
  hc.d.tuple_base = (uint32_t)tb;
  hc.d.tcount_base = (uint32_t)cb;
  hc.d.tstride = sh.tstride();
  return true;
}

// Set the owner maps of a chain's ranges to `c` (kNoChain to remove it).
bool set_owners(gesmc_pool_t p, const HostChain &hc, uint32_t c) {
  RoundArgs &a = p->args;
  cudaStream_t s = p->stream;
  const int sms = p->num_sms;
  bool ok = launch_fill_u32(const_cast<uint32_t *>(a.owner_slot) + hc.d.slot_base, hc.shape.slots(), c, s, sms) ==
            cudaSuccess;
  ok &= launch_fill_u32(const_cast<uint32_t *>(a.owner_switch) + hc.d.switch_base, hc.shape.L, c, s, sms) ==
        cudaSuccess;
  ok &= launch_fill_u32(const_cast<uint32_t *>(a.owner_bucket) + hc.d.bucket_base, hc.shape.nb, c, s, sms) ==
        cudaSuccess;
  ok &= launch_fill_u32(const_cast<uint32_t *>(a.owner_part) + hc.d.part_base, hc.shape.np, c, s, sms) ==
        cudaSuccess;
  return ok;
}

// Add a chain whose list is already on the device at E (the pool's staging
// buffer, or the caller's buffer for the allocation-free path).
int pool_add_device(gesmc_pool_t p, unsigned long long *E, uint64_t m, uint64_t n, uint64_t seed,
                    uint64_t start_round, uint64_t lazy_threshold, uint32_t flags, uint32_t *chain_out) {
  if (flags & ~GESMC_CHAIN_EXACT_ELL) return GESMC_E_INVALID;
  if (m > p->max_edges - p->live_edges) return GESMC_E_NOMEM;
  uint32_t c = 0;
  while (c < p->max_chains && p->chains[c].live) ++c;
  if (c == p->max_chains) return GESMC_E_NOMEM;
  HostChain hc;
  std::memset(&hc.d, 0, sizeof(hc.d));
  if (!chain_shape(m, p->tuple_log2, p->cap.bucket_log2, &hc.shape)) return GESMC_E_INVALID;
  uint64_t n_eff = 0;
  int rc = validate_list(p, E, m, n, &n_eff);
  if (rc != GESMC_OK) return rc;
  if (p->resident && !resident_fits(m, n_eff)) return GESMC_E_TOO_LARGE;
  {  // the starting list's degree fingerprint (gesmc_verify compares against it)
    uint32_t flags = 0;
    rc = list_check(E, m, 0, nullptr, 0, at<uint32_t>(p->base, p->lay.scratch) + 4, p->stream, p->num_sms, &flags,
                    &hc.fp);
    if (rc != GESMC_OK) return rc;
  }
  if (!alloc_ranges(p, hc)) return GESMC_E_NOMEM;
  ChainDesc &d = hc.d;
  d.m = hc.shape.m;
  d.L = hc.shape.L;
  d.B = hc.shape.B;
  d.P = hc.shape.P;
  d.capt = hc.shape.capt;
  d.seed = seed;
  d.start_round = start_round;
  d.join = p->pool_round;
  d.added = p->pool_round;
  d.lazy_threshold = lazy_threshold;
  d.exact_ell = (flags & GESMC_CHAIN_EXACT_ELL) ? 1u : 0u;
  hc.live = true;
  hc.n = n_eff;
  cudaStream_t s = p->stream;
  RoundArgs &a = p->args;
  bool ok = cudaMemcpyAsync(const_cast<ChainDesc *>(a.chains) + c, &d, sizeof(d), cudaMemcpyHostToDevice, s) ==
            cudaSuccess;
  ok &= cudaMemsetAsync(a.chain_accepted + c, 0, 8, s) == cudaSuccess;
  ok &= set_owners(p, hc, c);
  ok &= launch_load_chain(a, d, E, s, p->num_sms) == cudaSuccess;
  ok &= cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    release_ranges(p, hc);
    return GESMC_E_CUDA;
  }
  p->chains[c] = hc;
  ++p->live_chains;
  if (m >= 2) ++p->working_chains;
  p->live_edges += m;
  refresh_args(p);
  *chain_out = c;
  return GESMC_OK;
}

int pool_run(gesmc_pool_t p, uint64_t rounds) {
  if (p->broken) return p->broken;
  DeviceGuard g(p->device);
  cudaStream_t s = p->stream;
  const RoundArgs a = p->args;
  if (cudaMemsetAsync(&a.ctl->err, 0, sizeof(uint32_t), s) != cudaSuccess) return GESMC_E_CUDA;
  const size_t per_round = kNumStages + 1;
  const bool stage_events = p->profiling && !p->resident;  // resident rounds have no separate stages
  if (stage_events) {
    const size_t need = per_round * (size_t)rounds;
    while (p->events.size() < need) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return GESMC_E_CUDA;
      }
      p->events.push_back(e);
    }
  }
  uint32_t launches = 0;
  if (p->resident) {
    // one CTA per chain with two edges or more, all rounds of the call in one
    // launch (several if the rounds outnumber the wave-count scratch words)
    if (p->res_version != p->args_version) {
      // chain ids grouped by class (CTA size), class 0 first
      std::vector<uint32_t> by_class[kResidentClasses];
      for (uint32_t k = 0; k < kResidentClasses; ++k) p->res_count[k] = p->res_max_m[k] = 0;
      for (uint32_t c = 0; c < p->max_chains; ++c) {
        const HostChain &hc = p->chains[c];
        if (!hc.live || hc.shape.m < 2) continue;
        const uint32_t k = resident_class(hc.shape.m);
        by_class[k].push_back(c);
        p->res_max_m[k] = std::max(p->res_max_m[k], hc.shape.m);
      }
      std::vector<uint32_t> jobs;
      for (uint32_t k = 0; k < kResidentClasses; ++k) {
        jobs.insert(jobs.end(), by_class[k].begin(), by_class[k].end());
        p->res_count[k] = (uint32_t)by_class[k].size();
      }
      if (!jobs.empty() && (cudaMemcpyAsync(at<uint32_t>(p->base, p->lay.es_job_of), jobs.data(), 4 * jobs.size(),
                                            cudaMemcpyHostToDevice, s) != cudaSuccess ||
                            cudaStreamSynchronize(s) != cudaSuccess)) {
        cudaGetLastError();
        return GESMC_E_CUDA;
      }
      p->res_version = p->args_version;
    }
    // the target filter's words (unused by resident rounds) collect each
    // round's wave count and the last round's undecided switches per wave
    uint32_t *scratch = a.tfilter;
    const uint64_t words = (a.tfilter_mask >> 5) + 1;
    uint64_t per_launch = std::min<uint64_t>(kResidentMaxRoundsPerLaunch, words - kWaveHist);
    // a pool of few chains has its permutations sorted ahead of the rounds
    // on other SMs, into the permutation records' bytes (unused by resident
    // rounds): rounds x chains permutations of pstride u16, then their l
    uint32_t njobs = 0, max_m = 0;
    for (uint32_t k = 0; k < kResidentClasses; ++k) {
      njobs += p->res_count[k];
      max_m = std::max(max_m, p->res_max_m[k]);
    }
    const uint32_t pstride = (max_m + 7u) & ~7u;
    const uint64_t pre_bytes = (16ull << p->cap.bucket_log2) * p->cap.buckets;
    const uint64_t per_round = (uint64_t)njobs * (2ull * pstride + 4);
    const bool presort = njobs > 0 && 4ull * njobs <= (uint64_t)p->num_sms && per_round <= pre_bytes;
    if (presort) per_launch = std::min<uint64_t>(per_launch, pre_bytes / per_round);
    for (uint64_t done = 0; done < rounds;) {
      const uint32_t r = (uint32_t)std::min<uint64_t>(per_launch, rounds - done);
      const bool final = done + r == rounds;
      nvtxRangePushA("gesmc resident rounds");
      bool ok = cudaMemsetAsync(scratch, 0, 4ull * (r + kWaveHist), s) == cudaSuccess;
      uint16_t *pbuf = presort ? reinterpret_cast<uint16_t *>(a.prec) : nullptr;
      uint32_t *ebuf = presort ? reinterpret_cast<uint32_t *>(pbuf + (uint64_t)r * njobs * pstride) : nullptr;
      ok = ok && launch_round_resident(a, at<uint32_t>(p->base, p->lay.es_job_of), p->res_count, p->res_max_m, r,
                                       scratch + kWaveHist, scratch, final, pbuf, ebuf, pstride, s,
                                       &launches) == cudaSuccess;
      nvtxRangePop();
      if (!ok) {
        cudaGetLastError();
        p->broken = GESMC_E_CUDA;
        return GESMC_E_CUDA;
      }
      done += r;
    }
  } else if (p->fused_ctas && !p->profiling) {
    // one cooperative launch per round, replayed from a captured graph when
    // the driver captures it (else launched directly)
    if (p->use_graphs && !p->fused_graph_refused &&
        (!p->fused_exec || p->fused_version != p->args_version || p->fused_exec_ctas != p->fused_ctas)) {
      if (p->fused_exec) cudaGraphExecDestroy(p->fused_exec);
      p->fused_exec = nullptr;
      cudaGraph_t graph = nullptr;
      bool ok = cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const bool launched = launch_round_fused(a, p->gstream, p->fused_ctas) == cudaSuccess;
        ok = cudaStreamEndCapture(p->gstream, &graph) == cudaSuccess && launched && graph;
      }
      ok = ok && cudaGraphInstantiate(&p->fused_exec, graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
      if (!ok) {
        cudaGetLastError();
        if (p->fused_exec) cudaGraphExecDestroy(p->fused_exec);
        p->fused_exec = nullptr;
        p->fused_graph_refused = true;
      } else {
        p->fused_version = p->args_version;
        p->fused_exec_ctas = p->fused_ctas;
      }
    }
    if (p->fused_exec && !p->fused_graph_refused) {
      bool ok = cudaEventRecord(p->ev_in, s) == cudaSuccess && cudaStreamWaitEvent(p->gstream, p->ev_in, 0) == cudaSuccess;
      for (uint64_t r = 0; r < rounds && ok; ++r) {
        nvtxRangePushA("gesmc round");
        ok = cudaGraphLaunch(p->fused_exec, p->gstream) == cudaSuccess;
        nvtxRangePop();
      }
      ok = ok && cudaEventRecord(p->ev_out, p->gstream) == cudaSuccess &&
           cudaStreamWaitEvent(s, p->ev_out, 0) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        p->broken = GESMC_E_CUDA;
        return GESMC_E_CUDA;
      }
      launches = (uint32_t)rounds;
    } else {
      for (uint64_t r = 0; r < rounds; ++r) {
        nvtxRangePushA("gesmc round");
        const cudaError_t e = launch_round_fused(a, s, p->fused_ctas);
        nvtxRangePop();
        if (e != cudaSuccess) {
          cudaGetLastError();
          p->broken = GESMC_E_CUDA;
          return GESMC_E_CUDA;
        }
        ++launches;
      }
    }
  } else if (p->use_graphs && !p->profiling && rounds > 0) {
    if (!p->gexec || p->graph_version != p->args_version) {
      if (p->gexec) cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
      cudaGraph_t graph = nullptr;
      uint32_t n = 0;
      bool ok = cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const bool launched = launch_round(a, p->gstream, p->num_sms, nullptr, &n) == cudaSuccess;
        ok = cudaStreamEndCapture(p->gstream, &graph) == cudaSuccess && launched;
      }
      ok = ok && cudaGraphInstantiate(&p->gexec, graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
      if (!ok) {
        cudaGetLastError();
        p->gexec = nullptr;
        p->broken = GESMC_E_CUDA;
        return GESMC_E_CUDA;
      }
      p->graph_version = p->args_version;
      p->graph_launches = n;
    }
    bool ok = cudaEventRecord(p->ev_in, s) == cudaSuccess && cudaStreamWaitEvent(p->gstream, p->ev_in, 0) == cudaSuccess;
    for (uint64_t r = 0; r < rounds && ok; ++r) {
      nvtxRangePushA("gesmc round");
      ok = cudaGraphLaunch(p->gexec, p->gstream) == cudaSuccess;
      nvtxRangePop();
    }
    ok = ok && cudaEventRecord(p->ev_out, p->gstream) == cudaSuccess &&
         cudaStreamWaitEvent(s, p->ev_out, 0) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      p->broken = GESMC_E_CUDA;
      return GESMC_E_CUDA;
    }
    launches = (uint32_t)(rounds * p->graph_launches);
  } else {
    for (uint64_t r = 0; r < rounds; ++r) {
      cudaEvent_t *ev = p->profiling ? &p->events[per_round * r] : nullptr;
      nvtxRangePushA("gesmc round");
      const cudaError_t e = launch_round(a, s, p->num_sms, ev, &launches);
      nvtxRangePop();
      if (e != cudaSuccess) {
        p->broken = GESMC_E_CUDA;
        return GESMC_E_CUDA;
      }
    }
  }
  Counters ctl;
  if (cudaMemcpyAsync(&ctl, a.ctl, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    p->broken = GESMC_E_CUDA;
    return GESMC_E_CUDA;
  }
  if (stage_events) {
    for (uint64_t r = 0; r < rounds; ++r)
      for (int st = 0; st < kNumStages; ++st) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->events[per_round * r + st], p->events[per_round * r + st + 1]) ==
            cudaSuccess)
          p->stage_ms[st] += ms;
      }
    p->stage_rounds += rounds;
  }
  p->pool_round += rounds;
  p->rounds += rounds;
  p->launches += launches;
  uint64_t sw = 0;
  for (const HostChain &hc : p->chains)
    if (hc.live) sw += hc.shape.L;
  p->switches_run += rounds * sw;
  const int rc = map_device_errors(ctl.err);
  if (rc != GESMC_OK) p->broken = rc;
  // rounds that needed more than one wave: run that many on the whole GPU from now on
  const uint32_t want = ctl.waves > 1 ? std::min<uint32_t>(ctl.waves - 1, kMaxWaveKernels) : 0u;
  if (rc == GESMC_OK && want > p->wave_kernels) {
    p->wave_kernels = want;
    refresh_args(p);
  }
  return rc;
}

// ParES (Algorithm 2) on the live chains of the pool (all of them, or only
// `only`): each runs `switches` ES-MC switches with its own seed, numbered
// on from its last ES-MC switch.  Each chain's list leaves its slots for
// its tuple storage (position order); its edge set lives in its
// permutation records (the ParES kernel rebuilds the set when tombstones
// pass a quarter of its slots).
int pool_es_run(gesmc_pool_t p, uint64_t switches, uint32_t only) {
  if (p->broken) return p->broken;
  if (switches == 0) return GESMC_OK;
  DeviceGuard g(p->device);
  cudaStream_t s = p->stream;
  const RoundArgs &a = p->args;
  std::vector<EsJob> jobs;
  std::vector<uint32_t> job_of(p->max_chains, kNoChain);
  char *tup = reinterpret_cast<char *>(a.ptup);
  for (uint32_t c = 0; c < p->max_chains; ++c) {
    const HostChain &hc = p->chains[c];
    if (!hc.live || (only != kNoChain && c != only)) continue;
    EsJob jb;
    std::memset(&jb, 0, sizeof(jb));
    jb.m = hc.d.m;
    jb.seed = hc.d.seed;
    jb.k0 = hc.es_next;
    jb.count = switches;
    jb.chain = c;
    if (jb.m >= 2) {
      // the list (position order) in the chain's tuple storage (at least 32
      // bytes per edge), the edge set in its permutation records (at least
      // 32 bytes per edge: 2^h >= 2m slots)
      char *base = tup + 16ull * hc.d.tuple_base;
      const uint64_t bytes = 16ull * hc.d.capt << hc.d.P;
      if (8ull * jb.m > bytes) return GESMC_E_INTERNAL;
      char *hbase = reinterpret_cast<char *>(a.prec) + (16ull << p->cap.bucket_log2) * hc.d.bucket_base;
      const uint64_t hbytes = (16ull << p->cap.bucket_log2) * hc.shape.nb;
      uint32_t hlog2 = 0;
      while ((16ull << hlog2) <= hbytes && hlog2 < 31) ++hlog2;  // largest 2^h with 8 * 2^h <= room
      if ((1ull << hlog2) < 2ull * jb.m) return GESMC_E_INTERNAL;
      jb.E = reinterpret_cast<unsigned long long *>(base);
      jb.H = reinterpret_cast<unsigned long long *>(hbase);
      jb.hlog2 = hlog2;
    }
    jobs.push_back(jb);
  }
  if (jobs.empty()) return GESMC_OK;
  // chains by window size, largest windows first (each group keeps chain
  // order); chains with m < 2 have no list to move (their switches are only
  // counted)
  std::stable_sort(jobs.begin(), jobs.end(),
                   [](const EsJob &x, const EsJob &y) { return es_window(x.m) > es_window(y.m); });
  uint32_t group[4] = {0, 0, 0, 0};
  for (uint32_t t = 0; t < jobs.size(); ++t) {
    if (jobs[t].m >= 2) job_of[jobs[t].chain] = t;
    const uint32_t w = es_window(jobs[t].m);
    ++group[w == 1024u ? 0 : w == 256u ? 1 : w == 128u ? 2 : 3];
  }
  EsJob *djobs = at<EsJob>(p->base, p->lay.es_jobs);
  uint32_t *djob_of = at<uint32_t>(p->base, p->lay.es_job_of);
  uint32_t *err = &a.ctl->err;
  const uint32_t nj = (uint32_t)jobs.size();
  bool ok = cudaMemsetAsync(err, 0, sizeof(uint32_t), s) == cudaSuccess;
  ok &= cudaMemcpyAsync(djob_of, job_of.data(), 4ull * p->max_chains, cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaMemcpyAsync(djobs, jobs.data(), sizeof(EsJob) * nj, cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= launch_es_store(a, djobs, djob_of, s, p->num_sms) == cudaSuccess;
  const uint64_t set_launches = 2ull * ((nj + 65534) / 65535);
  ok &= launch_es_set(djobs, nj, err, s, p->num_sms, false) == cudaSuccess;
  p->launches += set_launches + 2;
  // chains of the largest window stop when their edge set needs a rebuild;
  // rebuild those sets on the whole GPU and launch them again until every
  // job is done (each launch advances every stopped job by a superstep at
  // least)
  uint32_t *nstop = &a.ctl->es_stopped;
  for (uint64_t iter = 0; ok; ++iter) {
    uint32_t run_launches = 0;
    const uint32_t groups[4] = {group[0], iter ? 0u : group[1], iter ? 0u : group[2], iter ? 0u : group[3]};
    if (group[0]) ok &= cudaMemsetAsync(nstop, 0, sizeof(uint32_t), s) == cudaSuccess;
    ok &= launch_es_run(djobs, groups, a.st, a.chain_accepted, err, nstop, s, p->gstream, p->ev_in, p->ev_out,
                        &run_launches) == cudaSuccess;
    p->launches += run_launches;
    if (!ok || group[0] == 0) break;  // only the largest windows stop
    uint32_t stopped = 0, e = 0;
    ok &= cudaMemcpyAsync(&stopped, nstop, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok &= cudaMemcpyAsync(&e, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok &= cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok || stopped == 0 || e != 0) break;
    ok &= launch_es_set(djobs, nj, err, s, p->num_sms, true) == cudaSuccess;
    p->launches += set_launches;
  }
  ok &= launch_es_load(a, djobs, djob_of, s, p->num_sms) == cudaSuccess;
  uint32_t host_err = 0;
  ok &= cudaMemcpyAsync(&host_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) == cudaSuccess;
  ok &= cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    p->broken = GESMC_E_CUDA;
    return GESMC_E_CUDA;
  }
  for (uint32_t t = 0; t < nj; ++t) p->chains[jobs[t].chain].es_next += switches;
  p->switches_run += switches * nj;
  const int rc = map_device_errors(host_err);
  if (rc != GESMC_OK) p->broken = rc;
  return rc;
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------- pools

void gesmc_pool_opts_default(gesmc_pool_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_chains = 1;
}

size_t gesmc_pool_device_bytes(uint64_t max_edges, uint32_t max_chains, uint32_t tuple_log2) {
  if (max_edges > kMaxEdges || max_chains == 0) return 0;
  if (!tuple_log2) tuple_log2 = kDefaultTupleLog2;
  const Capacity c = pool_capacity(max_edges, max_chains, tuple_log2);
  return capacity_fits(c) ? pool_layout(c, max_edges, max_chains).total : 0;
}

void gesmc_pool_destroy(gesmc_pool_t p) {
  if (!p) return;
  {
    DeviceGuard g(p->device);
    if (p->base) {
      cudaStreamSynchronize(p->stream);
      if (p->gstream) cudaStreamSynchronize(p->gstream);
      dev_free(p, p->base);
    }
    for (cudaEvent_t e : p->events) cudaEventDestroy(e);
    if (p->fused_exec) cudaGraphExecDestroy(p->fused_exec);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    if (p->gstream) cudaStreamDestroy(p->gstream);
  }
  delete p;
}

int gesmc_pool_create(const gesmc_pool_opts *opts, gesmc_pool_t *out) {
  if (!out || !opts) return GESMC_E_INVALID;
  *out = nullptr;
  const gesmc_pool_opts o = *opts;
  if (!valid_opts(o)) return GESMC_E_INVALID;
  gesmc_pool_t p = new (std::nothrow) gesmc_pool_ctx();
  if (!p) return GESMC_E_NOMEM;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return GESMC_E_CUDA;
  }
  cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
  if (p->num_sms < 1) p->num_sms = 1;
  p->stream = (cudaStream_t)o.stream;
  p->alloc = o.alloc;
  p->free_fn = o.free;
  p->alloc_ctx = o.alloc_ctx;
  p->max_edges = o.max_edges;
  p->max_chains = o.max_chains;
  p->tuple_log2 = o.tuple_log2 ? o.tuple_log2 : kDefaultTupleLog2;
  p->use_graphs = !(o.flags & GESMC_FLAG_NO_GRAPHS);
  p->verify_rounds = (o.flags & GESMC_FLAG_VERIFY_ROUNDS) != 0;
  p->cap = pool_capacity(p->max_edges, p->max_chains, p->tuple_log2);
  if (!capacity_fits(p->cap)) {
    delete p;
    return GESMC_E_INVALID;
  }
  p->lay = pool_layout(p->cap, p->max_edges, p->max_chains);
  if (p->use_graphs &&
      (cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking) != cudaSuccess ||
       cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
       cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    gesmc_pool_destroy(p);
    return GESMC_E_CUDA;
  }
  p->base = dev_alloc(p, p->lay.total);
  if (!p->base) {
    gesmc_pool_destroy(p);
    return GESMC_E_NOMEM;
  }
  const int rc = pool_init(p, o);
  if (rc != GESMC_OK) {
    gesmc_pool_destroy(p);
    return rc;
  }
  *out = p;
  return GESMC_OK;
}

int gesmc_pool_add(gesmc_pool_t p, const uint64_t *edges, uint64_t m, int edges_on_device, uint64_t n,
                   uint64_t seed, uint64_t start_round, uint64_t lazy_threshold, uint32_t flags,
                   uint32_t *chain_out) {
  if (!p || !chain_out || (m > 0 && !edges) || m > kMaxEdges || n > (1ull << 32)) return GESMC_E_INVALID;
  if (p->broken) return p->broken;
  if (m > p->max_edges - p->live_edges) return GESMC_E_NOMEM;
  DeviceGuard g(p->device);
  unsigned long long *E = at<unsigned long long>(p->base, p->lay.E);
  if (m > 0 && cudaMemcpyAsync(E, edges, 8 * m, edges_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               p->stream) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  return pool_add_device(p, E, m, n, seed, start_round, lazy_threshold, flags, chain_out);
}

int gesmc_pool_remove(gesmc_pool_t p, uint32_t chain) {
  if (!p || chain >= p->max_chains || !p->chains[chain].live) return GESMC_E_INVALID;
  DeviceGuard g(p->device);
  HostChain &hc = p->chains[chain];
  bool ok = set_owners(p, hc, kNoChain);
  ok &= cudaStreamSynchronize(p->stream) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  release_ranges(p, hc);
  --p->live_chains;
  if (hc.shape.m >= 2) --p->working_chains;
  p->live_edges -= hc.shape.m;
  hc.live = false;
  refresh_args(p);
  return GESMC_OK;
}

int gesmc_pool_run(gesmc_pool_t p, uint64_t global_switches) {
  if (!p) return GESMC_E_INVALID;
  if (!p->verify_rounds) return pool_run(p, global_switches);
  // debugging: one round at a time, every chain checked after each
  DeviceGuard g(p->device);
  for (uint64_t r = 0; r < global_switches; ++r) {
    int rc = pool_run(p, 1);
    for (uint32_t c = 0; rc == GESMC_OK && c < p->max_chains; ++c)
      if (p->chains[c].live) rc = verify_chain(p, c);
    if (rc != GESMC_OK) {
      if (!p->broken) p->broken = rc;
      return rc;
    }
  }
  return GESMC_OK;
}

int gesmc_pool_verify(gesmc_pool_t p, uint32_t chain) {
  if (!p || chain >= p->max_chains || !p->chains[chain].live) return GESMC_E_INVALID;
  DeviceGuard g(p->device);
  return verify_chain(p, chain);
}

int gesmc_verify_list(const uint64_t *edges, uint64_t m, const uint64_t *reference, uint64_t ref_m, uint64_t n) {
  if ((m && !edges) || (ref_m && !reference) || m > kMaxEdges || ref_m > kMaxEdges) return GESMC_E_INVALID;
  if (m != ref_m) return GESMC_E_INVARIANT;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t cap = 2 * m + 16;
  void *scratch = nullptr;
  if (cudaMalloc(&scratch, 8 * cap + 64) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_NOMEM;
  }
  uint32_t *words = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + 8 * cap);
  uint32_t fa = 0, fb = 0;
  unsigned long long pa = 0, pb = 0;
  int rc = list_check(reinterpret_cast<const unsigned long long *>(edges), m, n,
                      static_cast<unsigned long long *>(scratch), cap, words, nullptr, sms, &fa, &pa);
  if (rc == GESMC_OK)
    rc = list_check(reinterpret_cast<const unsigned long long *>(reference), ref_m, 0, nullptr, 0, words, nullptr, sms,
                    &fb, &pb);
  cudaFree(scratch);
  if (rc != GESMC_OK) return rc;
  return fa == 0 && pa == pb ? GESMC_OK : GESMC_E_INVARIANT;
}

int gesmc_pool_set_round_launch(gesmc_pool_t p, uint32_t ctas, uint32_t *effective) {
  if (!p) return GESMC_E_INVALID;
  if (ctas == GESMC_ROUND_RESIDENT) {
    for (const HostChain &hc : p->chains)
      if (hc.live && !resident_fits(hc.shape.m, hc.n)) return GESMC_E_TOO_LARGE;
    p->resident = true;
    p->res_version = 0;
    if (effective) *effective = GESMC_ROUND_RESIDENT;
    return GESMC_OK;
  }
  p->resident = false;
  if (ctas && p->fused_max == 0) return GESMC_E_INVALID;
  const uint32_t want = std::min(ctas, p->fused_max);
  if (want != p->fused_ctas) {
    // the grid barrier's count restarts with the new CTA count
    DeviceGuard g(p->device);
    if (cudaMemsetAsync(&p->args.ctl->gbar_arrived, 0, sizeof(unsigned long long), p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess) {
      cudaGetLastError();
      return GESMC_E_CUDA;
    }
  }
  p->fused_ctas = want;
  if (effective) *effective = p->fused_ctas;
  return GESMC_OK;
}

int gesmc_pool_edges(gesmc_pool_t p, uint32_t chain, uint64_t *out, uint64_t capacity, int out_on_device,
                     uint64_t *m_out) {
  if (!p || chain >= p->max_chains || !p->chains[chain].live) return GESMC_E_INVALID;
  const uint64_t m = p->chains[chain].shape.m;
  if (m_out) *m_out = m;
  if (capacity < m) return GESMC_E_CAPACITY;
  if (m == 0) return GESMC_OK;
  if (!out) return GESMC_E_INVALID;
  DeviceGuard g(p->device);
  // the list is kept in the last round's slot order: write it by position
  unsigned long long *E = out_on_device ? reinterpret_cast<unsigned long long *>(out)
                                        : at<unsigned long long>(p->base, p->lay.E);
  bool ok = launch_store_chain(p->args, p->chains[chain].d, E, p->stream, p->num_sms) == cudaSuccess;
  if (ok && !out_on_device) ok = cudaMemcpyAsync(out, E, 8 * m, cudaMemcpyDeviceToHost, p->stream) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(p->stream) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  return GESMC_OK;
}

int gesmc_pool_chain_info(gesmc_pool_t p, uint32_t chain, gesmc_chain_info_t *out) {
  if (!p || !out || chain >= p->max_chains || !p->chains[chain].live) return GESMC_E_INVALID;
  DeviceGuard g(p->device);
  const HostChain &hc = p->chains[chain];
  unsigned long long acc = 0;
  if (cudaMemcpyAsync(&acc, p->args.chain_accepted + chain, 8, cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  std::memset(out, 0, sizeof(*out));
  out->m = hc.shape.m;
  out->n = hc.n;
  out->seed = hc.d.seed;
  out->rounds = p->pool_round - hc.d.added;
  out->next_round = hc.d.start_round + (p->pool_round - hc.d.join);
  out->switches = out->rounds * hc.shape.L;
  out->accepted = acc;
  out->es_switches = hc.es_next;
  return GESMC_OK;
}

int gesmc_pool_es_run(gesmc_pool_t p, uint64_t switches) {
  return p ? pool_es_run(p, switches, kNoChain) : GESMC_E_INVALID;
}

uint32_t gesmc_pool_num_chains(gesmc_pool_t p) { return p ? p->live_chains : 0; }

uint64_t gesmc_pool_free_edges(gesmc_pool_t p) { return p ? p->max_edges - p->live_edges : 0; }

int gesmc_pool_stats(gesmc_pool_t p, gesmc_stats_t *out) {
  if (!p || !out) return GESMC_E_INVALID;
  DeviceGuard g(p->device);
  StatsDev st;
  if (cudaMemcpyAsync(&st, p->args.st, sizeof(StatsDev), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  std::memset(out, 0, sizeof(*out));
  out->rounds = p->rounds;
  out->switches = p->switches_run;
  out->lazy = st.lazy;
  out->accepted = st.accepted;
  out->rejected_loop = st.rej_loop;
  out->rejected_exists = st.rej_exists;
  out->kernel_launches = p->launches;
  out->perm_buckets = p->args.bucket_hw;
  out->tuple_partitions = p->args.part_hw;
  out->waves_total = st.waves_total;
  out->waves_max = st.waves_max;
  for (int w = 0; w < GESMC_WAVE_HIST && w < kWaveHist; ++w) {
    out->wave_hist[w] = st.wave_hist[w];
    out->last_round_pending[w] = st.last_pending[w];
  }
  out->overflow_tuples = st.overflow_tuples;
  out->subpass_partitions = st.subpass_partitions;
  return GESMC_OK;
}

int gesmc_pool_reset_stats(gesmc_pool_t p) {
  if (!p) return GESMC_E_INVALID;
  DeviceGuard g(p->device);
  if (cudaMemsetAsync(p->args.st, 0, sizeof(StatsDev), p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  p->rounds = 0;
  p->switches_run = 0;
  p->launches = 0;
  for (double &x : p->stage_ms) x = 0.0;
  p->stage_rounds = 0;
  return GESMC_OK;
}

int gesmc_pool_set_profiling(gesmc_pool_t p, int enable) {
  if (!p) return GESMC_E_INVALID;
  p->profiling = enable ? 1 : 0;
  return GESMC_OK;
}

int gesmc_pool_stage_times(gesmc_pool_t p, double *ms, int n_stages, uint64_t *rounds) {
  if (!p || (n_stages > 0 && !ms)) return GESMC_E_INVALID;
  for (int st = 0; st < n_stages; ++st) ms[st] = st < kNumStages ? p->stage_ms[st] : 0.0;
  if (rounds) *rounds = p->stage_rounds;
  return GESMC_OK;
}

// ---------------------------------------------------------------- single chain

void gesmc_opts_default(gesmc_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
}

size_t gesmc_device_bytes(uint64_t m) { return gesmc_pool_device_bytes(m, 1, 0); }

const char *gesmc_strerror(int code) {
  switch (code) {
    case GESMC_OK: return "ok";
    case GESMC_E_INVALID: return "invalid argument";
    case GESMC_E_LOOP: return "edge list contains a loop";
    case GESMC_E_MULTI: return "edge list contains a repeated edge";
    case GESMC_E_RANGE: return "node id out of range";
    case GESMC_E_NOMEM: return "device allocation failed, or the pool has no room";
    case GESMC_E_CUDA: return "CUDA runtime error";
    case GESMC_E_TABLE_FULL: return "dependency table full";
    case GESMC_E_WAVE_CAP: return "wave cap exceeded";
    case GESMC_E_INTERNAL: return "internal error (bucket overflow or stalled waves)";
    case GESMC_E_CAPACITY: return "output buffer too small";
    case GESMC_E_TOO_LARGE:
      return "edge list too large: above GESMC_NOALLOC_MAX_EDGES (no-alloc call), or above "
             "GESMC_RESIDENT_MAX_EDGES edges / GESMC_RESIDENT_MAX_NODES nodes (resident rounds)";
    case GESMC_E_INVARIANT: return "the list is not a simple graph with the starting degree sequence";
    default: return "unknown error";
  }
}

void gesmc_destroy(gesmc_t h) {
  if (!h) return;
  gesmc_pool_destroy(h->pool);
  delete h;
}

int gesmc_create(const uint64_t *edges, uint64_t m, int edges_on_device, const gesmc_opts *opts, gesmc_t *out) {
  if (!out) return GESMC_E_INVALID;
  *out = nullptr;
  gesmc_opts o;
  gesmc_opts_default(&o);
  if (opts) o = *opts;
  if (m > kMaxEdges || (m > 0 && !edges) || o.n > (1ull << 32)) return GESMC_E_INVALID;
  gesmc_pool_opts po;
  gesmc_pool_opts_default(&po);
  po.max_edges = m;
  po.max_chains = 1;
  po.max_waves = o.max_waves;
  po.tuple_log2 = o.tuple_log2;
  po.group_log2 = o.group_log2;
  po.flags = o.flags & (GESMC_FLAG_NO_GRAPHS | GESMC_FLAG_TINY_OVERFLOW | GESMC_FLAG_VERIFY_ROUNDS);
  po.stream = o.stream;
  po.alloc = o.alloc;
  po.free = o.free;
  po.alloc_ctx = o.alloc_ctx;
  gesmc_ctx *h = new (std::nothrow) gesmc_ctx();
  if (!h) return GESMC_E_NOMEM;
  int rc = gesmc_pool_create(&po, &h->pool);
  // the seed is given to gesmc_run; the chain starts with seed 0
  if (rc == GESMC_OK)
    rc = gesmc_pool_add(h->pool, edges, m, edges_on_device, o.n, 0, o.start_round, o.lazy_threshold,
                        (o.flags & GESMC_FLAG_EXACT_ELL) ? GESMC_CHAIN_EXACT_ELL : 0u, &h->chain);
  if (rc != GESMC_OK) {
    gesmc_destroy(h);
    return rc;
  }
  *out = h;
  return GESMC_OK;
}

int gesmc_run(gesmc_t h, uint64_t global_switches, uint64_t seed) {
  if (!h) return GESMC_E_INVALID;
  gesmc_pool_t p = h->pool;
  if (p->broken) return p->broken;
  HostChain &hc = p->chains[h->chain];
  if (seed != hc.d.seed) {
    // a new seed continues the chain's round numbering
    DeviceGuard g(p->device);
    hc.d.start_round += p->pool_round - hc.d.join;
    hc.d.join = p->pool_round;
    hc.d.seed = seed;
    if (cudaMemcpyAsync(const_cast<ChainDesc *>(p->args.chains) + h->chain, &hc.d, sizeof(ChainDesc),
                        cudaMemcpyHostToDevice, p->stream) != cudaSuccess) {
      cudaGetLastError();
      return GESMC_E_CUDA;
    }
  }
  return gesmc_pool_run(p, global_switches);
}

int gesmc_es_run(gesmc_t h, uint64_t switches, uint64_t seed) {
  if (!h) return GESMC_E_INVALID;
  gesmc_pool_t p = h->pool;
  if (p->broken) return p->broken;
  HostChain &hc = p->chains[h->chain];
  if (seed != hc.d.seed) {  // as gesmc_run: the round numbering goes on
    DeviceGuard g(p->device);
    hc.d.start_round += p->pool_round - hc.d.join;
    hc.d.join = p->pool_round;
    hc.d.seed = seed;
    if (cudaMemcpyAsync(const_cast<ChainDesc *>(p->args.chains) + h->chain, &hc.d, sizeof(ChainDesc),
                        cudaMemcpyHostToDevice, p->stream) != cudaSuccess) {
      cudaGetLastError();
      return GESMC_E_CUDA;
    }
  }
  return pool_es_run(p, switches, h->chain);
}

int gesmc_edges(gesmc_t h, uint64_t *out, uint64_t capacity, int out_on_device, uint64_t *m_out) {
  if (!h) return GESMC_E_INVALID;
  return gesmc_pool_edges(h->pool, h->chain, out, capacity, out_on_device, m_out);
}

int gesmc_stats(gesmc_t h, gesmc_stats_t *out) { return h ? gesmc_pool_stats(h->pool, out) : GESMC_E_INVALID; }
int gesmc_reset_stats(gesmc_t h) { return h ? gesmc_pool_reset_stats(h->pool) : GESMC_E_INVALID; }
int gesmc_set_profiling(gesmc_t h, int enable) {
  return h ? gesmc_pool_set_profiling(h->pool, enable) : GESMC_E_INVALID;
}
int gesmc_verify(gesmc_t h) { return h ? gesmc_pool_verify(h->pool, h->chain) : GESMC_E_INVALID; }
int gesmc_set_round_launch(gesmc_t h, uint32_t ctas, uint32_t *effective) {
  return h ? gesmc_pool_set_round_launch(h->pool, ctas, effective) : GESMC_E_INVALID;
}
int gesmc_stage_times(gesmc_t h, double *ms, int n_stages, uint64_t *rounds) {
  return h ? gesmc_pool_stage_times(h->pool, ms, n_stages, rounds) : GESMC_E_INVALID;
}

const char *gesmc_stage_name(int stage) {
  static const char *names[kNumStages] = {"clear",    "permute", "scan_perm", "sortpair", "boundary", "sources",
                                          "overflow", "group",   "wave1", "waves",     "tail"};
  return (stage >= 0 && stage < kNumStages) ? names[stage] : "";
}

uint64_t gesmc_next_round(gesmc_t h) {
  if (!h) return 0;
  const HostChain &hc = h->pool->chains[h->chain];
  return hc.d.start_round + (h->pool->pool_round - hc.d.join);
}
uint64_t gesmc_num_edges(gesmc_t h) { return h ? h->pool->chains[h->chain].shape.m : 0; }
uint64_t gesmc_num_nodes(gesmc_t h) { return h ? h->pool->chains[h->chain].n : 0; }

}  // extern "C"

// ---------------------------------------------------------------------------
// gesmc_run_noalloc: the round with every scratch byte in one fixed device
// array, for callers that may not allocate device memory (see gesmc.h).
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GESMC_NOALLOC_SCRATCH_BYTES];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_base[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once
// per device; the host-side name of the array is not a device address).
int noalloc_scratch(int dev, void **out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return GESMC_E_INVALID;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_base[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return GESMC_E_CUDA;
    }
    g_noalloc_base[dev] = p;
  }
  *out = g_noalloc_base[dev];
  return GESMC_OK;
}

}  // namespace

extern "C" int gesmc_run_noalloc(uint64_t *edges, uint64_t m, uint64_t n, uint64_t global_switches, uint64_t seed,
                                 uint64_t start_round, void *stream) {
  if (m > GESMC_NOALLOC_MAX_EDGES) return GESMC_E_TOO_LARGE;
  if ((m > 0 && !edges) || n > (1ull << 32)) return GESMC_E_INVALID;
  gesmc_pool_ctx p;  // host bookkeeping only; the device state lives in the scratch array
  if (cudaGetDevice(&p.device) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, p.device);
  if (p.num_sms < 1) p.num_sms = 1;
  int rc = noalloc_scratch(p.device, &p.base);
  if (rc != GESMC_OK) return rc;
  p.owns_memory = false;
  p.use_graphs = false;
  p.stream = (cudaStream_t)stream;
  p.max_edges = GESMC_NOALLOC_MAX_EDGES;
  p.max_chains = 1;
  p.tuple_log2 = kDefaultTupleLog2;
  p.cap = pool_capacity(p.max_edges, 1, p.tuple_log2);
  p.lay = pool_layout(p.cap, p.max_edges, 1);
  if (p.lay.total > GESMC_NOALLOC_SCRATCH_BYTES) return GESMC_E_INTERNAL;
  gesmc_pool_opts o;
  gesmc_pool_opts_default(&o);
  // the array keeps the previous call's contents: pool_init resets the owner
  // maps and counters, and adding the chain rebuilds all of its state
  rc = pool_init(&p, o);
  uint32_t chain = 0;
  if (rc == GESMC_OK)
    rc = pool_add_device(&p, reinterpret_cast<unsigned long long *>(edges), m, n, seed, start_round, 0, 0u, &chain);
  if (rc == GESMC_OK) rc = pool_run(&p, global_switches);
  if (rc == GESMC_OK &&
      (launch_store_chain(p.args, p.chains[chain].d, reinterpret_cast<unsigned long long *>(edges), p.stream,
                          p.num_sms) != cudaSuccess ||
       cudaStreamSynchronize(p.stream) != cudaSuccess)) {
    cudaGetLastError();
    rc = GESMC_E_CUDA;
  }
  return rc;
}
