// C ABI of libgesmc (declared in include/gesmc.h): handle life cycle, device
// memory plan, create-time validation and the round loop of Algorithm 3
// (ParGlobalES) of arXiv 2111.03005.
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/gesmc.h"
#include "gesmc_internal.cuh"

using namespace gesmc;

namespace {

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Sizes of the pieces of one handle's single device allocation.
struct Plan {
  uint64_t m = 0;
  uint32_t L = 0, B = 0, nb = 1, P = 0, np = 1, group_log2 = 0;
  size_t off_E, off_cpos, off_cedge, off_prec, off_pcount, off_poff, off_pib_pos, off_pib_edge, off_bnd, off_word,
      off_sw, off_status, off_list0, off_list1, off_ptup, off_otup, off_stup, off_tcount, off_ocount, off_ooff,
      off_ocursor, off_dep, off_ctl, off_st, off_scratch, total;
  uint32_t capt = 0;
};

// Largest m: switch indices must fit the 30 bits a tuple gives them.
constexpr uint64_t kMaxEdges = (1ull << 31) - 1;

bool make_plan(uint64_t m, Plan *p, uint32_t tuple_log2 = 0, uint32_t group_log2 = 0) {
  if (m > kMaxEdges) return false;
  if (!tuple_log2) tuple_log2 = kDefaultTupleLog2;
  if (!group_log2) group_log2 = kDefaultGroupLog2;
  if (tuple_log2 < 8 || tuple_log2 > 16 || group_log2 < 10 || group_log2 > (uint32_t)kMaxGroupLog2) return false;
  p->group_log2 = group_log2;
  p->m = m;
  p->L = (uint32_t)(m / 2);
  uint32_t B = 0;  // permutation buckets of about 2^kPermAvgLog2 positions
  while ((m >> B) > (1ull << kPermAvgLog2)) ++B;
  p->B = B;
  p->nb = 1u << B;
  const uint64_t ntuple = 4ull * p->L + 1;
  uint32_t P = 0;  // tuple partitions of about 2^tuple_log2 tuples
  while ((ntuple >> P) > (1ull << tuple_log2)) ++P;
  p->P = P;
  p->np = 1u << P;
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o = align_up(o + (bytes ? bytes : 1));
    return at;
  };
  const size_t L = p->L;
  p->off_E = take(8 * m);
  p->off_cpos = take(4 * m);
  p->off_cedge = take(8 * m);
  p->off_prec = take(16ull * p->nb * kPermBucketCap);
  p->off_pcount = take(4ull * p->nb);
  p->off_poff = take(4ull * (p->nb + 1));
  p->off_pib_pos = take(4 * m);
  p->off_pib_edge = take(8 * m);
  p->off_bnd = take(4ull * (p->nb + 1));
  p->off_word = take(4 * L);
  p->off_sw = take(8 * L);
  p->off_status = take(4 * L);
  p->off_list0 = take(4 * L);
  p->off_list1 = take(4 * L);
  // a partition has room for twice its mean (at least 64 tuples)
  p->capt = (uint32_t)((ntuple >> P) * 2 + 64);
  p->off_ptup = take(16ull * p->np * p->capt);
  p->off_otup = take(16 * ntuple);
  p->off_stup = take(16 * ntuple);
  p->off_tcount = take(4ull * p->np);
  p->off_ocount = take(4ull * p->np);
  p->off_ooff = take(4ull * (p->np + 1));
  p->off_ocursor = take(4ull * p->np);
  p->off_dep = take(8 * (2 * L + 1));
  p->off_ctl = take(sizeof(Counters));
  p->off_st = take(sizeof(StatsDev));
  p->off_scratch = take(64);
  p->total = o;
  return true;
}

template <class T>
T *at(void *base, size_t off) {
  return reinterpret_cast<T *>(static_cast<char *>(base) + off);
}

// Round arguments for a plan laid out at `base` (the edge list E is the
// plan's own piece unless `E` is given).
RoundArgs args_for(const Plan &p, void *base) {
  RoundArgs a;
  std::memset(&a, 0, sizeof(a));
  a.cpos = at<uint32_t>(base, p.off_cpos);
  a.cedge = at<unsigned long long>(base, p.off_cedge);
  a.prec = at<uint4>(base, p.off_prec);
  a.pcount = at<uint32_t>(base, p.off_pcount);
  a.poff = at<uint32_t>(base, p.off_poff);
  a.pib_pos = at<uint32_t>(base, p.off_pib_pos);
  a.pib_edge = at<unsigned long long>(base, p.off_pib_edge);
  a.bnd = at<uint32_t>(base, p.off_bnd);
  a.word = at<uint32_t>(base, p.off_word);
  a.sw = at<uint2>(base, p.off_sw);
  a.status = at<uint32_t>(base, p.off_status);
  a.list0 = at<uint32_t>(base, p.off_list0);
  a.list1 = at<uint32_t>(base, p.off_list1);
  a.ptup = at<uint4>(base, p.off_ptup);
  a.otup = at<uint4>(base, p.off_otup);
  a.stup = at<uint4>(base, p.off_stup);
  a.tcount = at<uint32_t>(base, p.off_tcount);
  a.ocount = at<uint32_t>(base, p.off_ocount);
  a.ooff = at<uint32_t>(base, p.off_ooff);
  a.ocursor = at<uint32_t>(base, p.off_ocursor);
  a.capt = p.capt;
  a.dep = at<uint2>(base, p.off_dep);
  a.ctl = at<Counters>(base, p.off_ctl);
  a.st = at<StatsDev>(base, p.off_st);
  a.m = (uint32_t)p.m;
  a.L = p.L;
  a.B = p.B;
  a.nb = p.nb;
  a.P = p.P;
  a.np = p.np;
  a.group_log2 = p.group_log2;
  a.apply = 0;
  return a;
}

// Validate and canonicalise E in place (loops, ids >= n_bound, repeated
// edges, in that precedence), then load it as the slot-order state of `a`.
// *n_out receives n_bound, or largest id + 1 if n_bound is 0.  Synchronises
// the stream.
int validate_and_load(const RoundArgs &a, unsigned long long *E, uint64_t m, uint64_t n_bound, uint32_t *flags,
                      cudaStream_t s, int sms, uint64_t *n_out) {
  uint32_t host_flags[2] = {0, 0};
  bool ok = cudaMemsetAsync(a.ctl, 0, sizeof(Counters), s) == cudaSuccess;
  ok &= cudaMemsetAsync(a.st, 0, sizeof(StatsDev), s) == cudaSuccess;
  ok &= cudaMemsetAsync(flags, 0, 8, s) == cudaSuccess;
  if (ok && m > 0) ok &= launch_canonicalise(E, (uint32_t)m, n_bound, flags, flags + 1, s, sms) == cudaSuccess;
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
  // the overflow-tuple array (16 bytes x (4L + 1)) serves as the duplicate set's slots
  ok &= launch_duplicate_check(E, (uint32_t)m, reinterpret_cast<unsigned long long *>(a.otup), 2 * (4ull * a.L + 1),
                               flags, s, sms) == cudaSuccess;
  ok &= launch_load_state(a, E, s, sms) == cudaSuccess;
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

}  // namespace

struct gesmc_ctx {
  int device = 0;
  int num_sms = 1;
  cudaStream_t stream = nullptr;
  gesmc_alloc_fn alloc = nullptr;
  gesmc_free_fn free_fn = nullptr;
  void *alloc_ctx = nullptr;
  void *base = nullptr;
  Plan plan;
  uint64_t n = 0;
  uint64_t next_round = 0;
  uint64_t lazy_threshold = 0;
  uint32_t max_waves = 0;
  uint64_t rounds = 0;
  uint64_t launches = 0;
  int broken = 0;
  RoundArgs args;
  // stage timing (gesmc_set_profiling): kNumStages + 1 events per round
  int profiling = 0;
  std::vector<cudaEvent_t> events;
  double stage_ms[kNumStages] = {};
  uint64_t stage_rounds = 0;
};

namespace {

void *dev_alloc(gesmc_ctx *h, size_t bytes) {
  if (h->alloc) return h->alloc(bytes, (void *)h->stream, h->alloc_ctx);
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(gesmc_ctx *h, void *p) {
  if (!p) return;
  if (h->free_fn) h->free_fn(p, h->alloc_ctx);
  else cudaFree(p);
}

int map_device_errors(uint32_t err) {
  if (err & kErrTableFull) return GESMC_E_TABLE_FULL;
  if (err & kErrWaveCap) return GESMC_E_WAVE_CAP;
  if (err & (kErrBucket | kErrNoProgress | kErrRecord | kErrGroup)) return GESMC_E_INTERNAL;
  return GESMC_OK;
}

}  // namespace

extern "C" {

void gesmc_opts_default(gesmc_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
}

size_t gesmc_device_bytes(uint64_t m) {
  Plan p;
  if (!make_plan(m, &p)) return 0;
  return p.total;
}

const char *gesmc_strerror(int code) {
  switch (code) {
    case GESMC_OK: return "ok";
    case GESMC_E_INVALID: return "invalid argument";
    case GESMC_E_LOOP: return "edge list contains a loop";
    case GESMC_E_MULTI: return "edge list contains a repeated edge";
    case GESMC_E_RANGE: return "node id out of range";
    case GESMC_E_NOMEM: return "device allocation failed";
    case GESMC_E_CUDA: return "CUDA runtime error";
    case GESMC_E_TABLE_FULL: return "dependency table full";
    case GESMC_E_WAVE_CAP: return "wave cap exceeded";
    case GESMC_E_INTERNAL: return "internal error (permutation bucket overflow)";
    case GESMC_E_CAPACITY: return "output buffer too small";
    case GESMC_E_TOO_LARGE: return "edge list larger than the no-alloc scratch allows (GESMC_NOALLOC_MAX_EDGES)";
    default: return "unknown error";
  }
}

void gesmc_destroy(gesmc_t h) {
  if (!h) return;
  {
    DeviceGuard g(h->device);
    if (h->base) {
      cudaStreamSynchronize(h->stream);
      dev_free(h, h->base);
    }
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  }
  delete h;
}

int gesmc_create(const uint64_t *edges, uint64_t m, int edges_on_device, const gesmc_opts *opts, gesmc_t *out) {
  if (!out) return GESMC_E_INVALID;
  *out = nullptr;
  gesmc_opts o;
  gesmc_opts_default(&o);
  if (opts) o = *opts;
  if (m > kMaxEdges || (m > 0 && !edges)) return GESMC_E_INVALID;
  if (o.n > (1ull << 32)) return GESMC_E_INVALID;
  if ((o.alloc == nullptr) != (o.free == nullptr)) return GESMC_E_INVALID;

  gesmc_ctx *h = new (std::nothrow) gesmc_ctx();
  if (!h) return GESMC_E_NOMEM;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return GESMC_E_CUDA;
  }
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (h->num_sms < 1) h->num_sms = 1;
  h->stream = (cudaStream_t)o.stream;
  h->alloc = o.alloc;
  h->free_fn = o.free;
  h->alloc_ctx = o.alloc_ctx;
  h->next_round = o.start_round;
  h->lazy_threshold = o.lazy_threshold;
  h->max_waves = o.max_waves;
  if (!make_plan(m, &h->plan, o.tuple_log2, o.group_log2)) {
    delete h;
    return GESMC_E_INVALID;
  }
  uint32_t group_grid = 0;
  if (prepare_kernels(h->plan.group_log2, h->num_sms, &group_grid) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return GESMC_E_CUDA;
  }
  const Plan &p = h->plan;
  h->base = dev_alloc(h, p.total);
  if (!h->base) {
    delete h;
    return GESMC_E_NOMEM;
  }
  h->args = args_for(p, h->base);
  h->args.group_grid = group_grid;
  h->args.lazy_threshold = o.lazy_threshold;
  h->args.max_waves = o.max_waves;
  unsigned long long *E = at<unsigned long long>(h->base, p.off_E);
  int rc = GESMC_OK;
  if (m > 0 && cudaMemcpyAsync(E, edges, 8 * m, edges_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               h->stream) != cudaSuccess) {
    cudaGetLastError();
    rc = GESMC_E_CUDA;
  }
  if (rc == GESMC_OK)
    rc = validate_and_load(h->args, E, m, o.n, at<uint32_t>(h->base, p.off_scratch), h->stream, h->num_sms, &h->n);
  if (rc != GESMC_OK) {
    gesmc_destroy(h);
    return rc;
  }
  *out = h;
  return GESMC_OK;
}

int gesmc_run(gesmc_t h, uint64_t global_switches, uint64_t seed) {
  if (!h) return GESMC_E_INVALID;
  if (h->broken) return h->broken;
  DeviceGuard g(h->device);
  cudaStream_t s = h->stream;
  RoundArgs a = h->args;
  a.seed = seed;
  if (cudaMemsetAsync(&a.ctl->err, 0, sizeof(uint32_t), s) != cudaSuccess) return GESMC_E_CUDA;
  const size_t per_round = kNumStages + 1;
  if (h->profiling) {
    const size_t need = per_round * (size_t)global_switches;
    while (h->events.size() < need) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return GESMC_E_CUDA;
      }
      h->events.push_back(e);
    }
  }
  uint32_t launches = 0;
  for (uint64_t r = 0; r < global_switches; ++r) {
    a.round = h->next_round + r;
    cudaEvent_t *ev = h->profiling ? &h->events[per_round * r] : nullptr;
    if (launch_round(a, s, h->num_sms, ev, &launches) != cudaSuccess) {
      h->broken = GESMC_E_CUDA;
      return GESMC_E_CUDA;
    }
    a.apply = 1;  // status[] now holds this round's decisions
    h->args.apply = 1;
  }
  Counters ctl;
  if (cudaMemcpyAsync(&ctl, a.ctl, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    h->broken = GESMC_E_CUDA;
    return GESMC_E_CUDA;
  }
  if (h->profiling) {
    for (uint64_t r = 0; r < global_switches; ++r) {
      for (int st = 0; st < kNumStages; ++st) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->events[per_round * r + st], h->events[per_round * r + st + 1]) ==
            cudaSuccess)
          h->stage_ms[st] += ms;
      }
    }
    h->stage_rounds += global_switches;
  }
  h->next_round += global_switches;
  h->rounds += global_switches;
  h->launches += launches;
  const int rc = map_device_errors(ctl.err);
  if (rc != GESMC_OK) h->broken = rc;
  return rc;
}

int gesmc_edges(gesmc_t h, uint64_t *out, uint64_t capacity, int out_on_device, uint64_t *m_out) {
  if (!h) return GESMC_E_INVALID;
  if (m_out) *m_out = h->plan.m;
  if (capacity < h->plan.m) return GESMC_E_CAPACITY;
  if (h->plan.m == 0) return GESMC_OK;
  if (!out) return GESMC_E_INVALID;
  DeviceGuard g(h->device);
  // the list is kept in the last round's slot order: write it by position
  unsigned long long *E = out_on_device ? reinterpret_cast<unsigned long long *>(out)
                                        : at<unsigned long long>(h->base, h->plan.off_E);
  bool ok = launch_store_state(h->args, E, h->stream, h->num_sms) == cudaSuccess;
  if (ok && !out_on_device)
    ok = cudaMemcpyAsync(out, E, 8 * h->plan.m, cudaMemcpyDeviceToHost, h->stream) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(h->stream) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  return GESMC_OK;
}

int gesmc_stats(gesmc_t h, gesmc_stats_t *out) {
  if (!h || !out) return GESMC_E_INVALID;
  DeviceGuard g(h->device);
  StatsDev st;
  if (cudaMemcpyAsync(&st, h->args.st, sizeof(StatsDev), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  std::memset(out, 0, sizeof(*out));
  out->rounds = h->rounds;
  out->switches = h->rounds * (uint64_t)h->plan.L;
  out->lazy = st.lazy;
  out->accepted = st.accepted;
  out->rejected_loop = st.rej_loop;
  out->rejected_exists = st.rej_exists;
  out->kernel_launches = h->launches;
  out->perm_buckets = h->plan.nb;
  out->tuple_partitions = h->plan.np;
  out->waves_total = st.waves_total;
  out->waves_max = st.waves_max;
  for (int w = 0; w < GESMC_WAVE_HIST && w < kWaveHist; ++w) {
    out->wave_hist[w] = st.wave_hist[w];
    out->last_round_pending[w] = st.last_pending[w];
  }
  return GESMC_OK;
}

int gesmc_reset_stats(gesmc_t h) {
  if (!h) return GESMC_E_INVALID;
  DeviceGuard g(h->device);
  if (cudaMemsetAsync(h->args.st, 0, sizeof(StatsDev), h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  h->rounds = 0;
  h->launches = 0;
  for (double &x : h->stage_ms) x = 0.0;
  h->stage_rounds = 0;
  return GESMC_OK;
}

int gesmc_set_profiling(gesmc_t h, int enable) {
  if (!h) return GESMC_E_INVALID;
  h->profiling = enable ? 1 : 0;
  return GESMC_OK;
}

int gesmc_stage_times(gesmc_t h, double *ms, int n_stages, uint64_t *rounds) {
  if (!h || (n_stages > 0 && !ms)) return GESMC_E_INVALID;
  for (int st = 0; st < n_stages; ++st) ms[st] = st < kNumStages ? h->stage_ms[st] : 0.0;
  if (rounds) *rounds = h->stage_rounds;
  return GESMC_OK;
}

const char *gesmc_stage_name(int stage) {
  static const char *names[kNumStages] = {"clear",    "permute", "scan_perm", "sortpair", "boundary",
                                          "overflow", "group",   "wave1",     "tail"};
  return (stage >= 0 && stage < kNumStages) ? names[stage] : "";
}

uint64_t gesmc_next_round(gesmc_t h) { return h ? h->next_round : 0; }
uint64_t gesmc_num_edges(gesmc_t h) { return h ? h->plan.m : 0; }
uint64_t gesmc_num_nodes(gesmc_t h) { return h ? h->n : 0; }

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
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  void *base = nullptr;
  int rc = noalloc_scratch(dev, &base);
  if (rc != GESMC_OK) return rc;
  Plan p;
  if (!make_plan(m, &p) || p.total > GESMC_NOALLOC_SCRATCH_BYTES) return GESMC_E_INTERNAL;
  uint32_t group_grid = 0;
  if (prepare_kernels(p.group_log2, sms, &group_grid) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }

  cudaStream_t s = (cudaStream_t)stream;
  RoundArgs a = args_for(p, base);
  a.group_grid = group_grid;
  a.seed = seed;
  unsigned long long *E = reinterpret_cast<unsigned long long *>(edges);  // in place on the caller's list
  uint64_t n_eff = 0;
  // the array keeps the previous call's contents: validate_and_load zeroes
  // the counters and rebuilds all state from the caller's list
  rc = validate_and_load(a, E, m, n, at<uint32_t>(base, p.off_scratch), s, sms, &n_eff);
  if (rc != GESMC_OK) return rc;
  for (uint64_t r = 0; r < global_switches; ++r) {
    a.round = start_round + r;
    if (launch_round(a, s, sms, nullptr, nullptr) != cudaSuccess) {
      cudaGetLastError();
      return GESMC_E_CUDA;
    }
    a.apply = 1;
  }
  Counters ctl;
  if (launch_store_state(a, E, s, sms) != cudaSuccess ||
      cudaMemcpyAsync(&ctl, a.ctl, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return GESMC_E_CUDA;
  }
  return map_device_errors(ctl.err);
}
