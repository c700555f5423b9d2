// Internal declarations shared by the CUDA translation units of libgesmc.
//
// Device state of one chain, for m edges and L = floor(m/2) switches a round:
//   E        u64[m]      edge list in position order (canonical ids, Sec. 5.2)
//   T        Slot[cap]   dependency table of Algorithm 1 (one slot per edge id
//                        touched in the round: every source edge and every
//                        target edge), open addressing, linear probing
//   buf      u64[m]      permutation buckets: (32 key bits << 32) | position
//   sw       uint4[L]    switch records {i, j, slot(e3), slot(e4)}
//   status   u32[L]      (wave << 2) | state of each switch
//   list0/1  u32[L]      undecided switches entering the next wave
//   pib      u32[m]      permutation entries of slots whose pair straddles
//                        two buckets
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gesmc {

// One slot of the dependency table T (Algorithm 1).  For the edge id `key`:
//   p  index of the switch that erases it (the edge is a source of that
//      switch), kPKeep if the edge is in E at the start of the round but no
//      switch of the round may erase it, kPNone if it is not in E then.
//   q  smallest index among the switches that insert it (target edge) and
//      are not known to be illegal; kQNone if there is none.
// Obs. 2 makes p unique per edge, so a single field suffices.
struct __align__(16) Slot {
  unsigned long long key;
  uint32_t p;
  uint32_t q;
};

constexpr unsigned long long kEmptyKey = ~0ull;  // would be the loop {2^32-1, 2^32-1}: never an edge
constexpr uint32_t kPNone = 0xFFFFFFFFu;
constexpr uint32_t kPKeep = 0xFFFFFFFEu;
constexpr uint32_t kQNone = 0xFFFFFFFFu;

// Codes stored in the third word of a switch record when the switch was
// decided while its record was built (no table slot for its targets).
constexpr uint32_t kSwCodeMin = 0xFFFFFFF0u;
constexpr uint32_t kSwLazy = 0xFFFFFFFDu;    // skipped by the laziness rule (Def. 2)
constexpr uint32_t kSwShared = 0xFFFFFFFEu;  // sources share a node: targets are the sources
constexpr uint32_t kSwLoop = 0xFFFFFFFFu;    // a target is a loop (Def. 1)

// Switch status word: (wave << 2) | state.  Wave 0 means "not decided".
constexpr uint32_t kUndecided = 0, kLegal = 1, kIllegal = 2;

// Sticky device error bits.
constexpr uint32_t kErrTableFull = 1u, kErrBucket = 2u, kErrWaveCap = 4u, kErrNoProgress = 8u, kErrRecord = 16u;

// Wave cap used when the caller passes max_waves = 0.  Every wave decides at
// least the smallest undecided switch, so a round needs at most L + 1 waves;
// rounds observed in practice need a handful.  The cap bounds the time a
// faulty input or build can spend in one round.
constexpr uint32_t kDefaultWaveCap = 10000;

// Permutation tiling: positions are scattered into 2^B buckets by the top B
// bits of their key (about 2^kBucketAvgLog2 per bucket), then each bucket is
// sorted in shared memory by one CTA.
constexpr int kSortThreads = 256;
constexpr int kBucketCap = 4096;
constexpr int kPerThread = kBucketCap / kSortThreads;
constexpr int kSubBits = 11;
constexpr int kBucketAvgLog2 = 10;

constexpr int kWaveHist = 64;

// Device-resident counters of the round in flight.
struct Counters {
  uint32_t pending[2];  // lengths of list0 / list1
  uint32_t boundary;    // straddling pairs listed by the sort kernel
  uint32_t err;         // sticky error bits (cleared by the host per call)
  uint32_t waves;       // waves the last round needed
  uint32_t pad[3];
};

// Device-resident statistics, accumulated over rounds.
struct StatsDev {
  unsigned long long lazy, accepted, rej_loop, rej_exists;
  unsigned long long waves_total, waves_max;
  unsigned long long wave_hist[kWaveHist];
  unsigned long long last_pending[kWaveHist];
};

// Everything a round kernel needs; passed by value.
struct RoundArgs {
  unsigned long long *E;
  Slot *T;
  unsigned long long cap;
  unsigned long long *buf;
  uint32_t *bucket_cnt;
  uint32_t *bucket_off;  // nb + 1 entries
  uint32_t *cursor;
  uint4 *sw;
  uint32_t *status;
  uint32_t *list0;
  uint32_t *list1;
  uint32_t *pib;
  uint32_t *bnd;
  Counters *ctl;
  StatsDev *st;
  unsigned long long seed, round, lazy_threshold;
  uint32_t m, L, B, nb, max_waves;
};

// Stages of a round, in launch order (one kernel each).
enum Stage {
  kStageClear = 0,
  kStageHist,
  kStageScan,
  kStageScatter,
  kStageSortPair,
  kStageBoundary,
  kStageDecide1,
  kStageTail,
  kNumStages
};

// Host-side launchers (round.cu).  launch_round records kNumStages + 1
// events into ev (if not null) around the stages and adds the number of
// kernels it launched to *launches (if not null).
cudaError_t launch_round(const RoundArgs &a, cudaStream_t s, int num_sms, cudaEvent_t *ev, uint32_t *launches);
cudaError_t launch_canonicalise(unsigned long long *E, uint32_t m, unsigned long long n_bound,
                                uint32_t *flags, uint32_t *max_id, cudaStream_t s, int num_sms);
cudaError_t launch_duplicate_check(const unsigned long long *E, uint32_t m, Slot *T, unsigned long long cap,
                                   uint32_t *flags, cudaStream_t s, int num_sms);
cudaError_t launch_clear_table(Slot *T, unsigned long long cap, cudaStream_t s, int num_sms);

// Flags written by the create-time validation kernels.
constexpr uint32_t kFlagLoop = 1u, kFlagRange = 2u, kFlagMulti = 4u, kFlagTableFull = 8u;

}  // namespace gesmc
