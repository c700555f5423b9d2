// Internal declarations shared by the CUDA translation units of libgesmc.
//
// Device state of one chain, for m edges and L = floor(m/2) switches a round.
// The list E is kept in the slot order of the last round, as (position,
// edge) pairs: cpos[s], cedge[s] hold the position and the edge that slot s
// of the last round's permutation had when that round started; status[k]
// says whether switch k (slots 2k, 2k+1) was legal.  The rewiring of a legal
// switch (Def. 1, E[i] <- e3, E[j] <- e4) is applied on the fly by the next
// pass that reads the pair, so no round writes E at random positions.
//
//   cpos/cedge   u32[m] / u64[m]   list in last-round slot order (see above)
//   prec         uint4[nb * cap]   permutation buckets: {32 key bits,
//                                  position, edge lo, edge hi}
//   word         u32[L]            per switch: outright-reject code | flags
//   sw           uint2[L]          per switch: dependency entry of e3, e4
//   status       u32[L]            (wave << 2) | state of each switch
//   ptup         uint4[np * capt]  Algorithm 1's tuples (four per switch),
//                                  appended to fixed-capacity hash partitions
//   otup/stup    uint4[4L+1]       tuples beyond a partition's capacity, and
//                                  the same grouped by partition (rare)
//   dep          uint2[2L+1]       {p, q} of every edge id with a dependency
//   E            u64[m]            position-order copy (input / output only)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gesmc {

constexpr unsigned long long kEmptyKey = ~0ull;  // would be the loop {2^32-1, 2^32-1}: never an edge

// Tuple value (Algorithm 1's (e, k, type)): bit 31 = the edge is a source
// (ERASE) of switch k, else a target (INSERT); bit 30 = which target (e3: 0,
// e4: 1); bits 29..0 = k, or kKeepK for a source that no switch erases.
constexpr uint32_t kTupleSource = 0x80000000u;
constexpr uint32_t kTupleWhich = 0x40000000u;
constexpr uint32_t kTupleK = 0x3FFFFFFFu;
constexpr uint32_t kKeepK = 0x3FFFFFFFu;

// {p, q} of an edge id with a dependency (one entry per such id and round):
//   p  switch that erases it, kPKeep if it is in E at the start of the
//      round but no switch erases it, kPNone if it is not in E then;
//   q  smallest switch that inserts it and is not known to be illegal,
//      kQNone if none is left.
// Obs. 2 makes p unique per edge id, so one field suffices.
constexpr uint32_t kPNone = 0xFFFFFFFFu;
constexpr uint32_t kPKeep = 0xFFFFFFFEu;
constexpr uint32_t kQNone = 0xFFFFFFFFu;
constexpr uint32_t kTrivial = 0xFFFFFFFFu;  // sw entry: target without a dependency

// word[k]: low two bits = code of a switch rejected as it was built
// (loop, shared node, lazy); flag bits set by the grouping of its targets.
constexpr uint32_t kCodeLoop = 1u, kCodeShared = 2u, kCodeLazy = 3u, kCodeMask = 3u;
constexpr uint32_t kFlagBad = 4u;  // a target is in E when k runs, certainly
constexpr uint32_t kFlagDep = 8u;  // a target depends on an undecided switch

// Switch status word: (wave << 2) | state.  Wave 0 means "not decided".
constexpr uint32_t kUndecided = 0, kLegal = 1, kIllegal = 2;

// Sticky device error bits.
constexpr uint32_t kErrTableFull = 1u, kErrBucket = 2u, kErrWaveCap = 4u, kErrNoProgress = 8u, kErrRecord = 16u,
                   kErrGroup = 32u;

// Wave cap used when the caller passes max_waves = 0.  Every wave decides at
// least the smallest undecided switch, so a round needs at most L + 1 waves;
// rounds observed in practice need a handful.  The cap bounds the time a
// faulty input or build can spend in one round.
constexpr uint32_t kDefaultWaveCap = 10000;

// Permutation buckets: positions go to 2^B buckets by the top B bits of
// their key (about 2^kPermAvgLog2 per bucket, at most kPermBucketCap), and
// each bucket is sorted in shared memory by one CTA.
constexpr int kSortThreads = 256;
constexpr int kPermBucketCap = 2048;
constexpr int kPermAvgLog2 = 10;
constexpr int kPerThread = kPermBucketCap / kSortThreads;
constexpr int kSubBits = 11;

// Tuple partitions: 2^P partitions by the top P bits of the hash of the
// edge id (about 2^tuple_log2 tuples each, room for twice that); one CTA
// groups a partition by edge id in a shared-memory table of 2^group_log2
// slots (22 bytes each, with the used-slot list).  A tuple is {edge id lo,
// edge id hi, value, 0}.
constexpr int kDefaultTupleLog2 = 10;
constexpr int kDefaultGroupLog2 = 11;
constexpr int kMaxGroupLog2 = 13;
constexpr int kGroupThreads = 256;
constexpr int kGroupSlotBytes = 22;

constexpr int kWaveHist = 64;

// Device-resident counters of the round in flight.
struct Counters {
  uint32_t pending[2];  // lengths of list0 / list1
  uint32_t boundary;    // straddling pairs listed by the sort kernel
  uint32_t err;         // sticky error bits (cleared by the host per call)
  uint32_t waves;       // waves the last round needed
  uint32_t dep_count;   // dependency entries allocated this round
  uint32_t ovf_count;   // tuples that did not fit their partition
  uint32_t pad;
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
  uint32_t *cpos;
  unsigned long long *cedge;
  uint4 *prec;
  uint32_t *pcount;  // nb: records per permutation bucket
  uint32_t *poff;    // nb + 1: slot offset of each bucket
  uint32_t *pib_pos;
  unsigned long long *pib_edge;
  uint32_t *bnd;
  uint32_t *word;
  uint2 *sw;
  uint32_t *status;
  uint32_t *list0;
  uint32_t *list1;
  uint4 *ptup;        // np * capt
  uint4 *otup;        // 4L + 1
  uint4 *stup;        // 4L + 1
  uint32_t *tcount;   // np: tuples appended per partition (may exceed capt)
  uint32_t *ocount;   // np: overflow tuples per partition
  uint32_t *ooff;     // np + 1
  uint32_t *ocursor;  // np
  uint2 *dep;
  Counters *ctl;
  StatsDev *st;
  unsigned long long seed, round, lazy_threshold;
  uint32_t m, L, B, nb, P, np, max_waves;
  uint32_t group_log2;  // shared-memory grouping table: 2^group_log2 slots
  uint32_t capt;        // tuple capacity of a partition
  uint32_t group_grid;  // CTAs of the persistent grouping kernel
  uint32_t apply;  // 1 if status[] holds the last round's decisions (apply them when reading)
};

// Stages of a round, in launch order (one kernel each).
enum Stage {
  kStageClear = 0,
  kStagePermute,
  kStageScanPerm,
  kStageSortPair,
  kStageBoundary,
  kStageOverflow,
  kStageGroup,
  kStageWave1,
  kStageTail,
  kNumStages
};

// Dynamic shared memory of the grouping kernel, and the one-time opt-in to
// more than 48 KB of it (call before the first round on a device).
// prepare_kernels also returns the persistent grouping grid for this table
// size (CTAs that fit on the device at once).
size_t group_smem_bytes(uint32_t group_log2);
cudaError_t prepare_kernels(uint32_t group_log2, int num_sms, uint32_t *group_grid);

// Host-side launchers (round.cu).  launch_round records kNumStages + 1
// events into ev (if not null) around the stages and adds the number of
// kernels it launched to *launches (if not null).
cudaError_t launch_round(const RoundArgs &a, cudaStream_t s, int num_sms, cudaEvent_t *ev, uint32_t *launches);
// Position-order list -> slot-order state (cpos[s] = s, cedge[s] = E[s]).
cudaError_t launch_load_state(const RoundArgs &a, const unsigned long long *E, cudaStream_t s, int num_sms);
// Slot-order state (with the last round's decisions applied) -> E by position.
cudaError_t launch_store_state(const RoundArgs &a, unsigned long long *E, cudaStream_t s, int num_sms);
cudaError_t launch_canonicalise(unsigned long long *E, uint32_t m, unsigned long long n_bound, uint32_t *flags,
                                uint32_t *max_id, cudaStream_t s, int num_sms);
// Repeated edges, with an open-addressing set of `cap` u64 slots as scratch.
cudaError_t launch_duplicate_check(const unsigned long long *E, uint32_t m, unsigned long long *set,
                                   unsigned long long cap, uint32_t *flags, cudaStream_t s, int num_sms);

// Flags written by the create-time validation kernels.
constexpr uint32_t kFlagLoop = 1u, kFlagRange = 2u, kFlagMulti = 4u, kFlagTableFull = 8u;

}  // namespace gesmc
