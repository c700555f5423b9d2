// Internal declarations shared by the CUDA translation units of libgesmc.
//
// A pool holds any number of independent chains (G-ES-MC runs on their own
// graphs, seeds and round counters).  Each chain owns contiguous ranges of
// five index spaces: slots (one per edge), switches (one per pair of slots),
// permutation buckets, tuple partitions and tuple storage.  Small owner
// arrays map an index back to its chain (kNoChain for an unused index).
// Every round runs the same kernels over all chains at once; a chain's
// randomness, buckets and partitions are its own, so its result does not
// depend on the other chains.
//
// Per chain, the edge list is kept in the slot order of its last round, as
// (position, edge) pairs: cpos[s], cedge[s] hold the position and the edge
// that slot s had when that round started; status[k] says whether switch k
// (slots 2k, 2k+1 of the chain) was legal.  The rewiring of a legal switch
// (Def. 1, E[i] <- e3, E[j] <- e4) is applied on the fly by the next pass
// that reads the pair, so no round writes edges at random positions.
//
//   cpos/cedge   u32 / u64 [slots]        list in last-round slot order
//   prec         uint4[buckets * cap]     permutation bucket records:
//                                         {32 key bits, position, edge lo, hi}
//   word         u32[switches]            outright-reject code | flags
//   sw           uint2[switches]          dependency entries of e3, e4
//   status       u32[switches]            (wave << 2) | state
//   ptup         uint4[tuple storage]     Algorithm 1's tuples (four per
//                                         switch) in fixed-capacity hash
//                                         partitions: {id lo, id hi, value,
//                                         low 32 bits of the id's hash}
//   otup/stup    uint4[overflow cap]      tuples beyond a partition's
//                                         capacity ({.., partition}), and
//                                         the same grouped by partition in
//                                         the ptup format (rare); stup
//                                         shares prec's bytes (the records
//                                         are dead after the sort)
//   dep          uint2[dep cap]           {p, q} of every edge id with a
//                                         dependency
//   tfilter      u32[bits / 32]           target filter: the bit of every
//                                         target id of the round is set
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gesmc {

constexpr unsigned long long kEmptyKey = ~0ull;  // would be the loop {2^32-1, 2^32-1}: never an edge
constexpr unsigned long long kTombKey = ~0ull - 1;  // {2^32-1, 2^32-2}: not canonical, never an edge
constexpr uint32_t kNoChain = 0xFFFFFFFFu;

// Tuple value (Algorithm 1's (e, k, type)): bit 31 = the edge is a source
// (ERASE) of switch k, else a target (INSERT); bit 30 = which target (e3: 0,
// e4: 1); bits 29..0 = k (pool-wide switch index), or kKeepK for a source
// that no switch erases.
constexpr uint32_t kTupleSource = 0x80000000u;
constexpr uint32_t kTupleWhich = 0x40000000u;
constexpr uint32_t kTupleK = 0x3FFFFFFFu;
constexpr uint32_t kKeepK = 0x3FFFFFFFu;

// {p, q} of an edge id with a dependency (one entry per such id and round):
//   p  switch that erases it, kPKeep if it is in E at the start of the
//      round but no switch erases it, kPNone if it is not in E then;
//   q  smallest switch that inserts it and is not known to be illegal,
//      kQNone if none is left.
// Obs. 2 makes p unique per edge id, so one field suffices.  Switch indices
// of one chain are contiguous and in the chain's own order, so comparing
// pool-wide indices compares positions in the chain's global switch.
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
                   kErrGroup = 32u, kErrCopy = 64u, kErrGridSync = 128u;

// Polls of the one-launch round's grid barrier before a CTA gives up (sets
// kErrGridSync and leaves the kernel); each poll sleeps about 64 ns, so the
// wait is bounded at about a second.
constexpr uint32_t kGridWaitPolls = 1u << 24;

// Polls of an mbarrier before a kernel gives up on a bulk copy (sets
// kErrCopy and returns instead of waiting on).
constexpr uint32_t kCopyWaitPolls = 1u << 22;

// Wave cap used when the caller passes max_waves = 0.  Every wave decides at
// least the smallest undecided switch of some chain, so a round needs at
// most (largest L) + 1 waves; rounds observed in practice need a handful.
// The cap bounds the time a faulty input or build can spend in one round.
constexpr uint32_t kDefaultWaveCap = 10000;

// Waves after the first run on the whole GPU as pairs of kernels (register,
// decide), as many pairs as the pool's rounds have needed so far, at most
// kMaxWaveKernels; k_tail runs any remaining waves on one CTA.
constexpr uint32_t kMaxWaveKernels = 8;

// Permutation buckets: a chain's positions go to 2^B buckets by the top B
// bits of their key, each bucket sorted in shared memory by one CTA.  A
// pool's buckets hold about 2^(c - 1) positions with room for 2^c, c =
// bucket_log2(max edges): 10 (CTAs of 128 threads, eight per SM) for pools
// of at most 2^27 edges, whose at most 2^18 buckets keep their write
// frontiers (one partly filled line per bucket) in L2; 11 (CTAs of 256
// threads) above that, where twice as many buckets would spill them.
constexpr uint32_t kBucketLog2Small = 10, kBucketLog2Large = 11;
constexpr unsigned long long kBucketSmallMaxEdges = 1ull << 27;
inline uint32_t bucket_log2(unsigned long long max_edges) {
  return max_edges <= kBucketSmallMaxEdges ? kBucketLog2Small : kBucketLog2Large;
}

// Tuple partitions: a chain's tuples go to 2^P partitions by the top P bits
// of the hash of the edge id (about 2^tuple_log2 tuples each, room for
// twice that); one CTA groups a partition by edge id in a shared-memory
// table of 2^group_log2 slots of 20 bytes.
constexpr int kDefaultTupleLog2 = 10;
constexpr int kDefaultGroupLog2 = 11;
constexpr int kMaxGroupLog2 = 13;
constexpr int kGroupThreads = 1024;
constexpr int kGroupSlotBytes = 20;

constexpr int kWaveHist = 64;

// A chain with at most 2^kSpreadLog2 partitions keeps its partition cursors
// kSpreadStride words (one L2 line) apart: all its sort CTAs append to them
// at once, and packed into a few lines they would contend for them.  Larger
// chains keep them packed (their cursors are spread by number already).
constexpr uint32_t kSpreadLog2 = 12;
constexpr uint32_t kSpreadStride = 32;

// One chain of the pool.  Its round number in pool round R (R rounds
// completed) is start_round + (R - join); its last round's decisions are
// pending in status[] once R > added, the pool round at which the chain was
// added.  (join and start_round move together when the seed changes.)
struct ChainDesc {
  uint32_t slot_base, m;      // slots [slot_base, slot_base + m); slot_base even
  uint32_t switch_base, L;    // switches [switch_base, switch_base + L), L = floor(m/2)
  uint32_t bucket_base, B;    // 2^B permutation buckets from bucket_base
  uint32_t part_base, P;      // 2^P tuple partitions from part_base
  uint32_t tuple_base, capt;  // partition j of the chain holds capt tuples from tuple_base + j * capt
  uint32_t exact_ell, tstride;  // exact l; distance of the chain's partition cursors (words)
  uint32_t tcount_base, pad;    // the chain's partition cursors start here
  unsigned long long seed, start_round, join, added, lazy_threshold;
};

// Device-resident counters of the round in flight.
struct Counters {
  uint32_t pending[2];  // lengths of list0 / list1
  uint32_t boundary;    // straddling pairs listed by the sort kernel
  uint32_t err;         // sticky error bits (cleared by the host per call)
  uint32_t waves;       // waves the last round needed
  uint32_t dep_count;   // dependency entries allocated this round
  uint32_t ovf_count;   // tuples that did not fit their partition
  uint32_t cur;         // list (0 or 1) holding the undecided switches of the next wave
  uint32_t wave_next;   // number of the next wave
  uint32_t wave_blocks; // CTAs of the running wave kernel that have finished
  unsigned long long pool_round;  // rounds the pool has completed
  uint32_t es_stopped;  // ParES jobs stopped for a rebuild of their edge set (per launch)
  uint32_t gbar_pad[19];  // the grid barrier below on an L2 line of its own
  // arrivals at the one-launch round's grid barriers, never reset between
  // launches of the same CTA count (each launch leaves it at a multiple of
  // its CTA count; the host zeroes it when the count changes)
  unsigned long long gbar_arrived;
};

// Device-resident statistics, accumulated over rounds (all chains).
struct StatsDev {
  unsigned long long lazy, accepted, rej_loop, rej_exists;
  unsigned long long waves_total, waves_max;
  unsigned long long wave_hist[kWaveHist];
  unsigned long long last_pending[kWaveHist];
  unsigned long long overflow_tuples, subpass_partitions;
};

// Everything a round kernel needs; passed by value.  The *_hw fields are
// high-water marks of the index spaces (kernels visit [0, hw)).
struct RoundArgs {
  const ChainDesc *chains;
  const uint32_t *owner_slot, *owner_switch, *owner_bucket, *owner_part;
  unsigned long long *chain_accepted;  // per chain
  uint32_t *chain_ell;                 // per chain: switches that run this round (exact-l chains)
  uint32_t *cpos;
  unsigned long long *cedge;
  uint4 *prec;
  uint32_t *pcount;  // per bucket: records appended
  uint32_t *poff;    // per bucket: exclusive scan of pcount within its block of 1024 buckets
  uint32_t *pblk;    // per block of 1024 buckets + 1: exclusive scan of the block sums
  uint32_t *bnd;
  uint32_t *word;
  uint2 *sw;
  uint32_t *status;
  uint32_t *list0;
  uint32_t *list1;
  uint4 *ptup;
  uint4 *otup;
  uint4 *stup;
  uint32_t *tcount;   // partition cursors: chain c's partition j at tcount_base + j * tstride (may exceed capt)
  uint32_t *ocount;   // per partition: overflow tuples
  uint32_t *ooff;     // per partition: offset of its overflow list within its block of 1024 partitions
  uint32_t *oblk;     // per block of 1024 partitions + 1: exclusive scan of the block sums
  uint32_t *ocursor;  // per partition
  uint2 *dep;
  uint32_t *tfilter;      // target filter: one bit per hash of a target id (all chains)
  uint32_t tfilter_mask;  // bits - 1
  Counters *ctl;
  StatsDev *st;
  uint32_t slot_hw, switch_hw, bucket_hw, part_hw, tcount_hw;
  uint32_t ovf_cap, dep_cap;
  uint32_t max_waves;
  uint32_t bucket_log2;  // permutation buckets: room for 2^bucket_log2 records each
  uint32_t group_log2;  // shared-memory grouping table: 2^group_log2 slots
  uint32_t group_grid;  // CTAs of the persistent grouping kernel
  uint32_t any_work;    // some chain has m >= 2
  uint32_t wave_kernels;  // pairs of whole-GPU wave kernels per round
  uint32_t chain_hw;      // chain ids in use are below this
  uint32_t any_exact;     // some chain uses exact l with a nonzero threshold
  // launch shapes (host side only, except the strides): the flat pair passes (k_permute, k_sources) take their CTAs' ranges in
  // the order b -> (b * cta_stride) mod CTAs, a bijection (the stride is
  // coprime with the CTA count), so that the CTAs resident at once are spread
  // over all chains of a pool instead of a few neighbouring ones
  uint32_t permute_ctas, permute_stride, sources_ctas, sources_stride;
  // the one-launch round sums each bucket's chain-local offset itself (every
  // chain has at most kLocalOffsetBuckets buckets) instead of a scan stage
  uint32_t fused_local_offsets;
  // the one chain of a pool with a single chain that has at most
  // kAggBuckets buckets (kNoChain otherwise): its positions are appended by
  // k_permute_agg, one cursor atomic per bucket and CTA instead of per record
  uint32_t agg_chain, agg_pairs;  // and its pairs of slots, (m + 1) / 2
};

constexpr uint32_t kAggBuckets = 8192;

constexpr uint32_t kLocalOffsetBuckets = 4096;

// Resident CTAs of the persistent and grid-stride round kernels on a device.
struct LaunchShapes {
  uint32_t group;
};

// Stages of a round, in launch order.
enum Stage {
  kStageClear = 0,
  kStagePermute,
  kStageScanPerm,
  kStageSortPair,
  kStageBoundary,
  kStageSources,
  kStageOverflow,
  kStageGroup,
  kStageWave1,
  kStageWaves,
  kStageTail,
  kNumStages
};

// Dynamic shared memory of the grouping kernel; prepare_kernels opts in to
// the largest table once and returns the persistent grid for this table
// size and the single-wave grids of the grid-stride kernels (CTAs that fit
// on the device at once).
size_t group_smem_bytes(uint32_t group_log2);
cudaError_t prepare_kernels(uint32_t group_log2, int num_sms, LaunchShapes *shapes);

// One pool round.  ev (optional) receives kNumStages + 1 events around the
// stages; *launches (optional) counts the kernels launched.
cudaError_t launch_round(const RoundArgs &a, cudaStream_t s, int num_sms, cudaEvent_t *ev, uint32_t *launches);

// The one-launch round: every stage of a pool round in one cooperative launch
// of `ctas` CTAs (at most fused_max_ctas() of them), the stages separated by
// grid barriers with bounded waits.  The same lists, counters and wave
// telemetry as launch_round; for pools whose rounds are bound by launch
// latency.
constexpr int kFusedThreads = 512;
size_t fused_smem_bytes(uint32_t group_log2);
cudaError_t prepare_fused(uint32_t group_log2, int num_sms, uint32_t *max_ctas);
cudaError_t launch_round_fused(const RoundArgs &a, cudaStream_t s, uint32_t ctas);
// One chain (host copy of its descriptor): load a position-order list into
// its slots, and write its current list by position.
cudaError_t launch_load_chain(const RoundArgs &a, const ChainDesc &ch, const unsigned long long *E, cudaStream_t s,
                              int num_sms);
cudaError_t launch_store_chain(const RoundArgs &a, const ChainDesc &ch, unsigned long long *E, cudaStream_t s,
                               int num_sms);
// Fill n u32 words with v.
cudaError_t launch_fill_u32(uint32_t *p, uint32_t n, uint32_t v, cudaStream_t s, int num_sms);
cudaError_t launch_canonicalise(unsigned long long *E, uint32_t m, unsigned long long n_bound, uint32_t *flags,
                                uint32_t *max_id, cudaStream_t s, int num_sms);
// Debug check of a list: kFlagLoop for an entry that is not canonical and
// loop-free, kFlagRange for an id >= n (if n), and its degree fingerprint
// added to *fp (zero it first).
cudaError_t launch_list_check(const unsigned long long *E, uint32_t m, unsigned long long n, uint32_t *flags,
                              unsigned long long *fp, cudaStream_t s, int num_sms);
// Repeated edges, with an open-addressing set of `cap` u64 slots as scratch.
cudaError_t launch_duplicate_check(const unsigned long long *E, uint32_t m, unsigned long long *set,
                                   unsigned long long cap, uint32_t *flags, cudaStream_t s, int num_sms);

// ParES (Algorithm 2) for one chain: its list in position order (in the
// chain's tuple storage) and its edge set (open addressing, 2^hlog2 slots,
// in the chain's permutation records), neither of which a round uses
// between rounds; ES-MC switches k0 .. k0 + count - 1 with the chain's seed.
struct EsJob {
  unsigned long long *E;
  unsigned long long *H;
  unsigned long long seed, k0, count;  // the kernel advances k0 and count as it goes
  uint32_t m, hlog2, chain;
  uint32_t stopped;  // the kernel stopped this job for a rebuild of its set on the whole GPU
};

// Shared-memory opt-in of the ParES kernels, once per device.
cudaError_t prepare_es_kernels();
// Switches per window of the ParES kernel for a chain of m edges (1024,
// 256, 128 or 32, by chain size).
uint32_t es_window(uint32_t m);
// Edge sets of all jobs (or only of the stopped ones) rebuilt from their lists.
cudaError_t launch_es_set(const EsJob *jobs, uint32_t njobs, uint32_t *err, cudaStream_t s, int num_sms,
                          bool only_stopped);
// All jobs' switches, one CTA per job: the first group[0] jobs with windows
// of 1024, the next group[1] with windows of 256, then group[2] with 128 and
// group[3] with 32 (these two on s2, forked from and joined back into s
// through the two events, if given).  *launches receives the number of
// launches.
// Jobs of the largest window stop when their set needs a rebuild (counted
// in *nstop); the caller rebuilds those sets and launches again.
cudaError_t launch_es_run(EsJob *jobs, const uint32_t (&group)[4], StatsDev *stats,
                          unsigned long long *chain_acc, uint32_t *err, uint32_t *nstop, cudaStream_t s,
                          cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join, uint32_t *launches);
// Lists of the chains with a job (job_of[chain] != kNoChain) out of their
// slots into the jobs' position-order lists, and back (slots in position
// order, nothing pending).
cudaError_t launch_es_store(const RoundArgs &a, const EsJob *jobs, const uint32_t *job_of, cudaStream_t s,
                            int num_sms);
cudaError_t launch_es_load(const RoundArgs &a, const EsJob *jobs, const uint32_t *job_of, cudaStream_t s,
                           int num_sms);

// Flags written by the create-time validation kernels.
constexpr uint32_t kFlagLoop = 1u, kFlagRange = 2u, kFlagMulti = 4u, kFlagTableFull = 8u;

}  // namespace gesmc
