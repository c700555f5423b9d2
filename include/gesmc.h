/*
 * gesmc.h -- C ABI of libgesmc, the GB300 (sm_103a) global switch round of
 * the Global Edge Switching Markov Chain (G-ES-MC) of Allendorf, Meyer,
 * Penschuck and Tran, "Parallel Global Edge Switching for the Uniform
 * Sampling of Simple Graphs with Prescribed Degrees" (arXiv 2111.03005).
 *
 * The state of a chain is an indexed edge list E[0..m) of a simple graph
 * (Sec. 2.1).  Edge ids are 64-bit: the smaller node id in the high 32 bits,
 * the larger in the low 32 bits (Sec. 5.2).  One call of gesmc_run performs
 * global switches (Def. 2) one after another, each being floor(m/2) edge
 * switches (Def. 1) over the disjoint pairs of a random permutation of the
 * positions, with exactly the result of running them in sequence (the
 * guarantee of ParallelSuperstep, Algorithm 1, driven as in Algorithm 3).
 *
 * Randomness is counter based: with Philox4x64-10 (Salmon et al., SC'11),
 * round r's permutation is the argsort of the words
 *   K(i) = Philox4x64-10(counter = (i >> 2, r, 0, 0), key = (seed, 0))[i & 3]
 * (ties: smaller position first), and with a nonzero lazy threshold t,
 * switch k of round r is skipped iff
 *   Philox4x64-10(counter = (k >> 2, r, 1, 0), key = (seed, 0))[k & 3] < t,
 * i.e. each switch is skipped with probability P_L = t / 2^64 (Def. 2).
 * Rounds are numbered cumulatively per handle from opts.start_round, so
 * run(a, s) followed by run(b, s) equals run(a + b, s).
 *
 * Errors: every int-returning call returns GESMC_OK (0) or a negative
 * GESMC_E_* code.  After GESMC_E_CUDA, GESMC_E_TABLE_FULL, GESMC_E_WAVE_CAP
 * or GESMC_E_INTERNAL from gesmc_run the edge list is unspecified and only
 * gesmc_stats, gesmc_edges and gesmc_destroy may be called.
 *
 * Threading: a handle may be used by one host thread at a time.  All device
 * work is ordered on opts.stream (the legacy default stream when NULL);
 * every call returns only after its device work has completed.
 */
#ifndef GESMC_H
#define GESMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gesmc_ctx *gesmc_t;

enum {
  GESMC_OK = 0,
  GESMC_E_INVALID = -1,    /* null argument, m >= 2^31, bad option value     */
  GESMC_E_LOOP = -2,       /* input edge {u, u} (not a simple graph)         */
  GESMC_E_MULTI = -3,      /* input edge listed twice (not a simple graph)   */
  GESMC_E_RANGE = -4,      /* input node id >= opts.n                        */
  GESMC_E_NOMEM = -5,      /* device allocation failed                       */
  GESMC_E_CUDA = -6,       /* a CUDA runtime call failed                     */
  GESMC_E_TABLE_FULL = -7, /* dependency table overflow (not expected)       */
  GESMC_E_WAVE_CAP = -8,   /* a round needed more waves than opts.max_waves  */
  GESMC_E_INTERNAL = -9,   /* bucket overflow or stalled waves (not expected) */
  GESMC_E_CAPACITY = -10,  /* caller's output buffer too small               */
  GESMC_E_TOO_LARGE = -11, /* m above GESMC_NOALLOC_MAX_EDGES (no-alloc call), or a chain
                              too large for resident rounds (GESMC_ROUND_RESIDENT) */
  GESMC_E_INVARIANT = -12  /* a checked list is not a simple graph with the
                              starting degree sequence (gesmc_verify)        */
};

/* Rounds are replayed from a captured CUDA graph of one round (launched on
 * a private stream ordered after and before the caller's stream); this flag
 * launches the kernels one by one instead.  Stage timing always launches
 * them one by one. */
#define GESMC_FLAG_NO_GRAPHS 1u
/* Def. 2 as printed: each round draws l ~ Binom(floor(m/2), 1 - P_L) and
 * runs only its first l switches, l = the number of switches whose laziness
 * word is >= lazy_threshold.  Without it, each switch is skipped on its own
 * (word < lazy_threshold), the equivalent per-switch form.  No effect when
 * lazy_threshold is 0. */
#define GESMC_FLAG_EXACT_ELL 2u
/* Fault injection for tests: cap the overflow-tuple list and the table of
 * dependency entries at 16 entries each (instead of room for every tuple
 * and edge id), so that a graph whose edge ids are proposed by many
 * switches makes a round run out of that room.  The kernels check every such
 * capacity before writing, so the round completes, reports
 * GESMC_E_INTERNAL and leaves the handle in the error state described above.
 * Not for production use. */
#define GESMC_FLAG_TINY_OVERFLOW 4u
/* Debugging: check the invariants of gesmc_verify on the device after every
 * round of gesmc_run (rounds then run one call at a time). */
#define GESMC_FLAG_VERIFY_ROUNDS 8u

/* Device allocation hooks: alloc returns device memory usable on `stream`
 * (or NULL on failure); free releases it.  Both NULL: cudaMalloc/cudaFree. */
typedef void *(*gesmc_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*gesmc_free_fn)(void *ptr, void *ctx);

typedef struct gesmc_opts {
  uint64_t n;              /* node ids must be < n; 0: n = largest id + 1       */
  uint64_t lazy_threshold; /* Def. 2 laziness, P_L = t / 2^64; 0: never lazy   */
  uint64_t start_round;    /* number of the first round this handle runs       */
  uint32_t max_waves;      /* cap on resolution waves per round; 0: 10000      */
  uint32_t tuple_log2;     /* tuning: log2 of the mean tuples per dependency
                              partition, 8..16; 0: default                      */
  uint32_t group_log2;     /* tuning: log2 of the shared-memory grouping table
                              slots, 10..13; 0: default                          */
  uint32_t flags;          /* GESMC_FLAG_* bits                                 */
  void *stream;            /* cudaStream_t for all device work; NULL: default  */
  gesmc_alloc_fn alloc;    /* optional device allocator                        */
  gesmc_free_fn free;
  void *alloc_ctx;
} gesmc_opts;

#define GESMC_WAVE_HIST 64

typedef struct gesmc_stats_s {
  uint64_t rounds;          /* global switches run since create / reset           */
  uint64_t switches;        /* floor(m/2) per round (Sec. 6: the unit of work)    */
  uint64_t lazy;            /* switches skipped by the laziness rule              */
  uint64_t accepted;        /* switches that rewired their two edges              */
  uint64_t rejected_loop;   /* a new edge would be a loop (Def. 1)                */
  uint64_t rejected_exists; /* a new edge is in E when the switch runs (Def. 1)   */
  uint64_t kernel_launches; /* CUDA kernels gesmc_run launched                     */
  uint64_t perm_buckets;    /* permutation buckets in use (all chains)            */
  uint64_t tuple_partitions; /* dependency-tuple hash partitions in use             */
  uint64_t waves_total;     /* resolution waves summed over rounds (Algorithm 1's
                               rounds of decide/delay)                            */
  uint64_t waves_max;       /* largest wave count of one round                    */
  uint64_t wave_hist[GESMC_WAVE_HIST]; /* rounds that needed w waves (w >= 63: last) */
  uint64_t last_round_pending[GESMC_WAVE_HIST]; /* undecided switches entering wave
                               w (index w, w >= 1) in the most recent round       */
  uint64_t overflow_tuples; /* dependency tuples that found their hash partition
                               full and took the exact overflow path (a graph
                               with an edge id proposed by many switches)         */
  uint64_t subpass_partitions; /* partitions grouped in several passes (more
                               tuples or distinct ids than one pass holds)        */
} gesmc_stats_t;

/* Fill *o with the defaults named above. */
void gesmc_opts_default(gesmc_opts *o);

/* Create a chain from a simple graph (Sec. 2.1, "degree-valid edge list").
 *   edges: m packed edge ids, either orientation; stored canonically
 *          (min << 32 | max).  Host memory if edges_on_device == 0, else a
 *          device pointer of the current device.  The library copies it; the
 *          caller keeps ownership.
 *   m:     number of edges, < 2^31.
 *   opts:  NULL for defaults.
 *   out:   receives the handle (owns all device state until gesmc_destroy).
 * Returns GESMC_E_LOOP / GESMC_E_RANGE / GESMC_E_MULTI (that precedence) if
 * the list is not a simple graph on [0, n). */
int gesmc_create(const uint64_t *edges, uint64_t m, int edges_on_device, const gesmc_opts *opts,
                 gesmc_t *out);

/* Run `global_switches` rounds of Algorithm 3 (ParGlobalES) with the given
 * seed: each round draws the permutation of Def. 2 and performs its
 * floor(m/2) edge switches with the sequential outcome (Algorithm 1). */
int gesmc_run(gesmc_t h, uint64_t global_switches, uint64_t seed);

/* ParES (Algorithm 2, Sec. 4): run `switches` switches of the plain Edge
 * Switching Markov Chain (Def. 1's chain, ES-MC) on the handle's graph, with
 * the sequential outcome.  Switch k draws Philox4x64-10(counter = (k, 0, 2,
 * 0), key = (seed, 0)) = (w0, w1, w2, w3): i = floor(w0 m / 2^64),
 * j = j' + [j' >= i] with j' = floor(w1 (m - 1) / 2^64), g = the top bit of
 * w2; switches are numbered on from the handle's last ES-MC switch.  Runs
 * in supersteps without source dependencies, one CTA per chain.  May be
 * mixed with gesmc_run on the same handle.  A seed different from the
 * handle's current one re-seeds it as gesmc_run does.  With m < 2 every
 * switch is counted as skipped (stats.lazy).  Synchronises the stream. */
int gesmc_es_run(gesmc_t h, uint64_t switches, uint64_t seed);

/* Copy E, in position order, to `out` (host memory, or device memory if
 * out_on_device != 0); `capacity` is out's length in edges.  *m_out (if not
 * NULL) receives m.  Returns GESMC_E_CAPACITY if capacity < m. */
int gesmc_edges(gesmc_t h, uint64_t *out, uint64_t capacity, int out_on_device, uint64_t *m_out);

/* Counters accumulated by gesmc_run since create or gesmc_reset_stats. */
int gesmc_stats(gesmc_t h, gesmc_stats_t *out);
int gesmc_reset_stats(gesmc_t h);

/* Stage timing.  With profiling on, gesmc_run brackets each kernel of every
 * round with CUDA events on the handle's stream and, after the call's final
 * synchronisation, adds each stage's elapsed time to a per-stage total.
 * gesmc_stage_times copies the totals (milliseconds, since create or
 * gesmc_reset_stats) of the first n_stages stages into ms and the number of
 * profiled rounds into *rounds.  Stage i is named by gesmc_stage_name(i);
 * GESMC_NUM_STAGES stages exist, in launch order, each one kernel except
 * "overflow" (three kernels that return at once when nothing overflowed)
 * and "waves" (a pair of kernels per wave after the first, run on the whole
 * GPU; as many pairs as the handle's rounds have needed extra waves so far,
 * at most 8, none while every round needed one wave; "tail" runs any waves
 * beyond those on one CTA). */
#define GESMC_NUM_STAGES 11
int gesmc_set_profiling(gesmc_t h, int enable);
int gesmc_stage_times(gesmc_t h, double *ms, int n_stages, uint64_t *rounds);
const char *gesmc_stage_name(int stage);

/* How a round is launched.  ctas == 0 (the default): the round's kernels one
 * after another (about 14 of them, replayed from a captured CUDA graph), each
 * shaped for large graphs.  ctas >= 1: the whole round in one cooperative
 * launch of that many 512-thread CTAs (at most as many as the device holds
 * at once; *effective, if not NULL, receives the count used), the stages
 * separated by grid-wide barriers whose waits are bounded (a wait that runs
 * out ends the call with GESMC_E_INTERNAL).  Results are the same either way;
 * the one-launch round saves the launch latency between stages, which
 * dominates the rounds of graphs with up to about 10^5 edges.  The paper has
 * no counterpart (its CPU rounds have no launches).  GESMC_E_INVALID if the
 * device cannot hold one CTA of the one-launch round.  Stage timing
 * (gesmc_set_profiling) always uses the separate kernels.
 *
 * ctas == GESMC_ROUND_RESIDENT: resident rounds, for small chains.  Each
 * chain runs on one 1024-thread CTA that keeps its list (one 32-bit word per
 * edge), the permutation, the switch statuses and a hash table of the round's
 * target edge ids in shared memory, and runs ALL rounds of a gesmc_run call
 * in that one launch (plus a one-CTA launch that folds the rounds' wave
 * counts into the statistics); a round's steps (Philox keys, the counting
 * sort of the positions, the switches, their erasers and inserters,
 * Algorithm 1's decide / delay waves, the rewiring) are separated by CTA
 * barriers only.  When a pool holds few chains, the permutations of the
 * call's rounds are sorted beforehand by one more launch (one CTA per chain
 * and round, on the other SMs), and the chains' CTAs load them.  Calls with
 * more rounds than the pool's scratch space holds take several launches.  Chains qualify with m <= GESMC_RESIDENT_MAX_EDGES and
 * n <= GESMC_RESIDENT_MAX_NODES (n: the node bound given at creation, else
 * the largest id + 1); GESMC_E_TOO_LARGE if a chain does not (and, in a pool,
 * for a later gesmc_pool_add of such a chain).  The same lists, counters and
 * wave telemetry as the other launches.  This is the dedicated base case the
 * paper suggests for small graphs (Sec. 7, Conclusions).  Stage
 * timing has no stages to time in this mode (gesmc_stage_times stays 0). */
#define GESMC_ROUND_RESIDENT 0xFFFFFFFFu
#define GESMC_RESIDENT_MAX_EDGES 10240u
#define GESMC_RESIDENT_MAX_NODES 65536u
int gesmc_set_round_launch(gesmc_t h, uint32_t ctas, uint32_t *effective);

/* Debug check, on the device, of what every round keeps (Sec. 2.1; Def. 1):
 * the handle's list is canonical, loop-free, has ids < n, repeats no edge
 * (so no edge id got two legal inserters in one round, Obs. 2), and has the
 * degree sequence it was created with.  Degrees are compared through a
 * 64-bit fingerprint of the multiset of endpoints (the sum over edges of a
 * fixed hash of each endpoint, mod 2^64), taken when the chain was created.
 * Returns GESMC_OK or GESMC_E_INVARIANT. */
int gesmc_verify(gesmc_t h);
/* The same check on a caller's list: `edges` (m ids, device memory) against
 * the degree sequence of `reference` (ref_m ids, device memory, e.g. the
 * starting list), ids < n if n != 0.  Allocates its scratch memory (a
 * debugging aid).  GESMC_OK, GESMC_E_INVARIANT, GESMC_E_NOMEM or
 * GESMC_E_INVALID. */
int gesmc_verify_list(const uint64_t *edges, uint64_t m, const uint64_t *reference, uint64_t ref_m, uint64_t n);

/* Number of the next round the handle will run (start_round + rounds run). */
uint64_t gesmc_next_round(gesmc_t h);

/* Number of edges and nodes of the chain. */
uint64_t gesmc_num_edges(gesmc_t h);
uint64_t gesmc_num_nodes(gesmc_t h);

/* Device bytes a handle with m edges allocates (0 if m is too large). */
size_t gesmc_device_bytes(uint64_t m);

/* Allocation-free variant of gesmc_create + gesmc_run + gesmc_edges.
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory while they run, for example code running inside
 * a framework that owns all device memory through its own pool, or a process
 * with a fixed memory budget checked at start-up.  Such callers cannot use
 * gesmc_create, which allocates the chain's state.
 *
 * It runs `global_switches` rounds, numbered start_round, start_round + 1, ...
 * with `seed`, in place on `edges`: m packed edge ids in DEVICE memory of the
 * current device (input: a simple graph on [0, n), any orientation, n == 0
 * meaning largest id + 1; output: the list after the rounds, canonical, in
 * position order).  The result equals gesmc_create on the same list (with
 * opts.start_round = start_round) followed by gesmc_run(global_switches, seed)
 * and gesmc_edges.  Work is ordered on `stream` (cudaStream_t; NULL: the
 * legacy default stream) and the call returns after it has completed.
 *
 * All scratch memory is one fixed array of GESMC_NOALLOC_SCRATCH_BYTES in the
 * library's device image, which every GPU that loads the library holds until
 * the process exits.  So m is limited to GESMC_NOALLOC_MAX_EDGES; larger m
 * returns GESMC_E_TOO_LARGE without touching the GPU.  The call makes no
 * device allocation (no cudaMalloc, no allocating library routine).  The
 * first call on a device looks the array's device address up and keeps it for
 * the life of the process; make that first call before any stream capture on
 * that device.  cudaDeviceReset destroys the array: after a reset of a device,
 * do not call this entry point on that device again in the same process (the
 * kept address would be stale).  Every call on a device shares the one array:
 * calls whose device work may overlap (other streams, other host threads) race
 * and must be serialised by the caller.  The device and stream must be the
 * ones `edges` lives on: the call runs on the current device.
 * Returns GESMC_OK, GESMC_E_INVALID, GESMC_E_TOO_LARGE, GESMC_E_LOOP,
 * GESMC_E_RANGE, GESMC_E_MULTI, GESMC_E_CUDA or a round error of gesmc_run.
 * On any error other than GESMC_E_TOO_LARGE and GESMC_E_INVALID, `edges` may
 * have been rewritten in canonical form (min << 32 | max, same positions)
 * before the error was found; nothing else about it changes. */
#define GESMC_NOALLOC_MAX_EDGES 65536
#define GESMC_NOALLOC_SCRATCH_BYTES (20u << 20)
int gesmc_run_noalloc(uint64_t *edges, uint64_t m, uint64_t n, uint64_t global_switches, uint64_t seed,
                      uint64_t start_round, void *stream);

/* Release the handle and its device memory (NULL is ignored). */
void gesmc_destroy(gesmc_t h);

/* ------------------------------------------------------------------------
 * Pools: many independent chains advanced together, one set of kernels per
 * round for all of them (an ensemble of null-model samples, or the chains
 * of a sampling service).  Each chain has its own edge list, seed, round
 * numbering and laziness; its result is bit for bit the one it would have
 * alone (gesmc_create + gesmc_run with the same seed and start round), since
 * every chain draws its permutation and its dependency partitions from its
 * own counters and index ranges.  Chains join and leave between rounds
 * without moving other chains' data (continuous batching).
 *
 * A pool allocates its device memory once, sized for max_edges edges in at
 * most max_chains chains (gesmc_pool_device_bytes tells how much).  Adding a
 * chain fails with GESMC_E_NOMEM when the edges or the chain slots are used
 * up, or when the free index ranges are too fragmented for it.  Threading
 * and errors as for single chains; all device work is on opts.stream.
 * max_edges is at most 2^31 - 1, and every index space the pool sizes from
 * it (tuple storage is the largest, about 2 max_edges) must fit 32 bits;
 * gesmc_pool_create returns GESMC_E_INVALID otherwise, and
 * gesmc_pool_device_bytes returns 0.
 */
typedef struct gesmc_pool_ctx *gesmc_pool_t;

typedef struct gesmc_pool_opts {
  uint64_t max_edges;      /* edges of all chains at once                    */
  uint32_t max_chains;     /* chains at once (>= 1)                          */
  uint32_t max_waves;      /* as gesmc_opts.max_waves                        */
  uint32_t tuple_log2;     /* as gesmc_opts.tuple_log2                       */
  uint32_t group_log2;     /* as gesmc_opts.group_log2                       */
  uint32_t flags;          /* GESMC_FLAG_* bits                              */
  void *stream;            /* cudaStream_t; NULL: the legacy default stream  */
  gesmc_alloc_fn alloc;    /* optional device allocator (as gesmc_opts)      */
  gesmc_free_fn free;
  void *alloc_ctx;
} gesmc_pool_opts;

typedef struct gesmc_chain_info_s {
  uint64_t m, n;           /* edges; node bound                               */
  uint64_t seed;
  uint64_t rounds;         /* rounds run since the chain was added            */
  uint64_t next_round;     /* number of the chain's next round                */
  uint64_t switches;       /* floor(m/2) per round run                        */
  uint64_t accepted;       /* switches that rewired (since added), both chains */
  uint64_t es_switches;    /* ES-MC switches run (gesmc_pool_es_run)          */
} gesmc_chain_info_t;

void gesmc_pool_opts_default(gesmc_pool_opts *o);
size_t gesmc_pool_device_bytes(uint64_t max_edges, uint32_t max_chains, uint32_t tuple_log2);
int gesmc_pool_create(const gesmc_pool_opts *opts, gesmc_pool_t *out);
void gesmc_pool_destroy(gesmc_pool_t p);

/* Add a chain (a simple graph, validated as in gesmc_create; host or device
 * memory, copied).  Its first round is numbered start_round; flags is 0 or
 * GESMC_CHAIN_EXACT_ELL (laziness as GESMC_FLAG_EXACT_ELL describes);
 * *chain_out receives its id (ids of removed chains are reused). */
#define GESMC_CHAIN_EXACT_ELL 1u
int gesmc_pool_add(gesmc_pool_t p, const uint64_t *edges, uint64_t m, int edges_on_device, uint64_t n,
                   uint64_t seed, uint64_t start_round, uint64_t lazy_threshold, uint32_t flags,
                   uint32_t *chain_out);
/* Remove a chain (its result should be read first with gesmc_pool_edges). */
int gesmc_pool_remove(gesmc_pool_t p, uint32_t chain);
/* Advance every chain of the pool by `global_switches` rounds. */
int gesmc_pool_run(gesmc_pool_t p, uint64_t global_switches);
/* Advance every chain of the pool by `switches` ES-MC switches (as
 * gesmc_es_run, each chain with its own seed). */
int gesmc_pool_es_run(gesmc_pool_t p, uint64_t switches);
/* Copy a chain's edge list, in position order, as gesmc_edges does. */
int gesmc_pool_edges(gesmc_pool_t p, uint32_t chain, uint64_t *out, uint64_t capacity, int out_on_device,
                     uint64_t *m_out);
int gesmc_pool_chain_info(gesmc_pool_t p, uint32_t chain, gesmc_chain_info_t *out);
uint32_t gesmc_pool_num_chains(gesmc_pool_t p);
uint64_t gesmc_pool_free_edges(gesmc_pool_t p);
/* Debug check of one chain of the pool, as gesmc_verify. */
int gesmc_pool_verify(gesmc_pool_t p, uint32_t chain);
/* Round launch of the pool, as gesmc_set_round_launch. */
int gesmc_pool_set_round_launch(gesmc_pool_t p, uint32_t ctas, uint32_t *effective);
/* Counters over all chains, stage timing: as for single chains. */
int gesmc_pool_stats(gesmc_pool_t p, gesmc_stats_t *out);
int gesmc_pool_reset_stats(gesmc_pool_t p);
int gesmc_pool_set_profiling(gesmc_pool_t p, int enable);
int gesmc_pool_stage_times(gesmc_pool_t p, double *ms, int n_stages, uint64_t *rounds);

/* Static description of an error code. */
const char *gesmc_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GESMC_H */
