// Resident rounds: every global switch of a small chain run by one CTA with
// the chain's list in shared memory, for all rounds of a call (one launch
// per call, not per round or per stage).  Declarations shared by
// resident.cu and api.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gesmc_internal.cuh"

namespace gesmc {

// A chain runs resident if it has at most kResidentMaxEdges edges and node
// ids below kResidentMaxNodes (an edge then packs into 32 bits: two 16-bit
// node ids; positions and switch indices fit 16 bits).
constexpr uint32_t kResidentMaxEdges = 10240;
constexpr uint64_t kResidentMaxNodes = 1ull << 16;
// Chains run in classes by size, each with its own CTA size: 1024 threads
// for more than 4096 edges, 512 up to 4096, 256 up to 2048, 128 up to 1024
// (a small chain's CTA leaves room on its SM for others).
constexpr uint32_t kResidentClasses = 4;
uint32_t resident_class(uint32_t m);
// Rounds per launch are bounded by the scratch words that collect each
// round's wave count (the target filter's bytes, unused by resident rounds).
constexpr uint32_t kResidentMaxRoundsPerLaunch = 4096;

// Dynamic shared memory of a CTA whose chain has m edges (grows with m).
size_t resident_smem_bytes(uint32_t m);
// Opt in to the shared memory of the largest resident chain (once per device).
cudaError_t prepare_resident();

// The chains in jobs (each with 2 <= m <= kResidentMaxEdges, ids <
// kResidentMaxNodes), grouped by class (count[c] chains of class c, class 0
// first; max_m[c] the largest m among them, which sizes the shared memory),
// run `rounds` rounds from the pool's current round, one CTA each (one
// launch per class), then a one-CTA kernel folds the rounds' wave counts
// into the statistics and advances the pool round.  round_waves (rounds
// words) and last_pending (kWaveHist words) must be zero; `final` says
// whether the call's last round is in this launch (its per-wave undecided
// counts become the statistics' last-round counts).  pbuf (optional): room
// for rounds x jobs permutations of pstride u16 each (pstride >= the largest
// m, a multiple of 8), ebuf for rounds x jobs words; then each class's
// permutations are sorted first by a kernel of one CTA per (chain, round) on
// the other SMs, and the chains' CTAs read them instead of sorting.
// *launches is increased by the number of kernels launched.
cudaError_t launch_round_resident(const RoundArgs &a, const uint32_t *jobs, const uint32_t (&count)[kResidentClasses],
                                  const uint32_t (&max_m)[kResidentClasses], uint32_t rounds, uint32_t *round_waves,
                                  uint32_t *last_pending, bool final, uint16_t *pbuf, uint32_t *ebuf, uint32_t pstride,
                                  cudaStream_t s, uint32_t *launches);

}  // namespace gesmc
