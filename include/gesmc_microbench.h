/*
 * gesmc_microbench.h -- device random-access ceiling, the denominator of the
 * random-access roofline of libgesmc's global switch round (arXiv
 * 2111.03005, Sec. 5.4 notes that edge switching is bound by unstructured
 * memory accesses).  Not part of the chain API.
 */
#ifndef GESMC_MICROBENCH_H
#define GESMC_MICROBENCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Time `accesses` uniformly random 8-byte accesses of one kind over a
 * freshly allocated device buffer of `bytes` bytes on the current device:
 * kind 0 = loads, 1 = stores, 2 = 64-bit atomicCAS, 3 = 32-bit atomicAdd with
 * its result used (a cursor), 4 = the same without result (a count).  With a
 * small buffer (a few MB) kinds 3 and 4 measure the L2 atomic rate that
 * bucket cursors and histograms see.  Best of three timed
 * repetitions (after one warm-up), each after a refill of the buffer.
 * Writes accesses per second to *accesses_per_s.  Allocates and frees the
 * buffer itself (cudaMalloc).  Returns 0, -1 (bad argument), -5 (allocation
 * failed) or -6 (CUDA error). */
int gesmc_probe_random_access(uint64_t bytes, int kind, uint64_t accesses, double *accesses_per_s);

#ifdef __cplusplus
}
#endif

#endif /* GESMC_MICROBENCH_H */
