/*
 * gesmc_gen.h -- on-GPU input generator of libgesmc: G(n, p) starting graphs
 * (the SynGnp inputs of arXiv 2111.03005, Sec. 6) written straight into
 * device memory, so that large chains need no host-side generation or
 * host-to-device copy.  Not part of the chain API; inputs only.
 */
#ifndef GESMC_GEN_H
#define GESMC_GEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* G(n, p): every pair {u, v}, u < v < n, is an edge independently with
 * probability p.  The pairs are numbered row by row (u ascending, then v) and
 * cut into chunks of ceil(128 / p) pairs; chunk c walks its pairs with
 * geometric skips (Batagelj and Brandes, Phys. Rev. E 71, 2005): from pair t
 * the next edge is pair t + 1 + floor(log(1 - U) / log(1 - p)), U uniform in
 * [0, 1) from the 53 top bits of Philox4x64-10 words (counter = (c, d >> 2,
 * 3, 0), key = (seed, 0), word d & 3 for the chunk's d-th draw).  Edges are
 * written canonically (u << 32 | v) in pair order.
 *
 *   n:        nodes, 2 <= n <= 2^31.
 *   p:        0 <= p <= 1.
 *   out:      device memory of `capacity` uint64 entries (may be NULL with
 *             capacity 0 to ask for the count).
 *   *m_out:   the number of edges (written even if they do not fit).
 *   stream:   cudaStream_t for the work, or NULL; the call synchronises it.
 * Returns 0, -1 (bad argument), -5 (capacity too small: *m_out says how
 * many), -6 (CUDA error).  Scratch: 8 bytes per chunk, allocated and freed
 * by the call (cudaMallocAsync on the stream). */
int gesmc_generate_gnp(uint64_t n, double p, uint64_t seed, uint64_t *out, uint64_t capacity, uint64_t *m_out,
                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GESMC_GEN_H */
