/* Seeded synthetic inputs: simple graphs shaped like the SynGnp and SynPld
 * families of arXiv 2111.03005 (Sec. 6, dataset list).  This file holds no
 * arithmetic of the edge-switching method; it only makes starting graphs,
 * which the CUDA library and the CPU oracle then both receive unchanged.
 *
 * Randomness: splitmix64 (Steele, Lea, Flood 2014), seeded per call.
 * Edges are returned packed as (min << 32) | max.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t sm64_next(uint64_t *s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* uniform double in (0, 1] */
static double sm64_unit(uint64_t *s) { return ((double)(sm64_next(s) >> 11) + 1.0) * (1.0 / 9007199254740992.0); }

static uint64_t pack_edge(uint32_t a, uint32_t b) {
  uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
  return ((uint64_t)lo << 32) | hi;
}

/* G(n, p) (Gilbert): every pair {w, v}, w < v, independently with
 * probability p, by geometric skipping over the pairs in the order
 * (v = 1, w = 0), (v = 2, w = 0..1), ... (Batagelj and Brandes 2005).
 * Writes at most `cap` edges; returns the number of edges the graph has
 * (which may exceed cap: call again with a larger buffer). */
uint64_t gen_gnp(uint32_t n, double p, uint64_t seed, uint64_t *out, uint64_t cap) {
  uint64_t s = seed, m = 0;
  if (n < 2 || p <= 0.0) return 0;
  if (p >= 1.0) {
    for (uint64_t v = 1; v < n; ++v)
      for (uint64_t w = 0; w < v; ++w) {
        if (m < cap) out[m] = pack_edge((uint32_t)w, (uint32_t)v);
        ++m;
      }
    return m;
  }
  const double lq = log1p(-p);
  int64_t v = 1, w = -1;
  while (v < (int64_t)n) {
    double r = sm64_unit(&s);
    w += 1 + (int64_t)floor(log(r) / lq);
    while (w >= v && v < (int64_t)n) {
      w -= v;
      ++v;
    }
    if (v < (int64_t)n) {
      if (m < cap) out[m] = pack_edge((uint32_t)w, (uint32_t)v);
      ++m;
    }
  }
  return m;
}

/* n i.i.d. draws from Pld([a..b], gamma): P(X = k) proportional to k^-gamma
 * for a <= k <= b (Sec. 2.1), by inverse transform over a table of the
 * cumulative weights. */
int gen_pld_degrees(uint32_t n, uint32_t a, uint32_t b, double gamma, uint64_t seed, uint32_t *deg) {
  if (a < 1 || b < a) return -1;
  uint32_t span = b - a + 1;
  double *cdf = (double *)malloc(sizeof(double) * span);
  if (!cdf) return -2;
  double acc = 0.0;
  for (uint32_t t = 0; t < span; ++t) {
    acc += pow((double)(a + t), -gamma);
    cdf[t] = acc;
  }
  uint64_t s = seed;
  for (uint32_t i = 0; i < n; ++i) {
    double u = sm64_unit(&s) * acc;
    uint32_t lo = 0, hi = span - 1;
    while (lo < hi) {
      uint32_t mid = lo + (hi - lo) / 2;
      if (cdf[mid] < u) lo = mid + 1;
      else hi = mid;
    }
    deg[i] = a + lo;
  }
  free(cdf);
  return 0;
}

static int cmp_desc_u32(const void *x, const void *y) {
  uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
  return a < b ? 1 : (a > b ? -1 : 0);
}

/* Erdos-Gallai test: 1 if the sequence is graphical, else 0 (-2: no memory). */
int gen_is_graphical(const uint32_t *deg, uint32_t n) {
  uint32_t *d = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  uint64_t *suffix = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
  if (!d || !suffix) {
    free(d); free(suffix);
    return -2;
  }
  memcpy(d, deg, sizeof(uint32_t) * n);
  qsort(d, n, sizeof(uint32_t), cmp_desc_u32);
  suffix[n] = 0;
  for (int64_t i = (int64_t)n - 1; i >= 0; --i) suffix[i] = suffix[i + 1] + d[i];
  int ok = (suffix[0] & 1) == 0;
  uint64_t lhs = 0;
  for (uint32_t k = 1; k <= n && ok; ++k) {
    lhs += d[k - 1];
    /* sum over i >= k (0-based) of min(d_i, k): entries above k give k each */
    uint32_t lo = k, hi = n;
    while (lo < hi) {
      uint32_t mid = lo + (hi - lo) / 2;
      if (d[mid] <= k) hi = mid;
      else lo = mid + 1;
    }
    uint64_t rhs = (uint64_t)k * (k - 1) + (uint64_t)k * (lo - k) + suffix[lo];
    if (lhs > rhs) ok = 0;
  }
  free(suffix);
  free(d);
  return ok;
}

/* Havel-Hakimi realisation.  Nodes sit in one stack per residual degree
 * (filled in ascending id order).  Each step pops a node u from the highest
 * non-empty stack and joins it to the d(u) other nodes of largest residual
 * degree, taken from the tops of the stacks from the highest down; those
 * nodes are then pushed, in the order taken, onto the stack one below.  Any
 * tie order realises a graphical sequence; this one is deterministic.
 * Returns the number of edges written to `out` (which must hold sum(deg)/2),
 * -1 if the sequence is not graphical, -2 on allocation failure. */
int64_t gen_havel_hakimi(const uint32_t *deg, uint32_t n, uint64_t *out) {
  uint64_t total = 0;
  uint32_t dmax = 0;
  for (uint32_t i = 0; i < n; ++i) {
    total += deg[i];
    if (deg[i] > dmax) dmax = deg[i];
  }
  if (total & 1) return -1;
  if (n > 0 && dmax >= n) return -1;
  /* linked stacks: top[r] is the top node of stack r, next[v] the node below v */
  uint32_t *next = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1)); /* next below in its stack */
  uint32_t *top = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)dmax + 1));
  uint64_t *size = (uint64_t *)calloc((size_t)dmax + 1, sizeof(uint64_t));
  uint32_t *res = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  uint32_t *taken = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)dmax + 1));
  if (!next || !top || !size || !res || !taken) {
    free(next); free(top); free(size); free(res); free(taken);
    return -2;
  }
  const uint32_t NIL = 0xFFFFFFFFu;
  for (uint32_t r = 0; r <= dmax; ++r) top[r] = NIL;
  for (uint32_t i = 0; i < n; ++i) {
    res[i] = deg[i];
    if (deg[i] == 0) continue;
    next[i] = top[deg[i]];
    top[deg[i]] = i;
    size[deg[i]]++;
  }
  int64_t m = 0;
  uint32_t hi = dmax;
  for (;;) {
    while (hi > 0 && top[hi] == NIL) --hi;
    if (hi == 0) break;
    uint32_t u = top[hi];
    top[hi] = next[u];
    size[hi]--;
    uint32_t d = res[u];
    res[u] = 0;
    uint32_t got = 0;
    for (uint32_t r = hi; r > 0 && got < d; --r) {
      while (top[r] != NIL && got < d) {
        uint32_t v = top[r];
        top[r] = next[v];
        size[r]--;
        taken[got++] = v;
      }
    }
    if (got < d) { m = -1; break; }
    for (uint32_t t = 0; t < d; ++t) {
      uint32_t v = taken[t];
      out[m++] = pack_edge(u, v);
      uint32_t r = --res[v];
      if (r > 0) {
        next[v] = top[r];
        top[r] = v;
        size[r]++;
      }
    }
  }
  free(next); free(top); free(size); free(res); free(taken);
  return m;
}
