// ORACLE -- test infrastructure only, never part of the product path.
//
// A plain, slow, sequential CPU statement of the Global Edge Switching Markov
// Chain (G-ES-MC) of Allendorf, Meyer, Penschuck and Tran, "Parallel Global
// Edge Switching for the Uniform Sampling of Simple Graphs with Prescribed
// Degrees" (arXiv 2111.03005).  Only tests/, __graft_entry__.smoke() and the
// cpu_baseline / reference leg of bench.py may load it.  It shares no source,
// header, table or helper with the CUDA library; both sides only agree on the
// published definitions restated below.
//
// What it computes, in the paper's order:
//   * Def. 1 (Sec. 2.2): an edge switch sigma = (i, j, g) on the indexed edge
//     list E: e1 = E[i] = (u, v), e2 = E[j] = (x, y); tau gives
//     g = 0 -> (u, x), (v, y) and g = 1 -> (u, y), (v, x).  The switch is
//     rejected if a new edge is a loop or is already in E, else
//     E[i] <- e3, E[j] <- e4.
//   * Def. 2 (Sec. 3): a global switch runs the switches
//     sigma_k = (pi(2k-1), pi(2k), 1[pi(2k-1) < pi(2k)]) one after another
//     (1-based in the paper; 0-based here: pi[2k], pi[2k+1]).
//   * Algorithm 3 (ParGlobalES): one global switch per round, r rounds.
//   * ES-MC (Def. 1's chain, the one Algorithm 2, ParES, parallelises): r
//     independent switches sigma_k = (i, j, g), i != j uniform in [m] and g
//     a fair bit, one after another.
//
// Readings where the paper leaves a choice open:
//   * Edges are stored canonically, (min << 32) | max (Sec. 5.2 edge ids;
//     Sec. 2.1 canonical orientation), also right after every accepted switch.
//   * The random permutation pi of round r is the argsort of 64-bit keys
//     K(i) = Philox4x64-10(counter = (i >> 2, r, 0, 0), key = (seed, 0))[i & 3]
//     with ties broken by the smaller position.  Philox4x64-10 is the
//     counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11).
//   * Laziness (Def. 2, P_L): switch k of round r is skipped iff
//     Philox4x64-10(counter = (k >> 2, r, 1, 0), key = (seed, 0))[k & 3]
//     < lazy_threshold; the default threshold 0 never skips (P_L = 0).
//   * Exact l (Def. 2 as printed, optional): the global switch draws
//     l ~ Binom(floor(m/2), 1 - P_L) and runs its first l switches only.
//     l is the number of k < floor(m/2) whose laziness word is
//     >= lazy_threshold (floor(m/2) independent trials, each passing with
//     probability 1 - P_L), so both implementations draw the same l.
//   * Rounds are numbered cumulatively, so run(a) then run(b) equals run(a+b).
//   * ES-MC switch k draws Philox4x64-10(counter = (k, 0, 2, 0),
//     key = (seed, 0)) = (w0, w1, w2, w3): i = floor(w0 * m / 2^64),
//     j = j' + [j' >= i] with j' = floor(w1 * (m - 1) / 2^64) (uniform over
//     [m] minus i), g = the top bit of w2.  Switches are numbered
//     cumulatively like rounds.  With m < 2 no switch exists; each requested
//     switch is counted as skipped.
//
// Parity pins live in tests/test_oracle_pins.py (worked example of Fig. 1,
// hand-worked global switches, special graphs, exact transition matrices
// against Thm. 1, chi-squared uniformity over brute-forced G(d), Philox
// against numpy's independent Philox implementation).

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

// ---- Philox4x64-10 (Salmon et al., SC'11, Sec. 3 and Table 2) --------------
// One round: two 64x64->128 multiplications of counter words 0 and 2 by fixed
// multipliers; the high halves are xor-ed with the other counter words and
// the round key, and the words are permuted.  The key is bumped by two Weyl
// constants between rounds.
const uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
const uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
const uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;
const uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;

void philox4x64_10(const uint64_t in_ctr[4], const uint64_t in_key[2], uint64_t out[4]) {
  uint64_t c[4] = {in_ctr[0], in_ctr[1], in_ctr[2], in_ctr[3]};
  uint64_t k0 = in_key[0], k1 = in_key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    unsigned __int128 p0 = (unsigned __int128)kPhiloxM0 * c[0];
    unsigned __int128 p1 = (unsigned __int128)kPhiloxM1 * c[2];
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t n0 = hi1 ^ c[1] ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c[3] ^ k1;
    uint64_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

uint64_t philox_word(uint64_t seed, uint64_t round, uint64_t purpose, uint64_t index) {
  const uint64_t ctr[4] = {index >> 2, round, purpose, 0};
  const uint64_t key[2] = {seed, 0};
  uint64_t out[4];
  philox4x64_10(ctr, key, out);
  return out[index & 3];
}

const uint64_t kPurposePermutation = 0;
const uint64_t kPurposeLazy = 1;
const uint64_t kPurposeEsSwitch = 2;

// ES-MC switch k: (i, j, g) from one Philox block, as stated in the header.
void es_sample(uint64_t seed, uint64_t k, uint64_t m, uint64_t* i, uint64_t* j, int* g) {
  const uint64_t ctr[4] = {k, 0, kPurposeEsSwitch, 0};
  const uint64_t key[2] = {seed, 0};
  uint64_t w[4];
  philox4x64_10(ctr, key, w);
  *i = (uint64_t)(((unsigned __int128)w[0] * m) >> 64);
  const uint64_t jj = (uint64_t)(((unsigned __int128)w[1] * (m - 1)) >> 64);
  *j = jj + (jj >= *i ? 1 : 0);
  *g = (int)(w[2] >> 63);
}

inline uint64_t pack(uint32_t a, uint32_t b) {
  // canonical id of the undirected edge {a, b}: smaller node in the high half
  uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
  return ((uint64_t)lo << 32) | hi;
}

// Outcome codes of one edge switch.
const int kAccepted = 0;
const int kRejectedLoop = 1;
const int kRejectedExists = 2;

// Def. 1 applied to E (positions i, j, direction bit g) against the current
// edge set S, which always equals the set of entries of E.
int edge_switch(uint64_t* E, std::unordered_set<uint64_t>& S, uint64_t i, uint64_t j, int g) {
  const uint64_t e1 = E[i], e2 = E[j];
  const uint32_t u = (uint32_t)(e1 >> 32), v = (uint32_t)e1;
  const uint32_t x = (uint32_t)(e2 >> 32), y = (uint32_t)e2;
  uint32_t a3, b3, a4, b4;  // e3 = (a3, b3), e4 = (a4, b4) as tau orients them
  if (g == 0) { a3 = u; b3 = x; a4 = v; b4 = y; }
  else        { a3 = u; b3 = y; a4 = v; b4 = x; }
  if (a3 == b3 || a4 == b4) return kRejectedLoop;
  const uint64_t e3 = pack(a3, b3), e4 = pack(a4, b4);
  if (S.count(e3) || S.count(e4)) return kRejectedExists;
  S.erase(e1);
  S.erase(e2);
  S.insert(e3);
  S.insert(e4);
  E[i] = e3;
  E[j] = e4;
  return kAccepted;
}

}  // namespace

extern "C" {

// Statistics of a call, summed over all switches it ran.
struct orc_stats {
  uint64_t switches;         // floor(m/2) per round: every pair of the permutation
  uint64_t lazy;             // switches skipped by the laziness rule
  uint64_t accepted;
  uint64_t rejected_loop;    // a new edge would be a loop
  uint64_t rejected_exists;  // a new edge is already in E when the switch runs
};

// Error codes of the oracle's own input check.
enum { ORC_OK = 0, ORC_E_INVALID = -1, ORC_E_LOOP = -2, ORC_E_MULTI = -3, ORC_E_RANGE = -4,
       ORC_E_INVARIANT = -20 };

void orc_philox4x64_10(const uint64_t* ctr, const uint64_t* key, uint64_t* out) {
  philox4x64_10(ctr, key, out);
}

uint64_t orc_perm_key(uint64_t seed, uint64_t round, uint64_t i) {
  return philox_word(seed, round, kPurposePermutation, i);
}

uint64_t orc_lazy_word(uint64_t seed, uint64_t round, uint64_t k) {
  return philox_word(seed, round, kPurposeLazy, k);
}

// pi of round r: positions 0..m-1 sorted by (K(i), i).
void orc_permutation(uint64_t seed, uint64_t round, uint64_t m, uint32_t* pi) {
  std::vector<std::pair<uint64_t, uint32_t>> keyed(m);
  for (uint64_t i = 0; i < m; ++i) keyed[i] = {orc_perm_key(seed, round, i), (uint32_t)i};
  std::sort(keyed.begin(), keyed.end());
  for (uint64_t s = 0; s < m; ++s) pi[s] = keyed[s].second;
}

// A "degree-valid" edge list is a simple graph on nodes [0, n): no loops, no
// repeated edge, ids < n (Sec. 2.1).  n == 0 means "no bound".  The list is
// canonicalised in place.  When several kinds of fault occur the code for a
// loop wins over an out-of-range id, which wins over a repeated edge.
int orc_validate(uint64_t* E, uint64_t m, uint64_t n) {
  if (E == nullptr && m > 0) return ORC_E_INVALID;
  if (m >= (1ull << 32)) return ORC_E_INVALID;
  bool loop = false, range = false, multi = false;
  std::unordered_set<uint64_t> seen;
  seen.reserve(m * 2 + 1);
  for (uint64_t i = 0; i < m; ++i) {
    const uint32_t a = (uint32_t)(E[i] >> 32), b = (uint32_t)E[i];
    if (a == b) loop = true;
    if (n != 0 && (a >= n || b >= n)) range = true;
    E[i] = pack(a, b);
    if (a != b && !seen.insert(E[i]).second) multi = true;
  }
  if (loop) return ORC_E_LOOP;
  if (range) return ORC_E_RANGE;
  if (multi) return ORC_E_MULTI;
  return ORC_OK;
}

// One edge switch (Def. 1) on a canonical simple edge list; the edge set is
// taken from E.  Returns 0 accepted, 1 rejected (loop), 2 rejected (exists).
int orc_edge_switch(uint64_t* E, uint64_t m, uint64_t i, uint64_t j, int g) {
  std::unordered_set<uint64_t> S(E, E + m);
  return edge_switch(E, S, i, j, g);
}

namespace {

bool degrees_and_set_ok(const uint64_t* E, uint64_t m, const std::unordered_set<uint64_t>& S,
                        const std::unordered_map<uint32_t, uint64_t>& deg0) {
  if (S.size() != m) return false;
  std::unordered_map<uint32_t, uint64_t> deg;
  for (uint64_t i = 0; i < m; ++i) {
    const uint32_t a = (uint32_t)(E[i] >> 32), b = (uint32_t)E[i];
    if (a >= b) return false;  // canonical and loop-free
    if (!S.count(E[i])) return false;
    ++deg[a];
    ++deg[b];
  }
  return deg == deg0;
}

std::unordered_map<uint32_t, uint64_t> degree_map(const uint64_t* E, uint64_t m) {
  std::unordered_map<uint32_t, uint64_t> deg;
  for (uint64_t i = 0; i < m; ++i) {
    ++deg[(uint32_t)(E[i] >> 32)];
    ++deg[(uint32_t)E[i]];
  }
  return deg;
}

void count(orc_stats* st, int outcome) {
  if (!st) return;
  if (outcome == kAccepted) ++st->accepted;
  else if (outcome == kRejectedLoop) ++st->rejected_loop;
  else ++st->rejected_exists;
}

}  // namespace

// One global switch (Def. 2) with an explicit permutation pi of [0, m): the
// first ell pairs run in order; skip[k] != 0 (if skip is given) skips pair k.
int orc_global_switch(uint64_t* E, uint64_t m, const uint32_t* pi, uint64_t ell,
                      const uint8_t* skip, orc_stats* st) {
  if (ell > m / 2) return ORC_E_INVALID;
  std::unordered_set<uint64_t> S(E, E + m);
  for (uint64_t k = 0; k < ell; ++k) {
    if (st) ++st->switches;
    if (skip && skip[k]) {
      if (st) ++st->lazy;
      continue;
    }
    const uint64_t i = pi[2 * k], j = pi[2 * k + 1];
    const int g = i < j ? 1 : 0;
    count(st, edge_switch(E, S, i, j, g));
  }
  return ORC_OK;
}

// Algorithm 3 run sequentially: `rounds` global switches numbered
// start_round, start_round + 1, ...  E must be a canonical simple edge list.
// If snapshots is given it receives E after every round (rounds * m words).
// check_every_switch re-verifies simplicity, |E| = m and the degree sequence
// after every single switch (slow; for small graphs).
int orc_run(uint64_t* E, uint64_t m, uint64_t seed, uint64_t start_round, uint64_t rounds,
            uint64_t lazy_threshold, int exact_ell, int check_every_switch, orc_stats* st, uint64_t* snapshots) {
  if (E == nullptr && m > 0) return ORC_E_INVALID;
  std::unordered_set<uint64_t> S;
  S.reserve(m * 2 + 1);
  for (uint64_t i = 0; i < m; ++i) S.insert(E[i]);
  if (S.size() != m) return ORC_E_MULTI;
  std::unordered_map<uint32_t, uint64_t> deg0;
  if (check_every_switch) deg0 = degree_map(E, m);
  std::vector<uint32_t> pi(m);
  const uint64_t L = m / 2;
  for (uint64_t t = 0; t < rounds; ++t) {
    const uint64_t r = start_round + t;
    orc_permutation(seed, r, m, pi.data());
    uint64_t ell = L;  // exact l: the number of trials that pass
    if (exact_ell && lazy_threshold != 0) {
      ell = 0;
      for (uint64_t k = 0; k < L; ++k) ell += orc_lazy_word(seed, r, k) >= lazy_threshold ? 1 : 0;
    }
    for (uint64_t k = 0; k < L; ++k) {
      if (st) ++st->switches;
      const bool skipped = exact_ell ? k >= ell
                                     : lazy_threshold != 0 && orc_lazy_word(seed, r, k) < lazy_threshold;
      if (skipped) {
        if (st) ++st->lazy;
        continue;
      }
      const uint64_t i = pi[2 * k], j = pi[2 * k + 1];
      const int g = i < j ? 1 : 0;
      count(st, edge_switch(E, S, i, j, g));
      if (check_every_switch && !degrees_and_set_ok(E, m, S, deg0)) return ORC_E_INVARIANT;
    }
    if (snapshots) std::memcpy(snapshots + t * m, E, m * sizeof(uint64_t));
  }
  return ORC_OK;
}

// ---- Algorithm 1 (ParallelSuperstep) with its rounds in Jacobi order --------
//
// Sec. 4 performs a superstep in rounds of decide / delay.  Taken in Jacobi
// order, every switch still undecided when round w starts is decided from the
// statuses known when round w - 1 ended, and round w's decisions all take
// effect at its closing barrier; Thm. 2's "worst-case scheduler" is this
// order, and it makes the number of rounds a function of the superstep alone.
//
// Per switch k with sources e1 = E[i], e2 = E[j] and targets tau(e1, e2, g):
// T holds (e1, k, ERASE), (e2, k, ERASE), (e3, k, INSERT), (e4, k, INSERT),
// plus the implicit (e, inf, ERASE, ILLEGAL) for every e in E that no switch
// erases.  Reading (where Algorithm 1 as printed and Def. 1 part): a switch
// that Def. 1 rejects without looking at E -- a target is a loop, or the
// sources share a node (then its targets re-create its sources) -- and a
// switch the laziness rule skips are stored in T with status ILLEGAL, i.e.
// known to fail before the first round; they leave U in round 1.
//
// A target e of an undecided switch k, with p = the switch that erases e (if
// any tuple erases it) and q = the smallest switch inserting e whose status
// is not ILLEGAL, makes k
//   ILLEGAL   if k < p or s_p = ILLEGAL (e is still in E when k runs), or
//             if q < k and s_q = LEGAL (an earlier switch inserted e);
//   UNDECIDED otherwise if p < k and s_p = UNDECIDED, or q < k and
//             s_q = UNDECIDED (delay to the next round);
// and k is ILLEGAL if either target says so, else UNDECIDED if either says
// so, else LEGAL (E[i] <- e3, E[j] <- e4).
namespace {

enum { kSUndecided = 0, kSLegal = 1, kSIllegal = 2 };
const uint64_t kInf = ~0ull;

// One superstep: switches k < L over pi's pairs; skip[k] != 0 marks a skipped
// (lazy) switch.  Rewires E in place; returns the number of rounds and, if
// entering is given, the undecided switches entering round w at entering[w]
// (w < max_w; entering[0] is left alone).  Returns 0 rounds for L == 0.
uint64_t superstep_jacobi(uint64_t* E, uint64_t m, const uint32_t* pi, uint64_t L,
                          const std::vector<uint8_t>& skip, uint64_t* entering, uint64_t max_w) {
  struct Sw {
    uint64_t i, j, e3, e4;
  };
  std::vector<Sw> sw(L);
  std::vector<int> status(L, kSUndecided);
  std::vector<uint8_t> known(L, 0);  // stored ILLEGAL (Def. 1 rejects it outright, or it is skipped)
  std::unordered_map<uint64_t, uint64_t> eraser;                 // e -> p
  std::unordered_map<uint64_t, std::vector<uint64_t>> inserters;  // e -> every k inserting e, ascending
  const std::unordered_set<uint64_t> in_E(E, E + m);  // the edge set when the superstep starts
  for (uint64_t k = 0; k < L; ++k) {
    const uint64_t i = pi[2 * k], j = pi[2 * k + 1];
    const int g = i < j ? 1 : 0;
    const uint64_t e1 = E[i], e2 = E[j];
    const uint32_t u = (uint32_t)(e1 >> 32), v = (uint32_t)e1;
    const uint32_t x = (uint32_t)(e2 >> 32), y = (uint32_t)e2;
    const uint32_t a3 = u, b3 = g ? y : x, a4 = v, b4 = g ? x : y;
    sw[k] = {i, j, pack(a3, b3), pack(a4, b4)};
    const bool loop = a3 == b3 || a4 == b4;
    const bool shared = u == x || u == y || v == x || v == y;
    if (skip[k] || loop || shared) {
      known[k] = 1;
      status[k] = kSIllegal;
    }
    eraser[e1] = k;  // Obs. 2: a superstep erases each edge at most once
    eraser[e2] = k;
    if (!known[k]) {
      inserters[sw[k].e3].push_back(k);
      inserters[sw[k].e4].push_back(k);
    }
  }
  std::vector<uint64_t> U;
  for (uint64_t k = 0; k < L; ++k) U.push_back(k);
  uint64_t rounds = 0;
  std::vector<int> prev;
  while (!U.empty()) {
    ++rounds;
    if (entering && rounds < max_w) entering[rounds] = U.size();
    prev = status;  // statuses as the last round's barrier left them
    std::vector<uint64_t> D;
    std::vector<std::pair<uint64_t, int>> decided;
    for (uint64_t k : U) {
      if (known[k]) {
        decided.push_back({k, kSIllegal});
        continue;
      }
      int s = kSLegal;
      for (int t = 0; t < 2; ++t) {
        const uint64_t e = t ? sw[k].e4 : sw[k].e3;
        // lookup(e, ERASE): the tuple of the switch that erases e, else the
        // implicit ILLEGAL tuple at infinity if e is in E, else none
        bool has_p = false;
        uint64_t p = 0;
        int sp = kSUndecided;
        auto it = eraser.find(e);
        if (it != eraser.end()) {
          has_p = true;
          p = it->second;
          sp = prev[p];
        } else if (in_E.count(e)) {
          has_p = true;
          p = kInf;
          sp = kSIllegal;
        }
        // lookup_min(e, INSERT): smallest inserter whose status is not ILLEGAL
        bool has_q = false;
        uint64_t q = 0;
        for (uint64_t c : inserters[e]) {
          if (prev[c] != kSIllegal) {
            has_q = true;
            q = c;
            break;
          }
        }
        if (has_p && (k < p || sp == kSIllegal)) s = kSIllegal;
        if (has_q && k > q && prev[q] == kSLegal) s = kSIllegal;
        if (s != kSIllegal) {
          if (has_p && k > p && sp == kSUndecided) s = kSUndecided;
          if (has_q && k > q && prev[q] == kSUndecided) s = kSUndecided;
        }
      }
      if (s == kSUndecided) D.push_back(k);
      else decided.push_back({k, s});
    }
    if (decided.empty()) return ~0ull;  // no progress: impossible for a valid superstep
    for (const auto& d : decided) {
      status[d.first] = d.second;
      if (d.second == kSLegal) {
        E[sw[d.first].i] = sw[d.first].e3;
        E[sw[d.first].j] = sw[d.first].e4;
      }
    }
    U.swap(D);
  }
  return rounds;
}

}  // namespace

// Algorithm 3 with each global switch performed by superstep_jacobi above:
// the same rounds, seed and laziness as orc_run (so the same list results),
// plus the number of decide / delay rounds of every global switch in
// rounds_out[t] and, if entering_out is given, the undecided switches entering
// round w of global switch t at entering_out[t * max_w + w].
int orc_run_rounds(uint64_t* E, uint64_t m, uint64_t seed, uint64_t start_round, uint64_t rounds,
                   uint64_t lazy_threshold, int exact_ell, uint64_t* rounds_out, uint64_t* entering_out,
                   uint64_t max_w) {
  if (E == nullptr && m > 0) return ORC_E_INVALID;
  std::vector<uint32_t> pi(m);
  const uint64_t L = m / 2;
  std::vector<uint8_t> skip(L);
  for (uint64_t t = 0; t < rounds; ++t) {
    const uint64_t r = start_round + t;
    orc_permutation(seed, r, m, pi.data());
    uint64_t ell = L;
    if (exact_ell && lazy_threshold != 0) {
      ell = 0;
      for (uint64_t k = 0; k < L; ++k) ell += orc_lazy_word(seed, r, k) >= lazy_threshold ? 1 : 0;
    }
    for (uint64_t k = 0; k < L; ++k)
      skip[k] = exact_ell ? (k >= ell) : (lazy_threshold != 0 && orc_lazy_word(seed, r, k) < lazy_threshold);
    const uint64_t w = superstep_jacobi(E, m, pi.data(), L, skip,
                                        entering_out ? entering_out + t * max_w : nullptr, max_w);
    if (w == ~0ull) return ORC_E_INVARIANT;
    if (rounds_out) rounds_out[t] = w;
  }
  return ORC_OK;
}

// The same for one global switch with an explicit permutation (as
// orc_global_switch: the first ell pairs, skip[k] != 0 skips pair k).
int orc_global_switch_rounds(uint64_t* E, uint64_t m, const uint32_t* pi, uint64_t ell, const uint8_t* skip,
                             uint64_t* rounds_out, uint64_t* entering_out, uint64_t max_w) {
  if (ell > m / 2) return ORC_E_INVALID;
  std::vector<uint8_t> sk(ell, 0);
  for (uint64_t k = 0; k < ell && skip; ++k) sk[k] = skip[k] ? 1 : 0;
  const uint64_t w = superstep_jacobi(E, m, pi, ell, sk, entering_out, max_w);
  if (w == ~0ull) return ORC_E_INVARIANT;
  if (rounds_out) *rounds_out = w;
  return ORC_OK;
}

// ES-MC switch k of a list of m >= 2 edges: out = {i, j, g}.
void orc_es_sample(uint64_t seed, uint64_t k, uint64_t m, uint64_t* out) {
  int g = 0;
  es_sample(seed, k, m, &out[0], &out[1], &g);
  out[2] = (uint64_t)g;
}

// ES-MC run sequentially: switches start_switch, start_switch + 1, ... (the
// result ParES must reproduce).  E must be a canonical simple edge list.
int orc_es_run(uint64_t* E, uint64_t m, uint64_t seed, uint64_t start_switch, uint64_t switches,
               int check_every_switch, orc_stats* st) {
  if (E == nullptr && m > 0) return ORC_E_INVALID;
  if (m < 2) {
    if (st) {
      st->switches += switches;
      st->lazy += switches;
    }
    return ORC_OK;
  }
  std::unordered_set<uint64_t> S;
  S.reserve(m * 2 + 1);
  for (uint64_t i = 0; i < m; ++i) S.insert(E[i]);
  if (S.size() != m) return ORC_E_MULTI;
  std::unordered_map<uint32_t, uint64_t> deg0;
  if (check_every_switch) deg0 = degree_map(E, m);
  for (uint64_t k = start_switch; k < start_switch + switches; ++k) {
    uint64_t i = 0, j = 0;
    int g = 0;
    es_sample(seed, k, m, &i, &j, &g);
    if (st) ++st->switches;
    count(st, edge_switch(E, S, i, j, g));
    if (check_every_switch && !degrees_and_set_ok(E, m, S, deg0)) return ORC_E_INVARIANT;
  }
  return ORC_OK;
}

}  // extern "C"
