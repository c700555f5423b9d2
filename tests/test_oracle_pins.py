"""Pins of the CPU oracle to facts that do not come from the oracle itself.

* Fig. 1 and hand-worked global switches (tests/golden/worked_examples.json),
  derived by hand from Def. 1 and Def. 2.
* Philox4x64-10 and the permutation against numpy's own Philox (a separate
  library implementation of the same published generator).
* Special graphs whose outcome the definitions fix (complete graph, star,
  perfect matching, m < 2).
* Invariants after every single switch (degree sequence, simplicity, |E| = m).
* Thm. 1: the exact graph-level transition matrix, enumerated over all m!
  permutations on tiny graphs, is stochastic and symmetric; G(d) is
  brute-forced from all edge subsets; a chi-squared test of the final graph
  after enough rounds against the uniform distribution on G(d).
* Algorithm 1's decide / delay rounds in Jacobi order: hand-worked round
  counts, the same list as the sequential run (Sec. 4: the superstep keeps
  the sequential outcome), and Thm. 2's corollaries (expected rounds <= 4
  on regular graphs and when every degree is <= sqrt(m)).
"""
import itertools
import json
import math
import os
from collections import Counter

import numpy as np
import pytest
from numpy.random import Philox

import oracle
from paper_2111_03005_gb300 import inputs


def P(pairs):
    if not pairs:
        return np.zeros(0, dtype=np.uint64)
    return oracle.pack([a for a, _ in pairs], [b for _, b in pairs])


# ---------------------------------------------------------------- worked examples

def test_fig1_worked_example(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "worked_examples.json")))["fig1"]
    for case in g["cases"]:
        outcome, after = oracle.edge_switch(P(g["edges"]), *case["switch"])
        assert outcome == case["outcome"], case["name"]
        assert np.array_equal(after, P(case["edges_after"])), case["name"]


def test_hand_worked_global_switches(golden_dir):
    cases = json.load(open(os.path.join(golden_dir, "worked_examples.json")))["global"]
    for case in cases:
        after, st = oracle.global_switch(P(case["edges"]), case["pi"])
        assert np.array_equal(after, P(case["edges_after"])), case["name"]
        assert st["accepted"] == case["accepted"], case["name"]


def test_hand_worked_superstep_rounds(golden_dir):
    # every global case carries the number of decide / delay rounds of
    # Algorithm 1 in Jacobi order and the undecided switches entering each
    # round, worked out by hand from Sec. 4's rules
    cases = json.load(open(os.path.join(golden_dir, "worked_examples.json")))["global"]
    assert sum(1 for c in cases if c["rounds"] >= 2) >= 6
    for case in cases:
        after, rounds, entering = oracle.global_switch_rounds(P(case["edges"]), case["pi"])
        assert np.array_equal(after, P(case["edges_after"])), case["name"]
        assert rounds == case["rounds"], case["name"]
        assert entering[1:1 + rounds].tolist() == case["entering"], case["name"]
        assert not entering[1 + rounds:].any(), case["name"]


def _jacobi_cases():
    yield "gnp", inputs.gnp(400, 0.02, 1), 0, False
    yield "power law 2.01", inputs.pld_graph(600, 2.01, 1, 80, seed=3), 0, False
    yield "power law 2.5", inputs.pld_graph(800, 2.5, 1, 60, seed=4), 0, False
    yield "dense", inputs.random_simple_graph(30, 300, 5), 0, False
    yield "lazy", inputs.random_simple_graph(100, 600, 6), 1 << 62, False
    yield "exact l", inputs.random_simple_graph(100, 601, 7), 1 << 63, True
    yield "complete", P([(a, b) for a in range(12) for b in range(a + 1, 12)]), 0, False


@pytest.mark.parametrize("case", list(range(7)))
def test_jacobi_rounds_give_the_sequential_list(case):
    # Sec. 4: the superstep of Algorithm 1 produces the graph of the
    # sequential run; every global switch of several graphs, both laziness forms
    name, e0, t, exact = list(_jacobi_cases())[case]
    want, st = oracle.run(e0, seed=90 + case, rounds=6, lazy_threshold=t, exact_ell=exact)
    got, rounds, entering = oracle.run_rounds(e0, seed=90 + case, rounds=6, lazy_threshold=t, exact_ell=exact)
    assert np.array_equal(got, want), name
    L = len(e0) // 2
    for w, ent in zip(rounds, entering):
        assert w >= 1 and ent[1] == L, name
        assert all(ent[r] > ent[r + 1] for r in range(1, w)), name  # every round decides a switch
        assert not ent[w + 1:].any(), name


def test_rounds_of_special_graphs():
    # m < 2: no switch, no round
    for lst in ([], [(3, 9)]):
        _, rounds, _ = oracle.run_rounds(P(lst), seed=1, rounds=3)
        assert rounds.tolist() == [0, 0, 0]
    # a star: every pair shares the centre, so every switch is known to fail
    # before round 1 (Def. 1) and one round decides them all
    _, rounds, _ = oracle.run_rounds(P([(0, v) for v in range(1, 12)]), seed=2, rounds=5)
    assert rounds.tolist() == [1] * 5
    # a perfect matching: no two switches share a target, so no dependency
    _, rounds, _ = oracle.run_rounds(P([(2 * v, 2 * v + 1) for v in range(40)]), seed=3, rounds=5)
    assert rounds.tolist() == [1] * 5


def _ring_lattice(n, d):
    return P([(v, (v + s) % n) for v in range(n) for s in range(1, d // 2 + 1)])


@pytest.mark.parametrize("name", ["4-regular ring", "10-regular ring", "gnp, max degree <= sqrt(m)"])
def test_thm2_corollaries_mean_rounds_at_most_4(name):
    # Thm. 2 with its corollaries: E[R] <= 4 on d-regular graphs and when
    # every degree is at most sqrt(m) (expectation over pi; mean of 40 rounds)
    if name == "4-regular ring":
        e0 = _ring_lattice(3000, 4)
    elif name == "10-regular ring":
        e0 = _ring_lattice(1000, 10)
    else:
        e0 = inputs.gnp(2000, 0.004, 8)
        deg = np.bincount(np.concatenate(oracle.unpack(e0)))
        assert deg.max() <= math.sqrt(len(e0))
    _, rounds, _ = oracle.run_rounds(e0, seed=5, rounds=40)
    assert rounds.mean() <= 4.0, (name, rounds.tolist())


# ---------------------------------------------------------------- randomness

def _numpy_philox_block(ctr, key):
    # numpy's bit generator increments its 256-bit counter before each block
    c = sum(int(x) << (64 * t) for t, x in enumerate(ctr))
    bg = Philox(key=np.array(key, dtype=np.uint64), counter=(c - 1) % (1 << 256))
    return bg.random_raw(4)


def test_philox_matches_numpy():
    rng = np.random.default_rng(7)
    for _ in range(100):
        ctr = [int(x) for x in rng.integers(0, 2**63, size=4)]
        ctr = [c * 2 + int(rng.integers(0, 2)) for c in ctr]
        key = [int(x) for x in rng.integers(0, 2**63, size=2)]
        assert np.array_equal(oracle.philox4x64_10(ctr, key), _numpy_philox_block(ctr, key))
    assert np.array_equal(oracle.philox4x64_10([0] * 4, [0, 0]), _numpy_philox_block([0] * 4, [0, 0]))
    full = (1 << 64) - 1
    assert np.array_equal(oracle.philox4x64_10([full] * 4, [full, full]), _numpy_philox_block([full] * 4, [full, full]))


@pytest.mark.parametrize("seed,rnd", [(0, 0), (42, 3), (2**64 - 1, 2**40 + 5)])
def test_permutation_is_argsort_of_numpy_philox_keys(seed, rnd):
    m = 1031
    keys = np.empty(m, dtype=np.uint64)
    for b in range((m + 3) // 4):
        blk = _numpy_philox_block([b, rnd, 0, 0], [seed, 0])
        for t in range(4):
            if 4 * b + t < m:
                keys[4 * b + t] = blk[t]
    for i in (0, 1, 5, m - 1):
        assert oracle.perm_key(seed, rnd, i) == int(keys[i])
    expected = np.lexsort((np.arange(m), keys)).astype(np.uint32)  # by key, then position
    assert np.array_equal(oracle.permutation(seed, rnd, m), expected)


def test_lazy_word_stream_is_purpose_one():
    seed, rnd = 99, 7
    blk = _numpy_philox_block([3, rnd, 1, 0], [seed, 0])
    for t in range(4):
        assert oracle.lazy_word(seed, rnd, 12 + t) == int(blk[t])


def test_permutation_uniform_chi2():
    from scipy.stats import chisquare
    m = 4
    counts = Counter()
    n_samples = 24 * 400
    for s in range(n_samples // 8):
        for r in range(8):
            counts[tuple(oracle.permutation(s, r, m))] += 1
    assert len(counts) == 24
    obs = np.array([counts[p] for p in itertools.permutations(range(m))])
    assert chisquare(obs).pvalue > 1e-4


# ---------------------------------------------------------------- special graphs

def test_small_m_is_noop():
    for m, lst in ((0, []), (1, [(3, 9)])):
        e, st = oracle.run(P(lst), seed=1, rounds=5)
        assert np.array_equal(e, P(lst))
        assert st["switches"] == 0 and st["accepted"] == 0


def test_complete_graph_rejects_everything():
    n = 7
    kn = P([(a, b) for a in range(n) for b in range(a + 1, n)])
    e, st = oracle.run(inputs.shuffle_edges(kn, 3), seed=5, rounds=6, check_every_switch=True)
    assert st["accepted"] == 0
    assert st["rejected_loop"] + st["rejected_exists"] == st["switches"] == 6 * (len(kn) // 2)
    assert np.array_equal(e, inputs.shuffle_edges(kn, 3))


def test_star_rejects_everything():
    star = P([(0, v) for v in range(1, 12)])
    e, st = oracle.run(star, seed=8, rounds=5)
    assert st["accepted"] == 0 and np.array_equal(e, star)
    # every pair shares the centre: one orientation is a loop, the other
    # reproduces the two source edges, which are still in E (Def. 1)
    assert st["rejected_loop"] > 0 and st["rejected_exists"] > 0


def test_perfect_matching_m2_follows_the_drawn_permutation():
    start = P([(0, 1), (2, 3)])
    after_01 = P([(0, 3), (1, 2)])   # pi = [0, 1]: g = 1 -> (u, y), (v, x)
    after_10 = P([(1, 3), (0, 2)])   # pi = [1, 0]: g = 0 -> (x, u), (y, v)
    seen = Counter()
    for seed in range(400):
        pi = tuple(oracle.permutation(seed, 0, 2))
        e, st = oracle.run(start, seed=seed, rounds=1)
        assert st["accepted"] == 1
        assert np.array_equal(e, after_01 if pi == (0, 1) else after_10)
        seen[pi] += 1
    assert abs(seen[(0, 1)] - 200) < 5 * math.sqrt(100)


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", range(6))
def test_invariants_after_every_switch(seed):
    e0 = inputs.random_simple_graph(24, 50, seed)
    e, st = oracle.run(e0, seed=seed, rounds=4, check_every_switch=True)
    assert st["switches"] == 4 * 25
    assert st["switches"] == st["lazy"] + st["accepted"] + st["rejected_loop"] + st["rejected_exists"]
    deg0 = np.bincount(np.concatenate(oracle.unpack(e0)), minlength=24)
    deg1 = np.bincount(np.concatenate(oracle.unpack(e)), minlength=24)
    assert np.array_equal(deg0, deg1)
    assert len(set(e.tolist())) == len(e)


def test_invariants_power_law_graph():
    e0 = inputs.pld_graph(300, 2.2, 1, 40, seed=11)
    e, st = oracle.run(e0, seed=3, rounds=3, check_every_switch=True)
    assert st["accepted"] > 0


def test_resume_equals_one_run():
    e0 = inputs.random_simple_graph(60, 200, 4)
    e10, _ = oracle.run(e0, seed=77, rounds=10)
    e5, _ = oracle.run(e0, seed=77, rounds=5)
    e55, _ = oracle.run(e5, seed=77, rounds=5, start_round=5)
    assert np.array_equal(e10, e55)


def test_lazy_rate_matches_threshold():
    e0 = inputs.random_simple_graph(200, 2000, 5)
    _, st = oracle.run(e0, seed=1, rounds=10, lazy_threshold=1 << 62)  # P_L = 1/4
    n = st["switches"]
    assert abs(st["lazy"] - n / 4) < 5 * math.sqrt(n * 3 / 16)


def test_validate_codes():
    assert oracle.validate(P([(0, 1), (1, 2)]), 3)[0] == oracle.OK
    assert oracle.validate(np.array([(2 << 32) | 2], dtype=np.uint64), 3)[0] == oracle.E_LOOP
    assert oracle.validate(P([(0, 1), (1, 0)]), 3)[0] == oracle.E_MULTI
    assert oracle.validate(P([(0, 1), (1, 5)]), 3)[0] == oracle.E_RANGE
    code, canon = oracle.validate(np.array([(5 << 32) | 1], dtype=np.uint64), 0)
    assert code == oracle.OK and int(canon[0]) == (1 << 32) | 5


# ---------------------------------------------------------------- Thm. 1

def enumerate_gd(deg):
    """All simple graphs on len(deg) nodes with exactly this degree sequence."""
    n = len(deg)
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    m = sum(deg) // 2
    out = []
    for combo in itertools.combinations(range(len(pairs)), m):
        d = [0] * n
        for c in combo:
            a, b = pairs[c]
            d[a] += 1
            d[b] += 1
        if d == list(deg):
            out.append(tuple(sorted(pairs[c] for c in combo)))
    return out


def graph_key(edges):
    u, v = oracle.unpack(edges)
    return tuple(sorted(zip(u.tolist(), v.tolist())))


def transition_counts(states, m, lazy_patterns=None):
    """counts[A][B] = #(pi, skip pattern) taking graph A to graph B."""
    index = {s: t for t, s in enumerate(states)}
    C = np.zeros((len(states), len(states)), dtype=np.int64)
    perms = list(itertools.permutations(range(m)))
    patterns = lazy_patterns or [None]
    for a, s in enumerate(states):
        e = P(list(s))
        for pi in perms:
            for pat in patterns:
                after, _ = oracle.global_switch(e, pi, skip=pat)
                C[a, index[graph_key(after)]] += 1
    return C


@pytest.mark.parametrize("deg", [(1, 1, 1, 1), (2, 2, 1, 1, 1, 1), (2, 2, 2, 2, 1, 1), (2, 2, 2, 2, 2, 2),
                                 (3, 2, 2, 2, 2, 1)])
def test_transition_matrix_symmetric_and_stochastic(deg):
    states = enumerate_gd(deg)
    m = sum(deg) // 2
    C = transition_counts(states, m)
    assert (C.sum(axis=1) == math.factorial(m)).all()      # every row is a distribution
    assert np.array_equal(C, C.T)                           # Thm. 1: P_AB = P_BA
    # irreducible and aperiodic on G(d): some power is entrywise positive
    Pm = C / math.factorial(m)
    Q = np.linalg.matrix_power(Pm, 4 * len(states))
    assert (Q > 0).all()


def test_transition_matrix_symmetric_with_laziness():
    deg = (2, 2, 2, 2, 1, 1)
    states = enumerate_gd(deg)
    m = sum(deg) // 2
    L = m // 2
    pats = [np.array(p, dtype=np.uint8) for p in itertools.product((0, 1), repeat=L)]
    C = transition_counts(states, m, lazy_patterns=pats)     # P_L = 1/2: equal weights
    assert (C.sum(axis=1) == math.factorial(m) * 2**L).all()
    assert np.array_equal(C, C.T)


def test_final_graph_uniform_on_gd_chi2():
    from scipy.stats import chisquare
    deg = (2, 2, 2, 2, 2, 2)
    states = enumerate_gd(deg)
    assert len(states) == 70            # 60 hexagons + 10 pairs of triangles
    m = sum(deg) // 2
    Pm = transition_counts(states, m) / math.factorial(m)
    start = inputs.havel_hakimi(np.array(deg, dtype=np.uint32))
    x = np.zeros(len(states))
    x[states.index(graph_key(start))] = 1.0
    rounds = 0
    while 0.5 * np.abs(x - 1.0 / len(states)).sum() > 1e-4:
        x = x @ Pm
        rounds += 1
    index = {s: t for t, s in enumerate(states)}
    counts = np.zeros(len(states), dtype=np.int64)
    n_samples = 21000
    for seed in range(n_samples):
        e, _ = oracle.run(start, seed=seed + 1000, rounds=rounds)
        counts[index[graph_key(e)]] += 1
    assert chisquare(counts).pvalue > 1e-4


# ---------------------------------------------------------------- exact l (Def. 2 as printed)

def _numpy_lazy_words(seed, rnd, L):
    words = []
    for b in range((L + 3) // 4):
        words.extend(int(x) for x in _numpy_philox_block([b, rnd, 1, 0], [seed, 0]))
    return words[:L]


@pytest.mark.parametrize("t", [1 << 62, 1 << 63, (1 << 64) - (1 << 60)])
def test_exact_ell_runs_the_first_ell_switches(t):
    # l from numpy's Philox (an independent implementation) and the permutation
    # from numpy keys; one exact-l round must equal the first l switches of pi
    e0 = inputs.random_simple_graph(60, 171, seed=5)
    m, L = len(e0), len(e0) // 2
    canon = oracle.validate(e0, 60)[1]
    for seed, rnd in ((3, 0), (11, 4)):
        ell = sum(w >= t for w in _numpy_lazy_words(seed, rnd, L))
        keys = np.empty(m, dtype=np.uint64)
        for b in range((m + 3) // 4):
            blk = _numpy_philox_block([b, rnd, 0, 0], [seed, 0])
            for q in range(4):
                if 4 * b + q < m:
                    keys[4 * b + q] = blk[q]
        pi = np.lexsort((np.arange(m), keys)).astype(np.uint32)
        want, wst = oracle.global_switch(canon, pi, ell=ell)
        got, st = oracle.run(canon, seed=seed, rounds=1, start_round=rnd, lazy_threshold=t, exact_ell=True)
        assert np.array_equal(got, want)
        assert st["lazy"] == L - ell and st["accepted"] == wst["accepted"]


def test_exact_ell_without_laziness_is_the_plain_round():
    e0 = inputs.random_simple_graph(40, 90, seed=2)
    a, sa = oracle.run(e0, seed=5, rounds=4)
    b, sb = oracle.run(e0, seed=5, rounds=4, exact_ell=True)
    assert np.array_equal(a, b) and sa == sb


def test_exact_ell_is_binomial():
    from scipy.stats import binom, chisquare
    # l over many rounds: Binom(L, 1 - P_L) with P_L = 3/8
    e0 = inputs.random_simple_graph(30, 24, seed=8)
    L, pl = 12, 3 / 8
    t = int(pl * 2**64)
    counts = np.zeros(L + 1, dtype=np.int64)
    for seed in range(1500):
        _, st = oracle.run(e0, seed=seed, rounds=1, lazy_threshold=t, exact_ell=True)
        counts[L - st["lazy"]] += 1
    expect = binom.pmf(np.arange(L + 1), L, 1 - pl) * counts.sum()
    keep = expect >= 5
    obs = np.append(counts[keep], counts[~keep].sum())
    exp = np.append(expect[keep], expect[~keep].sum())
    assert chisquare(obs, exp * obs.sum() / exp.sum()).pvalue > 1e-4


def test_transition_matrix_symmetric_with_exact_ell():
    # Def. 2 as printed: P = sum_l Binom(L, 1 - P_L)(l) * (1/m!) sum_pi T(pi, l); with P_L = 1/2 the
    # weights are C(L, l) / 2^L, so integer counts weighted by C(L, l) must be symmetric
    deg = (2, 2, 2, 2, 1, 1)
    states = enumerate_gd(deg)
    m = sum(deg) // 2
    L = m // 2
    index = {s: t for t, s in enumerate(states)}
    C = np.zeros((len(states), len(states)), dtype=np.int64)
    for a, s in enumerate(states):
        e = P(list(s))
        for pi in itertools.permutations(range(m)):
            for ell in range(L + 1):
                after, _ = oracle.global_switch(e, pi, ell=ell)
                C[a, index[graph_key(after)]] += math.comb(L, ell)
    assert (C.sum(axis=1) == math.factorial(m) * 2**L).all()
    assert np.array_equal(C, C.T)


# ---------------------------------------------------------------- ES-MC (the chain of Algorithm 2, ParES)

def _numpy_es_sample(seed, k, m):
    w = [int(x) for x in _numpy_philox_block([k, 0, 2, 0], [seed, 0])]
    i = (w[0] * m) >> 64
    jj = (w[1] * (m - 1)) >> 64
    return i, jj + (1 if jj >= i else 0), w[2] >> 63


def test_es_sample_matches_numpy_philox():
    for seed, k, m in ((0, 0, 2), (7, 12345, 1000), (2**64 - 1, 2**40, 134198120), (5, 3, 3)):
        assert oracle.es_sample(seed, k, m) == _numpy_es_sample(seed, k, m)
        i, j, g = oracle.es_sample(seed, k, m)
        assert 0 <= i < m and 0 <= j < m and i != j and g in (0, 1)


def test_es_run_is_the_sampled_switches_in_order():
    e0 = oracle.validate(inputs.random_simple_graph(40, 70, seed=6), 40)[1]
    want = e0.copy()
    acc = 0
    for k in range(5, 5 + 300):
        i, j, g = _numpy_es_sample(11, k, len(e0))
        outcome, want = oracle.edge_switch(want, i, j, g)
        acc += outcome == 0
    got, st = oracle.es_run(e0, seed=11, switches=300, start_switch=5)
    assert np.array_equal(got, want) and st["accepted"] == acc and st["switches"] == 300


def test_es_run_resumes_and_keeps_invariants():
    e0 = inputs.pld_graph(300, 2.2, 1, 40, seed=3)
    a, _ = oracle.es_run(e0, seed=2, switches=500, check_every_switch=True)
    a, _ = oracle.es_run(a, seed=2, switches=700, start_switch=500, check_every_switch=True)
    b, _ = oracle.es_run(e0, seed=2, switches=1200)
    assert np.array_equal(a, b)
    assert oracle.es_run(np.zeros(1, np.uint64), seed=1, switches=5)[1]["lazy"] == 5


def es_transition_counts(states, m):
    index = {s: t for t, s in enumerate(states)}
    C = np.zeros((len(states), len(states)), dtype=np.int64)
    for a, s in enumerate(states):
        e = P(list(s))
        for i in range(m):
            for j in range(m):
                if i == j:
                    continue
                for g in (0, 1):
                    _, after = oracle.edge_switch(e, i, j, g)
                    C[a, index[graph_key(after)]] += 1
    return C


@pytest.mark.parametrize("deg", [(2, 2, 1, 1, 1, 1), (2, 2, 2, 2, 2, 2), (3, 2, 2, 2, 2, 1)])
def test_es_transition_matrix_symmetric(deg):
    # ES-MC picks (i, j, g) uniformly: the lumped matrix is symmetric (Obs. 1)
    states = enumerate_gd(deg)
    m = sum(deg) // 2
    C = es_transition_counts(states, m)
    assert (C.sum(axis=1) == m * (m - 1) * 2).all()
    assert np.array_equal(C, C.T)


def test_es_final_graph_uniform_on_gd_chi2():
    from scipy.stats import chisquare
    deg = (2, 2, 2, 2, 2, 2)
    states = enumerate_gd(deg)
    m = sum(deg) // 2
    Pm = es_transition_counts(states, m) / (m * (m - 1) * 2)
    start = inputs.havel_hakimi(np.array(deg, dtype=np.uint32))
    x = np.zeros(len(states))
    x[states.index(graph_key(start))] = 1.0
    steps = 0
    while 0.5 * np.abs(x - 1.0 / len(states)).sum() > 1e-4:
        x = x @ Pm
        steps += 1
    index = {s: t for t, s in enumerate(states)}
    counts = np.zeros(len(states), dtype=np.int64)
    for seed in range(14000):
        e, _ = oracle.es_run(start, seed=seed + 77, switches=steps)
        counts[index[graph_key(e)]] += 1
    assert chisquare(counts).pvalue > 1e-4
