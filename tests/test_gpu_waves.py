"""The GPU's wave telemetry against Algorithm 1's decide / delay rounds.

The GPU resolves a global switch in Jacobi waves: a switch decided in wave w
only uses the decisions of waves < w (Sec. 4, Algorithm 1; Thm. 2's
worst-case scheduler).  The oracle's ``run_rounds`` restates Algorithm 1's
rounds in that order from the paper's rules (pinned in
tests/test_oracle_pins.py), so for every round the GPU's wave count must equal
the oracle's round count, and the undecided switches entering each wave must
equal the oracle's undecided switches entering each round.  For a pool, one
pool round resolves all chains together: its wave count is the largest over
the chains.
"""
import numpy as np
import pytest

import oracle
from paper_2111_03005_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_03005_gb300 import gesmc  # noqa: E402


def waves_of_last_round(before, after):
    """The wave count of the one round run between two stats snapshots."""
    diff = [a - b for a, b in zip(after["wave_hist"], before["wave_hist"])]
    assert sum(diff) == 1, diff
    return diff.index(1)


def compare_rounds(edges, n, seed, rounds, lazy_threshold=0, exact_ell=False, start_round=0, **opts):
    """Run one round per call; every round's waves and undecided counts must
    equal the oracle's.  Returns the wave counts."""
    want_list, want_w, want_ent = oracle.run_rounds(edges, seed=seed, rounds=rounds, start_round=start_round,
                                                    lazy_threshold=lazy_threshold, exact_ell=exact_ell)
    L = len(edges) // 2
    got_w = []
    with gesmc.Chain(edges, n=n, lazy_threshold=lazy_threshold, exact_ell=exact_ell, start_round=start_round,
                     **opts) as c:
        for r in range(rounds):
            before = c.stats()
            c.run(1, seed)
            after = c.stats()
            w = waves_of_last_round(before, after)
            got_w.append(w)
            assert w == want_w[r], f"round {r}: gpu {w} waves, Algorithm 1 in Jacobi order {want_w[r]} rounds"
            pend = after["last_round_pending"]
            assert pend[1] == L
            for v in range(2, min(w, oracle.MAX_ROUNDS_RECORDED - 1) + 1):
                assert pend[v] == want_ent[r][v], (r, v, pend[v], want_ent[r][v])
            assert not any(pend[w + 1:]), (r, pend[:w + 3])
        assert np.array_equal(c.edges(), want_list)
    return got_w


def test_small_gnp_waves():
    edges, n = inputs.workload_gnp_small(seed=1)
    w = compare_rounds(edges, n, seed=42, rounds=10)
    assert max(w) >= 2


@pytest.mark.parametrize("gamma", [2.01, 2.2, 2.5])
def test_power_law_waves(gamma):
    edges = inputs.pld_graph(5000, gamma, 1, 500, seed=17)
    w = compare_rounds(edges, 5000, seed=123, rounds=8)
    assert max(w) >= 2


def test_heavy_hub_waves_on_the_whole_gpu():
    # many waves per round: after the first rounds the chain runs waves >= 2
    # as whole-GPU kernel pairs, then the single-CTA tail
    edges = inputs.pld_graph(20000, 2.01, 1, 2000, seed=19)
    w = compare_rounds(edges, 20000, seed=31, rounds=6)
    assert max(w) >= 3


def test_dense_and_complete_graph_waves():
    compare_rounds(inputs.random_simple_graph(60, 900, seed=4), 60, seed=77, rounds=6)
    kn = oracle.pack(*zip(*[(a, b) for a in range(40) for b in range(a + 1, 40)]))
    compare_rounds(inputs.shuffle_edges(kn, 1), 40, seed=3, rounds=3)


def test_star_and_matching_need_one_wave():
    star = oracle.pack([0] * 500, list(range(1, 501)))
    assert compare_rounds(star, 501, seed=4, rounds=3) == [1, 1, 1]
    matching = oracle.pack(list(range(0, 2000, 2)), list(range(1, 2000, 2)))
    assert compare_rounds(matching, 2000, seed=5, rounds=3) == [1, 1, 1]


@pytest.mark.parametrize("exact", [False, True])
def test_lazy_waves(exact):
    edges = inputs.pld_graph(3000, 2.2, 1, 300, seed=23)
    compare_rounds(edges, 3000, seed=8, rounds=5, lazy_threshold=1 << 62, exact_ell=exact, start_round=11)


def test_power_law_one_million_nodes_waves():
    # the 1e6-node power-law workload, Pld([1..1000], 2.5) by Havel-Hakimi
    edges, n = inputs.workload_pld_1m()
    w = compare_rounds(edges, n, seed=9, rounds=5)
    assert max(w) >= 2


def test_graph_replay_keeps_the_wave_histogram():
    # a multi-round call replays the captured round; its histogram of wave
    # counts is the oracle's
    edges = inputs.pld_graph(8000, 2.1, 1, 800, seed=29)
    _, want_w, _ = oracle.run_rounds(edges, seed=3, rounds=12)
    with gesmc.Chain(edges, n=8000) as c:
        c.run(12, 3)
        st = c.stats()
    hist = np.bincount(want_w, minlength=gesmc.WAVE_HIST)
    assert st["wave_hist"] == hist.tolist()
    assert st["waves_max"] == int(want_w.max()) and st["waves_total"] == int(want_w.sum())


def test_pool_round_waves_are_the_largest_over_its_chains():
    graphs = [(inputs.pld_graph(3000, g, 1, 300, seed=40 + t), 3000) for t, g in enumerate((2.01, 2.3, 2.6, 3.0))]
    graphs.append(inputs.workload_gnp_small(seed=1))
    seeds = [700 + t for t in range(len(graphs))]
    rounds = 5
    per_chain = [oracle.run_rounds(e, seed=s, rounds=rounds)[1] for (e, _), s in zip(graphs, seeds)]
    want = np.max(np.stack(per_chain), axis=0)
    with gesmc.Pool(max_edges=sum(len(e) for e, _ in graphs), max_chains=len(graphs)) as pool:
        for (e, nn), s in zip(graphs, seeds):
            pool.add(e, n=nn, seed=s)
        got = []
        for _ in range(rounds):
            before = pool.stats()
            pool.run(1)
            got.append(waves_of_last_round(before, pool.stats()))
    assert got == want.tolist()


@pytest.mark.parametrize("name", ["4-regular ring", "gnp, max degree <= sqrt(m)"])
def test_thm2_corollary_on_the_gpu(name):
    # Thm. 2's corollaries: at most 4 rounds in expectation on regular graphs
    # and when every degree is at most sqrt(m); mean over 20 rounds
    if name == "4-regular ring":
        n = 100_000
        edges = oracle.pack([v for v in range(n) for s in (1, 2)], [(v + s) % n for v in range(n) for s in (1, 2)])
    else:
        n = 100_000
        edges = inputs.gnp(n, 8.0 / (n - 1), 13)
        assert np.bincount(np.concatenate(oracle.unpack(edges))).max() <= len(edges) ** 0.5
    with gesmc.Chain(edges, n=n) as c:
        c.run(20, 17)
        st = c.stats()
    assert st["waves_total"] / st["rounds"] <= 4.0
