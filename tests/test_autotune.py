"""Autotuner logic on the CPU: choice, cache, sampling and the agreement check
(with a fake timer; the GPU timer is exercised in the GPU tests)."""
import numpy as np
import pytest

from paper_2111_03005_gb300 import autotune


def fake_graphs(k):
    return [(np.arange(t + 2, dtype=np.uint64), t + 10) for t in range(k)], list(range(100, 100 + k))


def test_pick_is_the_fastest_and_ties_keep_candidate_order():
    assert autotune.pick({(9, 10): 3.0, (10, 11): 1.0, (11, 12): 2.0}) == (10, 11)
    assert autotune.pick({(9, 10): 1.0, (10, 11): 1.0}) == (9, 10)
    with pytest.raises(ValueError):
        autotune.pick({})


def test_tune_times_every_candidate_once_and_caches(tmp_path):
    graphs, seeds = fake_graphs(5)
    times = {(9, 10): 5.0, (9, 11): 4.0, (10, 11): 2.5, (10, 12): 3.0, (11, 11): 2.7, (11, 12): 9.0}
    calls = []

    def timer(g, s, rounds, cand):
        calls.append(cand)
        assert rounds == 2 and len(g) == len(s) == 5
        return times[cand], np.array([1, 2, 3], dtype=np.uint64)

    cache = autotune.TuneCache(str(tmp_path / "tune.json"))
    got = autotune.tune(graphs, seeds, rounds=2, timer=timer, cache=cache, device="dev", launch_candidates=())
    assert (got["tuple_log2"], got["group_log2"]) == (10, 11) and not got["cached"]
    assert calls == list(autotune.CANDIDATES)
    # a second tuner over the same problem class reads the file and times nothing
    again = autotune.tune(graphs, seeds, rounds=2, timer=timer, cache=autotune.TuneCache(str(tmp_path / "tune.json")),
                          device="dev", launch_candidates=())
    assert again["cached"] and (again["tuple_log2"], again["group_log2"]) == (10, 11)
    assert len(calls) == len(autotune.CANDIDATES)
    # another device is another problem class
    other = autotune.tune(graphs, seeds, rounds=2, timer=timer, cache=cache, device="other", launch_candidates=())
    assert not other["cached"]


def test_tune_rejects_a_candidate_that_changes_the_result():
    graphs, seeds = fake_graphs(3)

    def timer(g, s, rounds, cand):
        return 1.0, np.array([0 if cand == (10, 12) else 1], dtype=np.uint64)

    with pytest.raises(RuntimeError):
        autotune.tune(graphs, seeds, timer=timer, cache=None, device="dev", launch_candidates=())


def test_sample_keeps_order_and_pairs():
    graphs, seeds = fake_graphs(50)
    g, s = autotune.sample_graphs(graphs, seeds, 8, rng_seed=1)
    assert len(g) == len(s) == 8
    idx = [seeds.index(x) for x in s]
    assert idx == sorted(idx)
    assert all(g[k] is graphs[i] for k, i in enumerate(idx))
    g2, s2 = autotune.sample_graphs(graphs, seeds, 100)
    assert len(g2) == 50


def test_problem_key_rounds_sizes():
    assert autotune.problem_key("d", 1000, 4096) == autotune.problem_key("d", 1100, 4000)
    assert autotune.problem_key("d", 1000, 4096) != autotune.problem_key("d", 4000, 4096)


def test_ensemble_shards_cover_every_chain_once_and_balance_edges():
    from paper_2111_03005_gb300 import ensemble, inputs

    sizes = [len(e) for e, _ in inputs.ensemble_graphs(256, seed=41, n_lo=100, n_hi=20_000)]
    for world in (1, 2, 3, 8):
        shards = ensemble.shard(sizes, world)
        assert len(shards) == world
        assert sorted(t for sh in shards for t in sh) == list(range(len(sizes)))
        assert all(sh == sorted(sh) for sh in shards)
        loads = [sum(sizes[t] for t in sh) for sh in shards]
        # greedy largest-first: no shard exceeds the mean by more than the largest chain
        assert max(loads) - sum(loads) / world <= max(sizes)
        assert ensemble.shard(sizes, world) == shards          # every rank computes the same split
    assert ensemble.shard([], 4) == [[], [], [], []]


def test_launch_axis_is_tuned_for_small_problems_only(tmp_path):
    graphs, seeds = fake_graphs(4)
    calls = []

    def timer(g, s, rounds, cand):
        calls.append(cand)
        ms = {(11, 11): 1.0}.get(cand[:2], 2.0)
        if len(cand) == 3:
            ms = {0: 1.0, 8: 0.4, 16: 0.3, 32: 0.35}.get(cand[2], 0.9)
        return ms, np.array([7], dtype=np.uint64)

    cache = autotune.TuneCache(str(tmp_path / "t.json"))
    got = autotune.tune(graphs, seeds, timer=timer, cache=cache, device="dev", launch_candidates=(0, 8, 16, 32))
    assert (got["tuple_log2"], got["group_log2"], got["round_ctas"]) == (11, 11, 16)
    assert [c for c in calls if len(c) == 3] == [(11, 11, c) for c in (0, 8, 16, 32)]
    hit = autotune.tune(graphs, seeds, timer=timer, cache=autotune.TuneCache(str(tmp_path / "t.json")), device="dev")
    assert hit["cached"] and hit["round_ctas"] == 16
    # a large problem keeps the multi-kernel round and times no launch candidate
    calls.clear()
    big = autotune.tune(graphs, seeds, timer=timer, cache=None, device="dev", problem=(1 << 24, 1),
                        launch_candidates=(0, 8))
    assert big["round_ctas"] == 0 and all(len(c) == 2 for c in calls)


def test_resident_rounds_are_tried_only_when_every_chain_qualifies():
    R = autotune.ROUND_RESIDENT
    calls = []

    def timer(g, s, rounds, cand):
        calls.append(cand)
        ms = 1.0 if len(cand) == 2 else {0: 1.0, 8: 0.5, R: 0.2}[cand[2]]
        return ms, np.array([7], dtype=np.uint64)

    small = [(np.arange(100, dtype=np.uint64), 500), (np.arange(autotune.RESIDENT_MAX_EDGES, dtype=np.uint64), 65536)]
    got = autotune.tune(small, [1, 2], timer=timer, cache=None, device="dev", launch_candidates=(0, 8, R))
    assert got["round_ctas"] == R and any(len(c) == 3 and c[2] == R for c in calls)
    for bad in ([(np.arange(autotune.RESIDENT_MAX_EDGES + 1, dtype=np.uint64), 100000)],
                [(np.arange(10, dtype=np.uint64), autotune.RESIDENT_MAX_NODES + 1)]):
        calls.clear()
        got = autotune.tune(small + bad, [1, 2, 3], timer=timer, cache=None, device="dev",
                            launch_candidates=(0, 8, R))
        assert got["round_ctas"] == 8 and all(len(c) == 2 or c[2] != R for c in calls)


def test_resident_rounds_are_tried_for_large_pools_of_small_chains():
    R = autotune.ROUND_RESIDENT
    calls = []

    def timer(g, s, rounds, cand):
        calls.append(cand)
        return (1.0 if len(cand) == 2 else {0: 1.0, R: 0.3}[cand[2]]), np.array([7], dtype=np.uint64)

    graphs = [(np.arange(100, dtype=np.uint64), 500)] * 3
    got = autotune.tune(graphs, [1, 2, 3], timer=timer, cache=None, device="dev", problem=(1 << 26, 4096),
                        launch_candidates=(0, 8, 16, R))
    assert got["round_ctas"] == R
    assert [c[2] for c in calls if len(c) == 3] == [0, R]   # no one-launch candidate for a large problem
