"""GPU path (through the C ABI) against the sequential CPU oracle, bit for bit.

Every comparison is of the whole edge list in position order after every
round (Def. 2's sequential outcome), plus the accepted / rejected counts.
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


# kernels of a round whose rounds need one wave (clear, permute, two scans, sort, boundary,
# sources, three overflow kernels, group, wave 1, tail)
ROUND_LAUNCHES = 14


def first_diff(a, b):
    d = np.flatnonzero(a != b)
    return int(d[0]) if len(d) else -1


def run_and_compare(edges, n, seed, rounds, lazy_threshold=0, start_round=0, check_stats=True, exact_ell=False,
                    **opts):
    expect = oracle.validate(edges, n)[1]
    totals = {"accepted": 0, "rejected_loop": 0, "rejected_exists": 0, "lazy": 0}
    with gesmc.Chain(edges, n=n, lazy_threshold=lazy_threshold, start_round=start_round, exact_ell=exact_ell,
                     **opts) as chain:
        for r in range(rounds):
            chain.run(1, seed)
            expect, st = oracle.run(expect, seed=seed, rounds=1, start_round=start_round + r,
                                    lazy_threshold=lazy_threshold, exact_ell=exact_ell)
            for k in totals:
                totals[k] += st[k]
            got = chain.edges()
            assert got.dtype == np.uint64 and len(got) == len(expect)
            pos = first_diff(got, expect)
            assert pos < 0, f"round {start_round + r}: position {pos}: gpu {got[pos]:#x} oracle {expect[pos]:#x}"
        gst = chain.stats()
    if check_stats:
        for k in totals:
            assert gst[k] == totals[k], (k, gst[k], totals[k])
        assert gst["switches"] == rounds * (len(edges) // 2)
        assert gst["rounds"] == rounds
        assert sum(gst["wave_hist"]) == (rounds if len(edges) >= 2 else 0)
    return expect, gst


def test_small_gnp_every_round():
    edges, n = inputs.workload_gnp_small(seed=1)
    _, st = run_and_compare(edges, n, seed=42, rounds=10)
    assert st["accepted"] > 0 and st["waves_max"] >= 1


@pytest.mark.parametrize("m", [2, 3, 4, 5, 17, 64, 1000, 2047, 2048, 2049, 2050, 4095, 4097, 10001, 65537])
def test_sizes_across_bucket_boundaries(m):
    n = max(8, int(4 * m ** 0.5) + 8)
    for seed in (1, 2):
        edges = inputs.random_simple_graph(n, m, seed=m * 31 + seed)
        run_and_compare(edges, n, seed=seed * 1000 + m, rounds=3)


def test_larger_random_graph_with_ragged_tail():
    n = 20_000
    edges = inputs.random_simple_graph(n, 300_001, seed=9)
    run_and_compare(edges, n, seed=5, rounds=3)


@pytest.mark.parametrize("gamma", [2.01, 2.2, 2.5])
def test_power_law_hubs_multi_wave(gamma):
    edges = inputs.pld_graph(5000, gamma, 1, 500, seed=17)
    _, st = run_and_compare(edges, 5000, seed=123, rounds=8)
    assert st["waves_max"] >= 2  # hubs create dependency chains


def test_later_waves_on_the_whole_gpu():
    # the first call's rounds run waves >= 2 on one CTA; after it the chain
    # launches one pair of whole-GPU wave kernels per extra wave it has seen
    edges = inputs.pld_graph(20000, 2.01, 1, 2000, seed=19)
    expect = oracle.validate(edges, 20000)[1]
    with gesmc.Chain(edges, n=20000) as c:
        c.run(1, 31)
        first = c.stats()
        assert first["waves_max"] >= 3 and first["kernel_launches"] == ROUND_LAUNCHES
        c.set_profiling(True)
        c.run(3, 31)
        times, rounds = c.stage_times()
        st = c.stats()
        assert st["kernel_launches"] - ROUND_LAUNCHES > 3 * ROUND_LAUNCHES and times["waves"] > 0
        expect, ost = oracle.run(expect, seed=31, rounds=4)
        assert np.array_equal(c.edges(), expect)
        assert st["accepted"] == ost["accepted"] and st["rejected_exists"] == ost["rejected_exists"]


def test_dense_graph_many_dependencies():
    n = 60
    edges = inputs.random_simple_graph(n, 900, seed=4)   # half of all pairs
    _, st = run_and_compare(edges, n, seed=77, rounds=6)
    assert st["waves_max"] >= 2


def test_complete_graph_and_star_reject_everything():
    kn = oracle.pack(*zip(*[(a, b) for a in range(40) for b in range(a + 1, 40)]))
    _, st = run_and_compare(inputs.shuffle_edges(kn, 1), 40, seed=3, rounds=3)
    assert st["accepted"] == 0
    star = oracle.pack([0] * 500, list(range(1, 501)))
    _, st = run_and_compare(star, 501, seed=4, rounds=3)
    assert st["accepted"] == 0


def test_tiny_and_empty_inputs():
    for lst in ([], [(0, 1)], [(0, 1), (2, 3)], [(0, 1), (2, 3), (4, 5)]):
        e = oracle.pack([a for a, _ in lst], [b for _, b in lst]) if lst else np.zeros(0, np.uint64)
        run_and_compare(e, 6, seed=11, rounds=4)


def test_perfect_matchings_many_seeds():
    edges = oracle.pack(list(range(0, 2000, 2)), list(range(1, 2000, 2)))
    for seed in range(5):
        run_and_compare(edges, 2000, seed=seed, rounds=2)


def test_one_edge_id_proposed_thousands_of_times():
    # {0, 1} gets about L/4 insert tuples per round: its partition overflows
    # (exact overflow path) and holds more tuples than one grouping pass
    edges, n = inputs.double_star(10000, seed=5)
    _, st = run_and_compare(edges, n, seed=21, rounds=3)
    assert st["overflow_tuples"] > 0 and st["subpass_partitions"] > 0


@pytest.mark.parametrize("tuple_log2,group_log2", [(8, 10), (10, 11), (12, 10), (13, 13), (16, 12)])
def test_tuning_does_not_change_the_result(tuple_log2, group_log2):
    n = 20_000
    edges = inputs.random_simple_graph(n, 120_001, seed=12)
    _, st = run_and_compare(edges, n, seed=8, rounds=2, tuple_log2=tuple_log2, group_log2=group_log2)
    if tuple_log2 - group_log2 >= 2:  # more distinct ids per partition than table slots
        assert st["subpass_partitions"] > 0


def test_laziness():
    edges, n = inputs.workload_gnp_small(seed=2)
    _, st = run_and_compare(edges, n, seed=9, rounds=4, lazy_threshold=1 << 62)
    assert 0.2 < st["lazy"] / st["switches"] < 0.3


@pytest.mark.parametrize("t", [1 << 62, 3 << 62, (1 << 64) - 1])
def test_exact_ell(t):
    # Def. 2 as printed: only the first l ~ Binom(L, 1 - P_L) switches run
    edges = inputs.random_simple_graph(3000, 20_001, seed=14)
    _, st = run_and_compare(edges, 3000, seed=10, rounds=4, lazy_threshold=t, exact_ell=True)
    frac = st["lazy"] / st["switches"]
    assert abs(frac - t / 2**64) < 0.02
    edges, n = inputs.workload_gnp_small(seed=3)
    run_and_compare(edges, n, seed=4, rounds=3, lazy_threshold=t, exact_ell=True, graphs=False)


def test_input_orientation_is_canonicalised():
    edges = inputs.random_simple_graph(100, 400, seed=3)
    u, v = oracle.unpack(edges)
    flipped = (v.astype(np.uint64) << np.uint64(32)) | u.astype(np.uint64)
    mixed = np.where(np.arange(400) % 2 == 0, edges, flipped).astype(np.uint64)
    run_and_compare(mixed, 100, seed=8, rounds=2)


def test_resume_from_checkpoint_equals_one_run():
    edges, n = inputs.workload_gnp_small(seed=3)
    with gesmc.Chain(edges, n=n) as c:
        c.run(10, 2024)
        full = c.edges()
    with gesmc.Chain(edges, n=n) as c:
        c.run(4, 2024)
        mid = c.edges()
        assert c.next_round == 4
    with gesmc.Chain(mid, n=n, start_round=4) as c:
        c.run(6, 2024)
        assert np.array_equal(c.edges(), full)
    expect, _ = oracle.run(edges, seed=2024, rounds=10)
    assert np.array_equal(full, expect)


def test_multi_round_call_equals_single_rounds():
    edges, n = inputs.workload_gnp_small(seed=4)
    with gesmc.Chain(edges, n=n) as c:
        c.run(7, 31)
        got = c.edges()
    expect, _ = oracle.run(edges, seed=31, rounds=7)
    assert np.array_equal(got, expect)


def test_device_tensors_in_and_out():
    edges, n = inputs.workload_gnp_small(seed=5)
    dev = torch.from_numpy(edges.view(np.int64)).cuda()
    with gesmc.Chain(dev, n=n) as c:
        c.run(3, 99)
        out = torch.empty_like(dev)
        c.edges(out)
        torch.cuda.synchronize()
    expect, _ = oracle.run(edges, seed=99, rounds=3)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), expect)


def test_invalid_inputs_are_rejected_with_codes():
    loop = np.array([(1 << 32) | 2, (3 << 32) | 3], dtype=np.uint64)
    dup = oracle.pack([0, 1, 2], [1, 2, 1])
    rng = oracle.pack([0, 1], [1, 9])
    for e, n, code in ((loop, 10, gesmc.GESMC_E_LOOP), (dup, 3, gesmc.GESMC_E_MULTI),
                       (rng, 5, gesmc.GESMC_E_RANGE)):
        with pytest.raises(gesmc.GesmcError) as ei:
            gesmc.Chain(e, n=n)
        assert ei.value.code == code
        assert oracle.validate(e, n)[0] == {gesmc.GESMC_E_LOOP: oracle.E_LOOP, gesmc.GESMC_E_MULTI: oracle.E_MULTI,
                                            gesmc.GESMC_E_RANGE: oracle.E_RANGE}[code]


def test_wave_cap_reports_an_error_instead_of_spinning():
    edges = inputs.pld_graph(5000, 2.01, 1, 500, seed=17)
    c = gesmc.Chain(edges, n=5000, max_waves=1)
    with pytest.raises(gesmc.GesmcError) as ei:
        c.run(3, 123)
    assert ei.value.code == gesmc.GESMC_E_WAVE_CAP
    with pytest.raises(gesmc.GesmcError):
        c.run(1, 123)  # the handle stays in its error state
    c.close()


def test_stage_profiling_counts_every_stage():
    edges, n = inputs.workload_gnp_small(seed=6)
    with gesmc.Chain(edges, n=n) as c:
        c.set_profiling(True)
        c.run(5, 1)
        times, rounds = c.stage_times()
        st = c.stats()
    assert rounds == 5 and set(times) >= {"permute", "sortpair", "group", "wave1"}
    assert all(t >= 0 for t in times.values()) and sum(times.values()) > 0
    assert st["kernel_launches"] == 5 * ROUND_LAUNCHES


@pytest.mark.slow
def test_power_law_1m_full_100_rounds():
    """Pld([1..1000], 2.5), n = 1e6, Havel-Hakimi: all 100 rounds bit-exact."""
    edges, n = inputs.workload_pld_1m(seed=2)
    _, st = run_and_compare(edges, n, seed=42, rounds=100)
    assert st["waves_max"] >= 2


@pytest.mark.slow
def test_gnp_2p24_full_size_round():
    """G(2^24, 16/(n-1)), m ~ 1.34e8: the first round at full size, bit-exact,
    in the configuration the benchmark times (one multi-round call)."""
    edges, n = inputs.workload_gnp_2p24(seed=3)
    with gesmc.Chain(edges, n=n) as c:
        c.run(1, 7)
        got = c.edges()
        st = c.stats()
    expect, ost = oracle.run(edges, seed=7, rounds=1)
    pos = first_diff(got, expect)
    assert pos < 0, f"position {pos}"
    assert st["accepted"] == ost["accepted"] and st["rejected_exists"] == ost["rejected_exists"]


@pytest.mark.slow
def test_gnp_2p24_twenty_rounds_match_oracle_digests():
    """G(2^24, 16/(n-1)): all 20 global switches at full size against the
    sequential oracle's per-round SHA-256 digests of the list (written by
    tests/golden/make_gnp_2p24_digests.py), one round per call and then as
    one 20-round call, the configuration the benchmark times."""
    import hashlib
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "gnp_2p24_round_digests.json")) as f:
        gold = json.load(f)

    def digest(a):
        return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()

    edges, n = inputs.workload_gnp_2p24(seed=gold["gen_seed"])
    assert n == gold["n"] and len(edges) == gold["m"]
    assert digest(edges) == gold["input_sha256"], "the generator gave another graph on this machine"
    rounds = gold["rounds"]
    assert len(rounds) == 20
    with gesmc.Chain(edges, n=n) as c:
        accepted = 0
        for r, want in enumerate(rounds):
            c.run(1, gold["chain_seed"])
            accepted += want["accepted"]
            assert digest(c.edges()) == want["sha256"], f"round {r}"
            assert c.stats()["accepted"] == accepted, f"round {r}"   # counters run since create
    with gesmc.Chain(edges, n=n) as c:
        c.run(20, gold["chain_seed"])
        assert digest(c.edges()) == rounds[-1]["sha256"]
        assert c.stats()["accepted"] == sum(w["accepted"] for w in rounds)


def test_graph_replay_equals_direct_launches():
    edges, n = inputs.workload_gnp_small(seed=7)
    with gesmc.Chain(edges, n=n) as a, gesmc.Chain(edges, n=n, graphs=False) as b:
        for rounds in (1, 4, 2, 5):
            a.run(rounds, 77)
            b.run(rounds, 77)
            assert np.array_equal(a.edges(), b.edges())
        la, lb = a.stats()["kernel_launches"], b.stats()["kernel_launches"]
        assert la == lb and la >= 12 * ROUND_LAUNCHES and (la - 12 * ROUND_LAUNCHES) % 2 == 0
    expect, _ = oracle.run(edges, seed=77, rounds=12)
    with gesmc.Chain(edges, n=n) as c:
        c.run(12, 77)
        assert np.array_equal(c.edges(), expect)


@pytest.mark.slow
def test_gnp_2p27_largest_size_keeps_degrees_and_simplicity():
    """G(2^27, 16/(n-1)), about 1.07e9 edges generated on the GPU, near the
    largest chain one GPU holds (155 GB of state): two global switches keep
    every node's degree, the edge count, canonical order and simplicity,
    and accept about every switch (the oracle cannot run this size; these
    properties hold at any size)."""
    n = 1 << 27
    e = gesmc.generate_gnp(n, 16.0 / (n - 1), seed=11)
    m = e.numel()
    assert m > 1_000_000_000 and gesmc.gesmc_device_bytes(m) > 0

    def degrees(x):
        return torch.bincount(x >> 32, minlength=n) + torch.bincount(x & 0xFFFFFFFF, minlength=n)

    deg0 = degrees(e)
    with gesmc.Chain(e, n=n) as c:
        del e
        c.run(2, 5)
        st = c.stats()
        out = torch.empty(m, dtype=torch.int64, device="cuda")
        c.edges(out)
    assert bool(((out >> 32) < (out & 0xFFFFFFFF)).all())      # canonical, no loops
    assert torch.equal(degrees(out), deg0)
    srt = torch.sort(out).values
    assert not bool((srt[1:] == srt[:-1]).any())                # no repeated edge
    assert st["accepted"] + st["rejected_exists"] + st["rejected_loop"] + st["lazy"] == 2 * (m // 2)
    assert st["accepted"] > 0.99 * 2 * (m // 2)
