"""Resident rounds (one CTA per small chain, the list in shared memory for all
rounds of a call) against the sequential oracle and against the multi-kernel
round: the same lists after every round and after many rounds in one call,
the same counters, and the same wave telemetry as Algorithm 1's decide /
delay rounds in Jacobi order."""
import numpy as np
import pytest

import oracle
from paper_2111_03005_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_03005_gb300 import gesmc  # noqa: E402

RESIDENT = gesmc.ROUND_RESIDENT
COUNTERS = ("accepted", "rejected_loop", "rejected_exists", "lazy", "waves_total", "waves_max", "wave_hist",
            "last_round_pending")


def _cases():
    yield "gnp 1000 0.01", *inputs.workload_gnp_small(seed=1)
    yield "power law 2.01", inputs.pld_graph(5000, 2.01, 1, 500, seed=17), 5000
    yield "dense", inputs.random_simple_graph(60, 900, seed=4), 60
    yield "odd m", inputs.random_simple_graph(3000, 9001, seed=6), 3000
    yield "double star", *inputs.double_star(3000, seed=5)
    yield "largest", inputs.random_simple_graph(20000, gesmc.RESIDENT_MAX_EDGES, seed=8), 20000
    yield "ids up to 65535", inputs.random_simple_graph(65536, 4000, seed=9), 65536


@pytest.mark.parametrize("case", range(7))
def test_resident_rounds_match_the_oracle_every_round(case):
    name, edges, n = list(_cases())[case]
    assert len(edges) <= gesmc.RESIDENT_MAX_EDGES
    rounds = 5
    want, want_w, want_ent = oracle.run_rounds(edges, seed=11, rounds=rounds)
    expect = oracle.validate(edges, n)[1]
    L = len(edges) // 2
    with gesmc.Chain(edges, n=n) as c:
        assert c.set_round_launch(RESIDENT) == RESIDENT
        for r in range(rounds):
            before = c.stats()
            c.run(1, 11)
            after = c.stats()
            expect, st = oracle.run(expect, seed=11, rounds=1, start_round=r)
            assert np.array_equal(c.edges(), expect), (name, r)
            diff = [x - y for x, y in zip(after["wave_hist"], before["wave_hist"])]
            assert sum(diff) == 1 and diff.index(1) == want_w[r], (name, r, diff, want_w[r])
            w = int(want_w[r])
            pend = after["last_round_pending"]
            assert pend[1] == L
            for v in range(2, min(w, oracle.MAX_ROUNDS_RECORDED - 1) + 1):
                assert pend[v] == want_ent[r][v], (name, r, v, pend[v], want_ent[r][v])
            assert not any(pend[w + 1:])
            for k in ("accepted", "rejected_loop", "rejected_exists", "lazy"):
                assert after[k] - before[k] == st[k], (name, r, k)
        assert np.array_equal(c.edges(), want)


@pytest.mark.parametrize("case", range(7))
def test_many_rounds_in_one_call_equal_the_multi_kernel_round(case):
    name, edges, n = list(_cases())[case]
    rounds = 30
    want, st = oracle.run(edges, seed=3, rounds=rounds, start_round=4)
    out = {}
    for mode in (0, RESIDENT):
        with gesmc.Chain(edges, n=n, start_round=4) as c:
            c.set_round_launch(mode)
            before = c.stats()["kernel_launches"]
            c.run(rounds, 3)
            out[mode] = (c.edges(), c.stats(), c.stats()["kernel_launches"] - before)
    assert np.array_equal(out[RESIDENT][0], want), name
    assert np.array_equal(out[0][0], want), name
    for k in COUNTERS:
        assert out[0][1][k] == out[RESIDENT][1][k], (name, k)
    assert out[RESIDENT][1]["accepted"] == st["accepted"]
    # per launch of many rounds: the chain's CTA and the fold, and (a pool of
    # few chains) the kernel that sorts the rounds' permutations beforehand
    # (as many rounds per launch as their scratch space holds)
    assert out[RESIDENT][2] <= 3 * 3


def test_rounds_beyond_one_launch():
    # a pool of a few edges has 4096 scratch bits: 64 rounds per launch
    edges = inputs.random_simple_graph(12, 20, seed=3)
    want, _ = oracle.run(edges, seed=5, rounds=150)
    with gesmc.Chain(edges, n=12) as c:
        c.set_round_launch(RESIDENT)
        before = c.stats()["kernel_launches"]
        c.run(150, 5)
        assert np.array_equal(c.edges(), want)
        assert c.stats()["kernel_launches"] - before in (6, 9)   # three launches of 2 or 3 kernels
        assert sum(c.stats()["wave_hist"]) == 150


def test_resident_with_laziness_both_forms():
    edges = inputs.pld_graph(3000, 2.2, 1, 300, seed=23)
    for exact in (False, True):
        for thr in (1 << 62, 1 << 63, (1 << 64) - 1):
            want, st = oracle.run(edges, seed=8, rounds=6, start_round=11, lazy_threshold=thr, exact_ell=exact)
            with gesmc.Chain(edges, n=3000, lazy_threshold=thr, exact_ell=exact, start_round=11) as c:
                c.set_round_launch(RESIDENT)
                c.run(6, 8)
                assert np.array_equal(c.edges(), want), (exact, thr)
                assert c.stats()["lazy"] == st["lazy"], (exact, thr)
                assert c.stats()["accepted"] == st["accepted"], (exact, thr)


def test_switching_launch_modes_between_calls():
    # pending decisions of a multi-kernel round are applied on load; the
    # resident call leaves nothing pending for the next multi-kernel round
    edges, n = inputs.workload_gnp_small(seed=3)
    want, _ = oracle.run(edges, seed=9, rounds=12)
    with gesmc.Chain(edges, n=n) as c:
        c.run(3, 9)
        c.set_round_launch(RESIDENT)
        c.run(4, 9)
        c.set_round_launch(16)
        c.run(2, 9)
        c.set_round_launch(RESIDENT)
        c.run(1, 9)
        c.set_round_launch(0)
        c.run(2, 9)
        assert np.array_equal(c.edges(), want)
        assert c.verify() == gesmc.GESMC_OK


def test_resident_and_pares_on_one_chain():
    edges, n = inputs.workload_gnp_small(seed=4)
    mid, _ = oracle.run(edges, seed=2, rounds=3)
    mid, _ = oracle.es_run(mid, seed=2, switches=5000)
    want, _ = oracle.run(mid, seed=2, rounds=2, start_round=3)
    with gesmc.Chain(edges, n=n) as c:
        c.set_round_launch(RESIDENT)
        c.run(3, 2)
        c.es_run(5000, 2)
        c.run(2, 2)
        assert np.array_equal(c.edges(), want)


def test_resident_pool_matches_the_multi_kernel_pool():
    graphs = inputs.ensemble_graphs(64, seed=41, n_lo=20, n_hi=3000)
    graphs = [(e, n) for e, n in graphs if len(e) <= gesmc.RESIDENT_MAX_EDGES]
    seeds = [700 + t for t in range(len(graphs))]
    total = sum(len(e) for e, _ in graphs)
    out = {}
    for mode in (0, RESIDENT):
        with gesmc.Pool(max_edges=total, max_chains=len(graphs)) as pool:
            ids = [pool.add(e, n=nn, seed=s) for (e, nn), s in zip(graphs, seeds)]
            pool.set_round_launch(mode)
            pool.run(3)
            # chains leave and join between calls
            pool.remove(ids[5])
            extra = pool.add(graphs[5][0], n=graphs[5][1], seed=999)
            pool.run(4)
            out[mode] = ([pool.edges(c) for c in ids if c != ids[5]] + [pool.edges(extra)], pool.stats())
    (a, sa), (b, sb) = out[0], out[RESIDENT]
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    for k in COUNTERS:
        assert sa[k] == sb[k], k
    for t in (0, 1, 2):
        e, _ = oracle.run(graphs[t][0], seed=seeds[t], rounds=7)
        assert np.array_equal(b[t], e)


def test_tiny_chains():
    for m in (2, 3, 4, 5):
        edges = np.array([(2 * i << 32) | (2 * i + 1) for i in range(m)], dtype=np.uint64)  # a matching
        want, _ = oracle.run(edges, seed=1, rounds=9)
        with gesmc.Chain(edges, n=2 * m) as c:
            c.set_round_launch(RESIDENT)
            c.run(9, 1)
            assert np.array_equal(c.edges(), want), m
    star = np.array([(0 << 32) | i for i in range(1, 200)], dtype=np.uint64)  # every switch shares the hub
    with gesmc.Chain(star, n=200) as c:
        c.set_round_launch(RESIDENT)
        c.run(5, 1)
        assert np.array_equal(c.edges(), oracle.run(star, seed=1, rounds=5)[0])
        assert c.stats()["accepted"] == 0


def test_too_large_for_resident_rounds():
    big = inputs.random_simple_graph(30000, gesmc.RESIDENT_MAX_EDGES + 1, seed=2)
    with gesmc.Chain(big, n=30000) as c:
        with pytest.raises(gesmc.GesmcError) as ei:
            c.set_round_launch(RESIDENT)
        assert ei.value.code == gesmc.GESMC_E_TOO_LARGE
        c.run(1, 1)             # still runs on the multi-kernel round
    wide = inputs.random_simple_graph(70000, 1000, seed=2)
    with gesmc.Chain(wide, n=70000) as c:
        with pytest.raises(gesmc.GesmcError) as ei:
            c.set_round_launch(RESIDENT)
        assert ei.value.code == gesmc.GESMC_E_TOO_LARGE
    with gesmc.Pool(max_edges=40000, max_chains=4) as pool:
        pool.set_round_launch(RESIDENT)
        pool.add(inputs.random_simple_graph(500, 1000, seed=1), n=500, seed=1)
        with pytest.raises(gesmc.GesmcError) as ei:
            pool.add(big, n=30000, seed=2)
        assert ei.value.code == gesmc.GESMC_E_TOO_LARGE


def test_resident_wave_cap_reports_an_error():
    edges = inputs.pld_graph(5000, 2.01, 1, 500, seed=17)
    c = gesmc.Chain(edges, n=5000, max_waves=1)
    c.set_round_launch(RESIDENT)
    with pytest.raises(gesmc.GesmcError) as ei:
        c.run(3, 123)
    assert ei.value.code == gesmc.GESMC_E_WAVE_CAP
    c.close()


def test_few_chains_of_every_class_sorted_ahead():
    # a pool of few chains has its permutations sorted beforehand on other
    # SMs (one kernel per size class): the same lists as the oracle
    sizes = [(300, 800), (700, 1500), (1500, 3000), (2400, 6000), (4000, 9500)]
    graphs = [(inputs.random_simple_graph(n, m, seed=50 + t), n) for t, (n, m) in enumerate(sizes)]
    total = sum(len(e) for e, _ in graphs)
    with gesmc.Pool(max_edges=total, max_chains=len(graphs)) as pool:
        ids = [pool.add(e, n=n, seed=80 + t, start_round=t) for t, (e, n) in enumerate(graphs)]
        pool.set_round_launch(RESIDENT)
        pool.run(7)
        pool.run(5)
        outs = [pool.edges(c) for c in ids]
    for t, (e, n) in enumerate(graphs):
        want, _ = oracle.run(e, seed=80 + t, rounds=12, start_round=t)
        assert np.array_equal(outs[t], want), t


def test_many_chains_with_exact_laziness_sorted_in_their_own_ctas():
    # a pool of many chains sorts each round's permutation in the chain's own
    # CTA (no presort); exact l is counted there too
    graphs = inputs.ensemble_graphs(48, seed=43, n_lo=20, n_hi=2000)
    graphs = [(e, n) for e, n in graphs if len(e) <= gesmc.RESIDENT_MAX_EDGES]
    total = sum(len(e) for e, _ in graphs)
    thr = 1 << 62
    with gesmc.Pool(max_edges=total, max_chains=len(graphs)) as pool:
        ids = [pool.add(e, n=n, seed=90 + t, lazy_threshold=thr, exact_ell=True)
               for t, (e, n) in enumerate(graphs)]
        pool.set_round_launch(RESIDENT)
        pool.run(6)
        outs = [pool.edges(c) for c in ids]
    for t in range(0, len(graphs), 5):
        want, _ = oracle.run(graphs[t][0], seed=90 + t, rounds=6, lazy_threshold=thr, exact_ell=True)
        assert np.array_equal(outs[t], want), t
