"""The one-launch round (the whole round in one cooperative launch, stages
separated by bounded grid barriers) against the sequential oracle and
against the multi-kernel round: the same lists after every round, the same
counters and the same wave telemetry, for single chains and pools, with
every CTA count from one to the device's maximum."""
import numpy as np
import pytest

import oracle
from paper_2111_03005_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_03005_gb300 import gesmc  # noqa: E402


def _cases():
    yield "gnp small", *inputs.workload_gnp_small(seed=1)
    yield "power law 2.01", inputs.pld_graph(5000, 2.01, 1, 500, seed=17), 5000
    yield "dense", inputs.random_simple_graph(60, 900, seed=4), 60
    yield "odd m", inputs.random_simple_graph(3000, 20001, seed=6), 3000
    yield "double star", *inputs.double_star(3000, seed=5)


@pytest.mark.parametrize("case", range(5))
@pytest.mark.parametrize("ctas", [1, 7, 64, 10_000])
def test_one_launch_round_matches_the_oracle_every_round(case, ctas):
    name, edges, n = list(_cases())[case]
    rounds = 5
    want, want_w, want_ent = oracle.run_rounds(edges, seed=11, rounds=rounds)
    expect = oracle.validate(edges, n)[1]
    with gesmc.Chain(edges, n=n) as c:
        used = c.set_round_launch(ctas)
        assert 1 <= used <= ctas
        for r in range(rounds):
            before = c.stats()
            c.run(1, 11)
            after = c.stats()
            expect, st = oracle.run(expect, seed=11, rounds=1, start_round=r)
            assert np.array_equal(c.edges(), expect), (name, r)
            w = [x - y for x, y in zip(after["wave_hist"], before["wave_hist"])].index(1)
            assert w == want_w[r], (name, r, w, want_w[r])
            assert after["accepted"] - before["accepted"] == st["accepted"], (name, r)
            assert after["kernel_launches"] - before["kernel_launches"] == 1
        assert np.array_equal(c.edges(), want)


def test_one_launch_pool_matches_the_multi_kernel_pool():
    graphs = inputs.ensemble_graphs(48, seed=41, n_lo=100, n_hi=5000)
    seeds = [700 + t for t in range(len(graphs))]
    total = sum(len(e) for e, _ in graphs)
    out = {}
    for ctas in (0, 32):
        with gesmc.Pool(max_edges=total, max_chains=len(graphs)) as pool:
            ids = [pool.add(e, n=nn, seed=s) for (e, nn), s in zip(graphs, seeds)]
            pool.set_round_launch(ctas)
            pool.run(3)
            # chains leave and join between rounds
            pool.remove(ids[5])
            extra = pool.add(graphs[5][0], n=graphs[5][1], seed=999)
            pool.run(4)
            out[ctas] = ([pool.edges(c) for c in ids if c != ids[5]] + [pool.edges(extra)], pool.stats())
    (a, sa), (b, sb) = out[0], out[32]
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    for k in ("accepted", "rejected_loop", "rejected_exists", "lazy", "waves_total", "waves_max", "wave_hist"):
        assert sa[k] == sb[k], k
    # and the oracle, for one chain of each kind
    for t in (0, 1):
        e, _ = oracle.run(graphs[t][0], seed=seeds[t], rounds=7)
        assert np.array_equal(b[t], e)


def test_one_launch_round_with_laziness_both_forms():
    edges = inputs.pld_graph(3000, 2.2, 1, 300, seed=23)
    for exact in (False, True):
        want, _ = oracle.run(edges, seed=8, rounds=4, start_round=11, lazy_threshold=1 << 62, exact_ell=exact)
        with gesmc.Chain(edges, n=3000, lazy_threshold=1 << 62, exact_ell=exact, start_round=11) as c:
            c.set_round_launch(16)
            c.run(4, 8)
            assert np.array_equal(c.edges(), want)


def test_one_launch_round_wave_cap_reports_an_error():
    edges = inputs.pld_graph(5000, 2.01, 1, 500, seed=17)
    c = gesmc.Chain(edges, n=5000, max_waves=1)
    c.set_round_launch(8)
    with pytest.raises(gesmc.GesmcError) as ei:
        c.run(3, 123)
    assert ei.value.code == gesmc.GESMC_E_WAVE_CAP
    c.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_one_launch_rounds_replayed_or_launched_directly(graphs):
    # several rounds per call (the round's graph replayed, or one cooperative
    # launch per round without graphs), the CTA count changed between calls
    edges, n = inputs.workload_gnp_small(seed=2)
    want, _ = oracle.run(edges, seed=5, rounds=9)
    with gesmc.Chain(edges, n=n, graphs=graphs) as c:
        c.set_round_launch(16)
        c.run(4, 5)
        c.set_round_launch(48)
        c.run(3, 5)
        c.set_round_launch(16)
        c.run(2, 5)
        assert np.array_equal(c.edges(), want)
        assert c.stats()["kernel_launches"] == 9
