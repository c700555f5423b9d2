"""Serving (continuous batching over a pool) and ensembles: every result is
the same alone and in the mix, bit for bit, against the sequential oracle."""
import numpy as np
import pytest

import oracle
from paper_2111_03005_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_03005_gb300 import ensemble, gesmc, serve  # noqa: E402


@pytest.mark.parametrize("rounds_per_step,size_classes,timeout,small_ctas",
                         [(1, (), None, 0), (8, (), None, 0), (3, (2000,), None, 0), (8, (1000, 5000), 0.0005, 0),
                          (4, (2000, 8000), 0.0005, 16), (4, (2000, 8000), 0.0005, 0xFFFFFFFF)])
def test_served_requests_equal_their_oracle_runs(rounds_per_step, size_classes, timeout, small_ctas):
    rng = np.random.default_rng(3)
    reqs = []
    for rid in range(24):
        m_target = int(np.exp(rng.uniform(np.log(200), np.log(20000))))
        e, n = inputs.request_graph(m_target, seed=rid)
        reqs.append(serve.Request(rid=rid, edges=e, n=n, seed=900 + rid, rounds=int(rng.integers(1, 9)),
                                  start_round=int(rng.integers(0, 5))))
    cap = sum(len(r.edges) for r in reqs) // 3          # not everything fits at once
    cap = max(cap, max(len(r.edges) for r in reqs))
    # small_ctas: the size classes run one-launch rounds of that many CTAs
    # (0xFFFFFFFF: resident rounds), up to three times as many rounds between
    # admissions
    with serve.Server(max_edges=cap, max_chains=8, max_rounds_per_step=rounds_per_step,
                      size_classes=size_classes, small_round_ctas=small_ctas,
                      small_rounds_per_step=3 * rounds_per_step if small_ctas else None) as srv:
        assert len(srv.lanes) == len(size_classes) + 1
        arrivals = sorted(rng.integers(0, 30, size=len(reqs)))
        step, nxt = 0, 0
        while nxt < len(reqs) or not srv.idle():
            while nxt < len(reqs) and arrivals[nxt] <= step:   # requests arrive while others run
                srv.submit(reqs[nxt])
                nxt += 1
            srv.step(timeout)
            step += 1
            assert step < 1_000_000
        assert len(srv.done) == len(reqs)
    for r in reqs:
        expect, st = oracle.run(r.edges, seed=r.seed, rounds=r.rounds, start_round=r.start_round)
        assert np.array_equal(r.result, expect), r.rid
        assert r.accepted == st["accepted"], r.rid
        assert r.finished >= r.admitted >= r.arrival


def test_pooled_ensemble_equals_one_handle_per_graph():
    graphs = inputs.ensemble_graphs(48, seed=11, n_lo=100, n_hi=3000)
    seeds = [7000 + t for t in range(len(graphs))]
    pooled = ensemble.run_pool(graphs, seeds, rounds=4)
    alone = ensemble.run_one_by_one(graphs, seeds, rounds=4)
    assert ensemble.same_results(pooled, alone)
    for t in range(0, len(graphs), 7):
        expect, _ = oracle.run(graphs[t][0], seed=seeds[t], rounds=4)
        assert np.array_equal(pooled[t], expect)


def test_autotuned_layout_keeps_every_result(tmp_path):
    from paper_2111_03005_gb300 import autotune

    graphs = inputs.ensemble_graphs(40, seed=12, n_lo=100, n_hi=5000)
    seeds = [8000 + t for t in range(len(graphs))]
    cache = autotune.TuneCache(str(tmp_path / "tune.json"))
    choice = autotune.tune(graphs, seeds, rounds=2, cache=cache)
    assert (choice["tuple_log2"], choice["group_log2"]) in autotune.CANDIDATES and not choice["cached"]
    assert autotune.tune(graphs, seeds, rounds=2, cache=cache)["cached"]
    pooled = ensemble.run_pool(graphs, seeds, rounds=3, tuple_log2=choice["tuple_log2"],
                               group_log2=choice["group_log2"])
    for t in range(0, len(graphs), 9):
        expect, _ = oracle.run(graphs[t][0], seed=seeds[t], rounds=3)
        assert np.array_equal(pooled[t], expect)


def test_autotuned_round_launch_keeps_every_result(tmp_path):
    # the tuner's launch axis (small problems): every candidate launch must give the same lists
    from paper_2111_03005_gb300 import autotune

    graphs = inputs.ensemble_graphs(12, seed=13, n_lo=100, n_hi=2000)
    seeds = [8100 + t for t in range(len(graphs))]
    choice = autotune.tune(graphs, seeds, rounds=2, cache=autotune.TuneCache(str(tmp_path / "t.json")),
                           launch_candidates=(0, 8, 32))
    assert choice["round_ctas"] in (0, 8, 32)
    assert set(choice["launch_timings_ms_per_round"]) == {"0", "8", "32"}
