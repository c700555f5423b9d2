"""Pools: many chains advanced by one set of kernels per round.  Every chain's
edge list must equal, bit for bit, the sequential oracle run on that chain
alone (its own seed, start round and laziness), whatever else is in the pool
and whenever the chain joined."""
import numpy as np
import pytest

import oracle
from paper_2111_03005_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_03005_gb300 import gesmc  # noqa: E402


def mixed_graphs(seed=0):
    rng = np.random.default_rng(seed)
    graphs = []
    for t in range(12):
        n = int(rng.integers(20, 3000))
        m = int(rng.integers(1, min(4 * n, n * (n - 1) // 2)))
        graphs.append((inputs.random_simple_graph(n, m, seed=100 + t), n))
    graphs.append((inputs.pld_graph(4000, 2.1, 1, 300, seed=5), 4000))
    graphs.append((inputs.workload_gnp_small(seed=2)[0], 1000))
    graphs.append(inputs.double_star(12000, seed=6))   # overflowing partitions: {0, 1} gets ~3000 inserts
    graphs.append(inputs.double_star(16000, seed=7))
    for lst in ([], [(0, 1)], [(0, 1), (2, 3)], [(0, 1), (2, 3), (4, 5)]):
        e = oracle.pack([a for a, _ in lst], [b for _, b in lst]) if lst else np.zeros(0, np.uint64)
        graphs.append((e, 6))
    return graphs


def test_every_chain_matches_its_oracle_alone():
    graphs = mixed_graphs()
    total = sum(len(e) for e, _ in graphs)
    with gesmc.Pool(max_edges=total, max_chains=len(graphs)) as pool:
        ids, expect, meta = [], [], []
        for t, (e, n) in enumerate(graphs):
            seed, start, lazy = 1000 + 7 * t, 3 * t, (1 << 61) if t % 5 == 0 else 0
            exact = t % 10 == 0                   # exact l for half of the lazy chains
            ids.append(pool.add(e, n=n, seed=seed, start_round=start, lazy_threshold=lazy, exact_ell=exact))
            expect.append(oracle.validate(e, n)[1])
            meta.append((seed, start, lazy, exact))
        done = 0
        for rounds in (1, 3, 2):
            pool.run(rounds)
            for t, c in enumerate(ids):
                seed, start, lazy, exact = meta[t]
                expect[t], st = oracle.run(expect[t], seed=seed, rounds=rounds, start_round=start + done,
                                           lazy_threshold=lazy, exact_ell=exact)
                got = pool.edges(c)
                assert np.array_equal(got, expect[t]), (t, rounds)
            done += rounds
        for t, c in enumerate(ids):
            info = pool.chain_info(c)
            assert info["rounds"] == done and info["next_round"] == meta[t][1] + done
            assert info["m"] == len(graphs[t][0])
        total_acc = sum(pool.chain_info(c)["accepted"] for c in ids)
        assert total_acc == pool.stats()["accepted"]
        assert pool.stats()["overflow_tuples"] > 0


def test_chains_join_and_leave_between_rounds():
    graphs = mixed_graphs(seed=1)
    cap = max(sum(len(e) for e, _ in graphs[:8]), max(len(e) for e, _ in graphs))
    with gesmc.Pool(max_edges=cap, max_chains=6) as pool:
        live = {}   # chain id -> (graph index, seed, rounds run, expected list)
        queue = list(range(len(graphs)))
        step = 0
        while queue or live:
            # admit while there is room; "no room" (edges, chain slots or a
            # free range long enough) means: wait until a chain leaves
            while queue:
                g = queue[0]
                e, n = graphs[g]
                try:
                    c = pool.add(e, n=n, seed=50 + g, start_round=g)
                except gesmc.GesmcError as err:
                    assert err.code == gesmc.GESMC_E_NOMEM and live, "an empty pool must admit"
                    break
                queue.pop(0)
                live[c] = [g, 50 + g, 0, oracle.validate(e, n)[1]]
            if not live:
                break
            pool.run(1)
            step += 1
            for c, rec in list(live.items()):
                g, seed, done, exp = rec
                rec[3], _ = oracle.run(exp, seed=seed, rounds=1, start_round=g + done)
                rec[2] = done + 1
                assert np.array_equal(pool.edges(c), rec[3]), (c, g, rec[2])
                if rec[2] == 2 + g % 3:      # each request asks for its own number of rounds
                    pool.remove(c)
                    del live[c]
        assert step > 0 and pool.num_chains == 0


def test_pool_full_and_bad_chain_ids():
    e = inputs.random_simple_graph(50, 100, seed=3)
    with gesmc.Pool(max_edges=150, max_chains=2) as pool:
        a = pool.add(e, n=50, seed=1)
        with pytest.raises(gesmc.GesmcError) as ei:
            pool.add(e, n=50, seed=2)            # 200 edges > 150
        assert ei.value.code == gesmc.GESMC_E_NOMEM
        pool.add(e[:40], n=50, seed=2)
        with pytest.raises(gesmc.GesmcError):
            pool.add(e[:5], n=50, seed=3)         # no chain slot left
        pool.remove(a)
        with pytest.raises(gesmc.GesmcError):
            pool.edges(a)
        pool.add(e[:100], n=50, seed=4)           # the freed room is reused


def test_invalid_chain_does_not_disturb_the_pool():
    e = inputs.random_simple_graph(40, 80, seed=4)
    with gesmc.Pool(max_edges=200, max_chains=3) as pool:
        c = pool.add(e, n=40, seed=9)
        bad = np.array([(1 << 32) | 1], dtype=np.uint64)
        with pytest.raises(gesmc.GesmcError) as ei:
            pool.add(bad, n=40, seed=1)
        assert ei.value.code == gesmc.GESMC_E_LOOP
        pool.run(3)
        expect, _ = oracle.run(e, seed=9, rounds=3)
        assert np.array_equal(pool.edges(c), expect)


@pytest.mark.slow
def test_ensemble_4096_fifty_rounds_match_oracle_digests(golden_dir):
    """The whole null-model ensemble (4096 graphs, 1.46e8 edges) in one pool
    with the autotuner's layout, 50 global switches: every chain's final list
    and accepted count against the sequential oracle run on that chain alone
    (digests written by tests/golden/make_ensemble_digests.py)."""
    import hashlib
    import json
    import os

    with open(os.path.join(golden_dir, "ensemble_4096_digests.json")) as f:
        gold = json.load(f)
    graphs = inputs.ensemble_graphs(gold["count"], seed=gold["gen_seed"])
    h = hashlib.sha256()
    for e, n in graphs:
        h.update(np.array([n, len(e)], dtype="<u8").tobytes())
        h.update(np.ascontiguousarray(e, dtype="<u8").tobytes())
    assert h.hexdigest() == gold["inputs_sha256"], "the generator gave other graphs on this machine"
    total = sum(len(e) for e, _ in graphs)
    with gesmc.Pool(max_edges=total, max_chains=len(graphs), tuple_log2=11, group_log2=11) as pool:
        ids = [pool.add(e, n=n, seed=gold["seed0"] + t) for t, (e, n) in enumerate(graphs)]
        pool.run(gold["rounds"])
        bad = []
        for t, c in enumerate(ids):
            out = pool.edges(c)
            d = hashlib.sha256(np.ascontiguousarray(out, dtype="<u8").tobytes()).hexdigest()[:16]
            if d != gold["digests"][t] or pool.chain_info(c)["accepted"] != gold["accepted"][t]:
                bad.append(t)
    assert not bad, f"{len(bad)} chains differ, first {bad[:8]}"


@pytest.mark.parametrize("max_edges", [5000, 2 * 1024 + 1, 70_000])
def test_one_chain_pool_holds_any_smaller_chain(max_edges):
    """A one-chain pool is sized for its largest chain's own shape; every
    smaller chain (sizes across the steps where the bucket and partition
    counts double) fits in it, one after another, for rounds and for ParES."""
    sizes = sorted({2, 3, 1023, 1024, 1025, 2048, 2049, max_edges // 3, max_edges - 1, max_edges} - {0})
    with gesmc.Pool(max_edges=max_edges, max_chains=1) as pool:
        for t, m in enumerate(s for s in sizes if s <= max_edges):
            n = max(8, int(m ** 0.5 * 4))
            edges = inputs.random_simple_graph(n, m, seed=300 + t)
            c = pool.add(edges, n=n, seed=40 + t)
            pool.run(3)
            expect, _ = oracle.run(edges, seed=40 + t, rounds=3)
            assert np.array_equal(pool.edges(c), expect), m
            pool.es_run(500)
            expect_es, _ = oracle.es_run(expect, seed=40 + t, switches=500)
            assert np.array_equal(pool.edges(c), expect_es), m
            pool.remove(c)
