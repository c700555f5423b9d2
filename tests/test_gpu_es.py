"""ParES (Algorithm 2) through the C ABI against the sequential ES-MC oracle,
bit for bit: the edge list in position order after every call, and the
accepted / rejected counts."""
import numpy as np
import pytest

import oracle
from paper_2111_03005_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_03005_gb300 import gesmc  # noqa: E402

COUNTS = ("accepted", "rejected_loop", "rejected_exists", "lazy")


def es_compare(edges, n, seed, calls):
    expect = oracle.validate(edges, n)[1]
    done, totals = 0, dict.fromkeys(COUNTS, 0)
    with gesmc.Chain(edges, n=n) as c:
        for r in calls:
            c.es_run(r, seed)
            expect, st = oracle.es_run(expect, seed=seed, switches=r, start_switch=done)
            done += r
            for k in COUNTS:
                totals[k] += st[k]
            got = c.edges()
            d = np.flatnonzero(got != expect)
            assert len(d) == 0, f"after {done} switches: position {d[0]}"
        gst = c.stats()
    for k in COUNTS:
        assert gst[k] == totals[k], (k, gst[k], totals[k])
    return gst


def test_small_graph_many_calls():
    edges, n = inputs.workload_gnp_small(seed=1)
    st = es_compare(edges, n, seed=5, calls=[1, 7, 100, 1000, 20000])
    assert st["accepted"] > 0


@pytest.mark.parametrize("m", [2, 3, 17, 1023, 1025, 4097])
def test_sizes(m):
    n = max(8, int(3 * m ** 0.5) + 8)
    edges = inputs.random_simple_graph(n, m, seed=m)
    es_compare(edges, n, seed=m + 1, calls=[3 * m + 5])


def test_power_law_hubs_and_dense_graph():
    edges = inputs.pld_graph(5000, 2.01, 1, 500, seed=17)
    es_compare(edges, 5000, seed=4, calls=[5000, 30000])
    dense = inputs.random_simple_graph(60, 900, seed=4)
    es_compare(dense, 60, seed=9, calls=[20000])


def test_many_supersteps_and_edge_set_rebuilds():
    # a call much longer than the edge set's chunk (about an eighth of its slots)
    edges = inputs.random_simple_graph(20_000, 50_001, seed=3)
    es_compare(edges, 20_000, seed=12, calls=[400_000])


def test_empty_and_single_edge():
    for lst in ([], [(0, 1)]):
        e = oracle.pack([a for a, _ in lst], [b for _, b in lst]) if lst else np.zeros(0, np.uint64)
        st = es_compare(e, 4, seed=1, calls=[10, 5])
        assert st["lazy"] == 15


def test_mixed_with_global_switches_and_reseed():
    edges, n = inputs.workload_gnp_small(seed=2)
    expect = oracle.validate(edges, n)[1]
    with gesmc.Chain(edges, n=n) as c:
        c.run(2, 7)
        c.es_run(500, 7)
        c.run(1, 7)
        c.es_run(300, 7)
        c.es_run(200, 8)   # a new seed: ES switches and rounds are numbered on
        c.run(2, 8)
        got = c.edges()
    expect, _ = oracle.run(expect, seed=7, rounds=2)
    expect, _ = oracle.es_run(expect, seed=7, switches=500)
    expect, _ = oracle.run(expect, seed=7, rounds=1, start_round=2)
    expect, _ = oracle.es_run(expect, seed=7, switches=300, start_switch=500)
    expect, _ = oracle.es_run(expect, seed=8, switches=200, start_switch=800)
    expect, _ = oracle.run(expect, seed=8, rounds=2, start_round=3)
    assert np.array_equal(got, expect)


def test_pool_of_chains():
    rng = np.random.default_rng(5)
    graphs = []
    for t in range(20):
        n = int(rng.integers(10, 2000))
        m = int(rng.integers(0, min(3 * n, n * (n - 1) // 2)))
        graphs.append((inputs.random_simple_graph(n, m, seed=200 + t), n))
    total = sum(len(e) for e, _ in graphs)
    with gesmc.Pool(max_edges=total, max_chains=len(graphs)) as pool:
        ids = [pool.add(e, n=n, seed=300 + t) for t, (e, n) in enumerate(graphs)]
        pool.run(1)
        pool.es_run(2000)
        pool.run(1)
        outs = [pool.edges(c) for c in ids]
        infos = [pool.chain_info(c) for c in ids]
    for t, (e, n) in enumerate(graphs):
        x = oracle.validate(e, n)[1]
        x, _ = oracle.run(x, seed=300 + t, rounds=1)
        x, _ = oracle.es_run(x, seed=300 + t, switches=2000)
        x, _ = oracle.run(x, seed=300 + t, rounds=1, start_round=1)
        assert np.array_equal(outs[t], x), t
        assert infos[t]["es_switches"] == 2000


def test_large_chain_wide_windows_and_rebuild():
    """A chain above 2^19 edges runs windows of 1024 switches; 700,000
    switches pass the edge set's rebuild threshold (a quarter of its slots
    in tombstones) at least once."""
    n = 1 << 17
    edges = inputs.gnp(n, 10.0 / (n - 1), seed=21)
    assert len(edges) >= 1 << 19
    st = es_compare(edges, n, seed=6, calls=[1000, 700_000])
    assert st["accepted"] > 600_000


def test_pool_mixes_wide_and_narrow_windows():
    """Chains for every window size in one call (four kernel variants, the
    two small ones on a second stream, jobs reordered by window size): each
    equals its sequential run."""
    n_big = 1 << 17
    graphs = [(inputs.random_simple_graph(300, 900, seed=31), 300),
              (inputs.gnp(n_big, 9.0 / (n_big - 1), seed=22), n_big),
              (inputs.random_simple_graph(2000, 5000, seed=32), 2000),
              (inputs.random_simple_graph(6000, 20_000, seed=33), 6000),
              (inputs.random_simple_graph(40_000, 100_000, seed=34), 40_000),
              (np.zeros(0, np.uint64), 4),
              (inputs.gnp(n_big, 9.5 / (n_big - 1), seed=23), n_big)]
    assert len(graphs[1][0]) >= 1 << 19 and len(graphs[6][0]) >= 1 << 19
    total = sum(len(e) for e, _ in graphs)
    with gesmc.Pool(max_edges=total, max_chains=len(graphs)) as pool:
        ids = [pool.add(e, n=n, seed=500 + t) for t, (e, n) in enumerate(graphs)]
        pool.es_run(30_000)
        outs = [pool.edges(c) for c in ids]
        infos = [pool.chain_info(c) for c in ids]
    for t, (e, n) in enumerate(graphs):
        x = oracle.validate(e, n)[1]
        x, st = oracle.es_run(x, seed=500 + t, switches=30_000)
        assert np.array_equal(outs[t], x), t
        assert infos[t]["es_switches"] == 30_000


def test_chain_above_four_million_edges_with_rebuilds():
    """A chain above 2^22 edges (windows of 1024 switches); 2.4 million
    switches pass the edge set's rebuild threshold (an eighth of its slots in
    tombstones) and relaunch the chain after the set is rebuilt on the whole
    GPU."""
    n = 600_000
    edges = inputs.gnp(n, 15.0 / (n - 1), seed=24)
    assert len(edges) >= 1 << 22
    st = es_compare(edges, n, seed=8, calls=[3000, 2_400_000])
    assert st["accepted"] > 2_000_000


def test_pool_mixes_window_sizes_with_rebuilds():
    """Chains of every window size in one call, with enough switches that
    the largest ones stop for rebuilds of their edge sets on the whole GPU
    and are launched again while the small ones are done."""
    n_huge, n_big = 600_000, 1 << 17
    graphs = [(inputs.gnp(n_huge, 15.0 / (n_huge - 1), seed=25), n_huge),
              (inputs.random_simple_graph(300, 900, seed=35), 300),
              (inputs.gnp(n_big, 9.0 / (n_big - 1), seed=26), n_big),
              (inputs.random_simple_graph(6000, 20_000, seed=36), 6000),
              (inputs.random_simple_graph(40_000, 100_000, seed=37), 40_000)]
    assert len(graphs[0][0]) >= 1 << 22 and len(graphs[2][0]) >= 1 << 19
    total = sum(len(e) for e, _ in graphs)
    with gesmc.Pool(max_edges=total, max_chains=len(graphs)) as pool:
        ids = [pool.add(e, n=n, seed=600 + t) for t, (e, n) in enumerate(graphs)]
        pool.es_run(1_200_000)
        outs = [pool.edges(c) for c in ids]
    for t, (e, n) in enumerate(graphs):
        x = oracle.validate(e, n)[1]
        x, _ = oracle.es_run(x, seed=600 + t, switches=1_200_000)
        assert np.array_equal(outs[t], x), t
