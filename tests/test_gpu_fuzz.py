"""Randomised parity: many seeded random cases, each compared bit for bit
with the sequential oracle.  Graph families (G(n, p), power law realised by
Havel-Hakimi, uniform random simple graphs, dense graphs, double stars),
sizes across bucket and partition boundaries, seeds, start rounds,
laziness in both forms, layouts, ParES calls mixed with global switches, and
pools whose chains join and leave on a random schedule.  Every case is drawn
from a fixed seed, so a failure names a case that can be rerun alone."""
import numpy as np
import pytest

import oracle
from paper_2111_03005_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_03005_gb300 import gesmc  # noqa: E402

LAYOUTS = [(0, 0), (9, 10), (10, 11), (11, 11), (11, 12)]


def random_graph(rng):
    """(edges, n) of a random family and size."""
    kind = int(rng.integers(0, 5))
    if kind == 0:
        n = int(np.exp(rng.uniform(np.log(10), np.log(20_000))))
        return inputs.gnp(n, float(rng.uniform(1.0, 12.0)) / max(n - 1, 1), int(rng.integers(1 << 30))), n
    if kind == 1:
        n = int(rng.integers(50, 6000))
        gamma = float(rng.uniform(2.0, 3.0))
        return inputs.graphical_pld_graph(n, gamma, max(2, int(n ** 0.5)), int(rng.integers(1 << 30))), n
    if kind == 2:
        n = int(rng.integers(4, 3000))
        m = int(rng.integers(0, min(6 * n, n * (n - 1) // 2) + 1))
        return inputs.random_simple_graph(n, m, int(rng.integers(1 << 30))), n
    if kind == 3:
        n = int(rng.integers(8, 70))
        m = int(rng.integers(n * (n - 1) // 4, n * (n - 1) // 2 + 1))
        return inputs.random_simple_graph(n, m, int(rng.integers(1 << 30))), n
    return inputs.double_star(int(rng.integers(2, 3000)), int(rng.integers(1 << 30)))


def lazy_setting(rng):
    """(threshold, exact_ell): none, per-switch laziness, or the exact-l form."""
    c = int(rng.integers(0, 4))
    if c <= 1:
        return 0, False
    t = int(rng.integers(1, 1 << 63))
    return t, c == 3


@pytest.mark.parametrize("block", range(12))
def test_random_single_chains(block):
    """50 cases per block: a chain, some rounds in one or several calls, against the oracle."""
    for case in range(50):
        rng = np.random.default_rng(10_000 * block + case)
        edges, n = random_graph(rng)
        seed = int(rng.integers(1 << 62))
        start = int(rng.integers(0, 6))
        lazy, exact = lazy_setting(rng)
        tl, gl = LAYOUTS[int(rng.integers(0, len(LAYOUTS)))]
        calls = [int(x) for x in rng.integers(1, 4, size=int(rng.integers(1, 4)))]
        expect = oracle.validate(edges, n)[1]
        done = 0
        with gesmc.Chain(edges, n=n, start_round=start, lazy_threshold=lazy, exact_ell=exact, tuple_log2=tl,
                         group_log2=gl, graphs=bool(rng.integers(0, 2))) as c:
            for r in calls:
                c.run(r, seed)
                expect, _ = oracle.run(expect, seed=seed, rounds=r, start_round=start + done, lazy_threshold=lazy,
                                       exact_ell=exact)
                done += r
                got = c.edges()
                bad = np.flatnonzero(got != expect)
                assert len(bad) == 0, (block, case, len(edges), done, int(bad[0]))


@pytest.mark.parametrize("block", range(8))
def test_random_pools_join_leave_and_pares(block):
    """A pool under a random schedule: chains join and leave between calls,
    global switches and ParES calls alternate; every chain is followed by
    its own oracle sequence."""
    rng = np.random.default_rng(777 + block)
    graphs = [random_graph(rng) for _ in range(24)]
    # one chain large enough for the 256-switch ParES window
    graphs.append((inputs.random_simple_graph(30_000, 70_000, int(rng.integers(1 << 30))), 30_000))
    cap_edges = sum(len(e) for e, _ in graphs)
    tl, gl = LAYOUTS[block % len(LAYOUTS)]
    with gesmc.Pool(max_edges=cap_edges, max_chains=12, tuple_log2=tl, group_log2=gl) as pool:
        live = {}       # chain id -> [graph index, expected list, seed, next round, next ES switch]
        waiting = list(range(len(graphs)))
        rng.shuffle(waiting)
        for step in range(14):
            # joins (the pool refuses when full: that chain waits)
            for _ in range(int(rng.integers(0, 5))):
                if not waiting:
                    break
                g = waiting[0]
                e, n = graphs[g]
                seed = int(rng.integers(1 << 62))
                start = int(rng.integers(0, 4))
                try:
                    cid = pool.add(e, n=n, seed=seed, start_round=start)
                except gesmc.GesmcError as err:
                    assert err.code == gesmc.GESMC_E_NOMEM
                    break
                waiting.pop(0)
                live[cid] = [g, oracle.validate(e, n)[1], seed, start, 0]
            if rng.integers(0, 3) == 0:
                k = int(rng.integers(100, 3000))
                pool.es_run(k)
                for st in live.values():
                    st[1], _ = oracle.es_run(st[1], seed=st[2], switches=k, start_switch=st[4])
                    st[4] += k
            else:
                r = int(rng.integers(1, 4))
                pool.run(r)
                for st in live.values():
                    st[1], _ = oracle.run(st[1], seed=st[2], rounds=r, start_round=st[3])
                    st[3] += r
            for cid, st in live.items():
                assert np.array_equal(pool.edges(cid), st[1]), (block, step, st[0])
            # leaves
            for cid in list(live):
                if rng.integers(0, 4) == 0:
                    pool.remove(cid)
                    waiting.append(live.pop(cid)[0])
