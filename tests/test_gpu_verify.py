"""The device-side debug check of what every round keeps (Sec. 2.1, Def. 1,
Obs. 2): a simple graph (canonical, loop-free, ids in range, no repeated
edge, so no edge id got two legal inserters) with the starting degree
sequence.  Run after every round of real chains it never fires; on lists
broken on purpose (host-side injection) it does."""
import numpy as np
import pytest

import oracle
from paper_2111_03005_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_03005_gb300 import gesmc  # noqa: E402


@pytest.mark.parametrize("case", ["gnp", "power law", "dense", "one launch"])
def test_every_round_keeps_the_invariants(case):
    if case == "power law":
        edges, n = inputs.pld_graph(5000, 2.01, 1, 500, seed=17), 5000
    elif case == "dense":
        edges, n = inputs.random_simple_graph(60, 900, seed=4), 60
    else:
        edges, n = inputs.workload_gnp_small(seed=1)
    with gesmc.Chain(edges, n=n, verify_rounds=True) as c:
        if case == "one launch":
            c.set_round_launch(16)
        c.run(6, 21)                       # each round checked on the device
        assert c.verify() == gesmc.GESMC_OK
        assert np.array_equal(c.edges(), oracle.run(edges, seed=21, rounds=6)[0])


def test_pool_chains_keep_the_invariants():
    graphs = inputs.ensemble_graphs(16, seed=41, n_lo=100, n_hi=3000)
    with gesmc.Pool(max_edges=sum(len(e) for e, _ in graphs), max_chains=len(graphs)) as pool:
        ids = [pool.add(e, n=nn, seed=300 + t) for t, (e, nn) in enumerate(graphs)]
        pool.run(5)
        assert all(pool.verify(c) == gesmc.GESMC_OK for c in ids)


def test_the_check_rejects_broken_lists():
    edges, n = inputs.workload_gnp_small(seed=1)
    ref = torch.from_numpy(edges.view(np.int64).copy()).cuda()
    after = oracle.run(edges, seed=5, rounds=3)[0]

    def check(lst, nn=n):
        return gesmc.gesmc_verify_list(torch.from_numpy(np.asarray(lst, dtype=np.uint64).view(np.int64)).cuda(),
                                       ref, nn)

    assert check(after) == gesmc.GESMC_OK              # rewired, same degrees
    bad = after.copy()
    bad[1] = bad[0]                                     # a repeated edge (two inserters of one id)
    assert check(bad) == gesmc.GESMC_E_INVARIANT
    u, v = oracle.unpack(after[:1])
    present = set(after.tolist())
    w = next(x for x in range(n) if x != u[0] and x != v[0] and int(oracle.pack(u[0], x)) not in present)
    bad = after.copy()
    bad[0] = oracle.pack(u[0], w)                       # degrees of v and w change
    assert check(bad) == gesmc.GESMC_E_INVARIANT
    bad = after.copy()
    bad[0] = (bad[0] << np.uint64(32)) | (bad[0] >> np.uint64(32))   # not canonical
    assert check(bad) == gesmc.GESMC_E_INVARIANT
    assert check(after, nn=int(oracle.unpack(after)[1].max())) == gesmc.GESMC_E_INVARIANT   # id out of range
    assert check(after[:-1]) == gesmc.GESMC_E_INVARIANT  # an edge missing
