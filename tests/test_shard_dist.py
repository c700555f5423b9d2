"""The multi-GPU host logic of the ensemble and serving workloads, run as two
gloo ranks on the CPU with a CPU stand-in for the pool (each chain advanced
by the sequential oracle): each rank runs its share of the chains or
requests, the union of the ranks' results equals the single-rank results
chain by chain, no chain or request runs on two ranks, and the reported rate
is all ranks' switches over the slowest rank's time."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OraclePool:
    """CPU stand-in for gesmc.Pool: the same calls, each chain advanced by the
    sequential oracle (a chain's result depends only on its own inputs)."""

    runs = []

    def __init__(self, max_edges, max_chains, **_):
        self.max_edges, self.max_chains = max_edges, max_chains
        self.chains, self.next_id = {}, 0

    def add(self, edges, n=0, seed=0, start_round=0, lazy_threshold=0):
        from paper_2111_03005_gb300 import gesmc

        if sum(len(c["e"]) for c in self.chains.values()) + len(edges) > self.max_edges or \
                len(self.chains) == self.max_chains:
            err = gesmc.GesmcError.__new__(gesmc.GesmcError)
            err.code = gesmc.GESMC_E_NOMEM
            RuntimeError.__init__(err, "pool full")
            raise err
        cid = self.next_id
        self.next_id += 1
        self.chains[cid] = {"e": np.asarray(edges, dtype=np.uint64).copy(), "seed": seed, "round": start_round,
                            "lazy": lazy_threshold, "accepted": 0}
        return cid

    def run(self, k):
        import oracle

        for c in self.chains.values():
            c["e"], st = oracle.run(c["e"], seed=c["seed"], rounds=k, start_round=c["round"],
                                    lazy_threshold=c["lazy"])
            c["round"] += k
            c["accepted"] += st["accepted"]
            OraclePool.runs.append(len(c["e"]))
        return self

    def edges(self, cid):
        return self.chains[cid]["e"].copy()

    def chain_info(self, cid):
        return {"accepted": self.chains[cid]["accepted"]}

    def remove(self, cid):
        del self.chains[cid]

    def close(self):
        pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ensemble():
    from paper_2111_03005_gb300 import inputs

    graphs = inputs.ensemble_graphs(24, seed=41, n_lo=100, n_hi=2000)
    return graphs, [5000 + t for t in range(len(graphs))]


def _requests():
    from paper_2111_03005_gb300 import inputs, serve

    rng = np.random.default_rng(3)
    reqs = []
    for rid in range(14):
        e, n = inputs.request_graph(int(rng.integers(300, 3000)), seed=rid)
        reqs.append(serve.Request(rid=rid, edges=e, n=n, seed=100 + rid, rounds=int(rng.integers(1, 5))))
    return reqs


def _worker(rank, world, port, q):
    import time

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist

    from paper_2111_03005_gb300 import ensemble, gesmc, serve
    from test_shard_dist import OraclePool

    gesmc.Pool = OraclePool   # this rank's "GPU" is the CPU stand-in
    dist.init_process_group("gloo", rank=rank, world_size=world)
    graphs, seeds = _ensemble()
    t0 = time.perf_counter()
    local = ensemble.run_shard(graphs, seeds, rounds=3, rank=rank, world=world)
    dt = time.perf_counter() + 0.05 * rank - t0     # rank 1 reports itself slower
    switches = sum(3 * (len(graphs[t][0]) // 2) for t in local)
    merged = ensemble.gather_shards(dist, local)
    rate = ensemble.rate_over_ranks(dist, switches, dt)
    reqs = _requests()
    mine = serve.split_requests(reqs, world)[rank]
    served = serve.serve_all(mine, max_edges=20_000, max_chains=8)
    served_all = ensemble.gather_shards(dist, served)
    q.put((rank, sorted(local), switches, dt, rate, {t: v.tobytes() for t, v in merged.items()},
           sorted(served), {r: v.tobytes() for r, v in served_all.items()}))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_ensemble_and_requests(monkeypatch):
    import torch.multiprocessing as mp

    from paper_2111_03005_gb300 import ensemble, gesmc, serve

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, own0, sw0, dt0, rate0, merged0, srv0, sall0), (_, own1, sw1, dt1, rate1, merged1, srv1, sall1) = res
    graphs, seeds = _ensemble()
    # every chain on exactly one rank, and both ranks did work
    assert not set(own0) & set(own1) and sorted(own0 + own1) == list(range(len(graphs)))
    assert own0 and own1
    # the rate: all ranks' switches over the slowest rank's time, the same on both ranks
    assert rate0 == rate1 == pytest.approx((sw0 + sw1) / max(dt0, dt1))
    # the union equals the single-rank run, chain by chain
    monkeypatch.setattr(gesmc, "Pool", OraclePool)
    single = ensemble.run_shard(graphs, seeds, rounds=3, rank=0, world=1)
    assert merged0 == merged1 == {t: v.tobytes() for t, v in single.items()}
    # requests: each served once, the union equals one server over all requests
    reqs = _requests()
    assert not set(srv0) & set(srv1) and sorted(srv0 + srv1) == [r.rid for r in reqs]
    alone = serve.serve_all(_requests(), max_edges=20_000, max_chains=8)
    assert sall0 == sall1 == {r: v.tobytes() for r, v in alone.items()}
