"""Host logic of the serving scheduler, on the CPU: routing to size classes,
admission by capacity, lanes that run on their own schedules, and the
rounds each request gets.  The pool is a stand-in that records the rounds
each chain ran (its result is a function of its inputs and round count), so
no device is needed."""
import threading
import time

import numpy as np
import pytest

from paper_2111_03005_gb300 import gesmc, serve


def _nomem():
    err = gesmc.GesmcError.__new__(gesmc.GesmcError)
    err.code = gesmc.GESMC_E_NOMEM
    RuntimeError.__init__(err, "pool full")
    return err


class FakePool:
    """Chains with a capacity in edges and chain slots; run(k) sleeps in
    proportion to the edges held, so that lanes overlap in time."""

    instances = []

    def __init__(self, max_edges, max_chains, stream=None, **_):
        self.max_edges, self.max_chains, self.stream = max_edges, max_chains, stream
        self.chains, self.next_id, self.calls = {}, 0, []
        self.lock = threading.Lock()   # must never be contended: one thread at a time per pool
        FakePool.instances.append(self)

    def add(self, edges, n=0, seed=0, start_round=0, lazy_threshold=0):
        assert self.lock.acquire(blocking=False)
        try:
            used = sum(len(e) for e, _, _ in self.chains.values())
            if used + len(edges) > self.max_edges or len(self.chains) == self.max_chains:
                raise _nomem()
            cid = self.next_id
            self.next_id += 1
            self.chains[cid] = (edges, seed, start_round)
            self.calls.append(("add", cid))
            self.rounds = getattr(self, "rounds", {})
            self.rounds[cid] = 0
            return cid
        finally:
            self.lock.release()

    def run(self, k):
        assert self.lock.acquire(blocking=False)
        try:
            self.calls.append(("run", k))
            time.sleep(1e-7 * sum(len(e) for e, _, _ in self.chains.values()))
            for cid in self.chains:
                self.rounds[cid] += k
        finally:
            self.lock.release()
        return self

    def edges(self, cid):
        e, seed, start = self.chains[cid]
        return np.roll(e, seed + start + self.rounds[cid])

    def chain_info(self, cid):
        return {"accepted": self.rounds[cid]}

    def remove(self, cid):
        del self.chains[cid]

    def close(self):
        pass


@pytest.fixture
def fake_pool(monkeypatch):
    FakePool.instances = []
    monkeypatch.setattr(gesmc, "Pool", FakePool)
    monkeypatch.setattr(serve, "_new_stream", lambda: object())
    return FakePool


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for rid in range(count):
        m = int(np.exp(rng.uniform(np.log(50), np.log(50_000))))
        reqs.append(serve.Request(rid=rid, edges=np.arange(m, dtype=np.uint64), n=0, seed=rid,
                                  rounds=int(rng.integers(0, 12)), start_round=int(rng.integers(0, 3))))
    return reqs


def _serve(srv, reqs, timeout=None):
    nxt, steps = 0, 0
    while nxt < len(reqs) or not srv.idle():
        if nxt < len(reqs):
            srv.submit(reqs[nxt])
            nxt += 1
        srv.step(timeout)
        steps += 1
        assert steps < 100_000
    return steps


@pytest.mark.parametrize("size_classes,cap_rounds,timeout", [((), 1, None), ((), 5, None), ((1000,), 4, None),
                                                             ((300, 3000), 8, 0.0), ((300, 3000), 2, 1e-4)])
def test_every_request_runs_exactly_its_rounds(fake_pool, size_classes, cap_rounds, timeout):
    reqs = _requests(60, seed=len(size_classes) + cap_rounds)
    with serve.Server(max_edges=120_000, max_chains=6, max_rounds_per_step=cap_rounds,
                      size_classes=size_classes) as srv:
        _serve(srv, reqs, timeout)
        assert len(srv.done) == len(reqs)
        assert srv.switches_run == sum(r.rounds * (len(r.edges) // 2) for r in reqs)
    for r in reqs:
        assert np.array_equal(r.result, np.roll(r.edges, r.seed + r.start_round + r.rounds)), r.rid
        assert r.accepted == r.rounds
        assert r.finished >= r.admitted >= r.arrival
    for pool in fake_pool.instances:
        assert all(k <= cap_rounds for what, k in pool.calls if what == "run")


def test_requests_go_to_their_size_class(fake_pool):
    reqs = _requests(40, seed=5)
    with serve.Server(max_edges=200_000, max_chains=64, size_classes=(100, 2000), small_fraction=0.1) as srv:
        pools = [lane.pool for lane in srv.lanes]
        assert [p.max_edges for p in pools] == [20_000, 20_000, 200_000]
        assert len({id(p.stream) for p in pools}) == 3         # one stream per class
        for r in reqs:
            srv.submit(r)
        expect = [[r.rid for r in reqs if len(r.edges) <= 100],
                  [r.rid for r in reqs if 100 < len(r.edges) <= 2000],
                  [r.rid for r in reqs if len(r.edges) > 2000]]
        assert [[q.rid for q in lane.queue] for lane in srv.lanes] == expect
        _serve(srv, [])


def test_small_requests_do_not_wait_for_the_large_lane(fake_pool):
    """A large request runs many rounds; small ones submitted meanwhile finish
    while it is still running (one pool would have held them)."""
    big = serve.Request(rid=0, edges=np.arange(40_000, dtype=np.uint64), n=0, seed=0, rounds=60)
    small = [serve.Request(rid=1 + t, edges=np.arange(100, dtype=np.uint64), n=0, seed=t, rounds=2)
             for t in range(5)]
    with serve.Server(max_edges=100_000, max_chains=8, max_rounds_per_step=4, size_classes=(1000,)) as srv:
        srv.submit(big)
        srv.step(0.0)
        for r in small:
            srv.submit(r)
        while not all(r.finished for r in small):
            srv.step(0.0)
        assert big.finished is None
        _serve(srv, [])
    assert big.finished > max(r.finished for r in small)


def test_admission_waits_for_room(fake_pool):
    reqs = [serve.Request(rid=t, edges=np.arange(600, dtype=np.uint64), n=0, seed=t, rounds=3) for t in range(7)]
    with serve.Server(max_edges=1500, max_chains=8, max_rounds_per_step=8) as srv:
        for r in reqs:
            srv.submit(r)
        srv.step()
        assert len(srv.done) == 2 and len(srv.lanes[0].queue) == 5   # two fit, ran their rounds, left
        _serve(srv, [])
    assert [r.accepted for r in reqs] == [3] * 7


def test_oversized_request_and_bad_classes_are_refused(fake_pool):
    with serve.Server(max_edges=1000, max_chains=4, size_classes=(10,)) as srv:
        with pytest.raises(ValueError):
            srv.submit(serve.Request(rid=0, edges=np.arange(1001, dtype=np.uint64), n=0, seed=0, rounds=1))
    with pytest.raises(ValueError):
        serve.Server(max_edges=1000, max_chains=4, size_classes=(100, 10))
    with pytest.raises(ValueError):
        serve.Server(max_edges=1000, max_chains=4, max_rounds_per_step=0)


def test_resident_small_class_routing_and_rounds_cap(fake_pool, monkeypatch):
    # small_round_ctas = ROUND_RESIDENT: only classes bounded by RESIDENT_MAX_EDGES
    # run resident rounds; a request with too many nodes skips such a class;
    # resident classes take up to small_rounds_per_step rounds per step
    launches = []
    monkeypatch.setattr(FakePool, "set_round_launch", lambda self, c: launches.append((self.max_edges, c)) or c,
                        raising=False)
    R = gesmc.ROUND_RESIDENT
    with serve.Server(max_edges=200_000, max_chains=8, max_rounds_per_step=2, size_classes=(5000, 50_000),
                      small_fraction=0.1, small_round_ctas=R, small_rounds_per_step=7) as srv:
        assert [lane.resident for lane in srv.lanes] == [True, False, False]
        assert launches == [(srv.lanes[0].max_edges, R)]
        small = serve.Request(rid=0, edges=np.arange(100, dtype=np.uint64), n=500, seed=1, rounds=9)
        wide = serve.Request(rid=1, edges=np.arange(100, dtype=np.uint64), n=gesmc.RESIDENT_MAX_NODES + 1,
                             seed=2, rounds=9)
        unknown_n = serve.Request(rid=2, edges=np.arange(100, dtype=np.uint64), n=0, seed=3, rounds=9)
        assert srv._lane_of(small) is srv.lanes[0]
        assert srv._lane_of(wide) is srv.lanes[1]
        assert srv._lane_of(unknown_n) is srv.lanes[1]
        _serve(srv, [small, wide, unknown_n])
        assert len(srv.done) == 3
    runs = [[k for what, k in pool.calls if what == "run"] for pool in fake_pool.instances]
    assert runs[0] == [7, 2] and all(k <= 2 for k in runs[1])
