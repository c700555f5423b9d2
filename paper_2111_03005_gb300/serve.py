"""Continuous batching of sampling requests over one pool of chains.

A request is a starting graph (a simple graph with the degree sequence to
sample from), a seed, and a number of global switches (rounds of Algorithm 3
of arXiv 2111.03005).  The server keeps the state of every admitted request
on the device, runs one round for all admitted requests at a time, and
between rounds

* retires the requests that have run their rounds (their edge lists are read
  back and handed to the caller), and
* admits queued requests, first come first served, while the pool has room
  for them (edges, chain slots and contiguous index ranges: the admission is
  by device-memory footprint, since the pool's memory is fixed).

A step runs as many rounds as every admitted request still needs, at most
``max_rounds_per_step``: no request leaves earlier, so no queued request
could have been admitted earlier, and the cap bounds how long a request that
arrives during a step waits for its admission.  Fewer steps mean fewer host
synchronisations and longer runs of replayed round graphs.

With size classes the server keeps one pool per class, each on its own
CUDA stream and worker thread and each on its own admission schedule, so
that the rounds of small requests run beside (not after) those of large
ones and a small request is not held for the rounds a large one needs.

A request's result does not depend on what else is in the pool: each chain
draws its permutations from its own seed and round numbers and owns its own
index ranges, so the result equals a single-chain run with the same inputs.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque
from concurrent.futures import FIRST_COMPLETED, ThreadPoolExecutor, wait

import numpy as np

from . import gesmc


@dataclasses.dataclass
class Request:
    rid: int
    edges: np.ndarray
    n: int
    seed: int
    rounds: int
    start_round: int = 0
    lazy_threshold: int = 0
    arrival: float = 0.0          # time.perf_counter() when submitted
    admitted: float | None = None
    finished: float | None = None
    result: np.ndarray | None = None
    accepted: int = 0


class _Lane:
    """One size class of requests: a pool (on its own stream), its queue,
    its admitted requests and the rounds it is running."""

    def __init__(self, max_edges: int, max_chains: int, pool_opts: dict, rounds_per_step: int,
                 round_ctas: int = 0):
        self.pool = gesmc.Pool(max_edges=max_edges, max_chains=max_chains, **pool_opts)
        if round_ctas:
            self.pool.set_round_launch(round_ctas)
        self.resident = round_ctas == gesmc.ROUND_RESIDENT
        self.max_edges = max_edges
        self.rounds_per_step = rounds_per_step
        self.queue: deque[Request] = deque()
        self.live: dict[int, tuple[Request, int]] = {}  # chain id -> (request, rounds run)
        self.rounds_run = 0
        self.running = None  # (future, rounds) while a worker runs this lane's rounds

    def admit(self, server: "Server"):
        while self.queue:
            req = self.queue[0]
            try:
                cid = self.pool.add(req.edges, n=req.n, seed=req.seed, start_round=req.start_round,
                                    lazy_threshold=req.lazy_threshold)
            except gesmc.GesmcError as err:
                if err.code == gesmc.GESMC_E_NOMEM and self.live:
                    return          # no room now: wait for a request to leave
                raise
            self.queue.popleft()
            req.admitted = time.perf_counter()
            if req.rounds == 0:
                self.retire(server, cid, req)
            else:
                self.live[cid] = (req, 0)

    def retire(self, server: "Server", cid: int, req: Request):
        req.result = self.pool.edges(cid)
        req.accepted = self.pool.chain_info(cid)["accepted"]
        req.finished = time.perf_counter()
        self.pool.remove(cid)
        server.done.append(req)

    def rounds_now(self) -> int:
        cap = self.rounds_per_step
        return min(cap, min(req.rounds - done for req, done in self.live.values())) if self.live else 0

    def advance(self, server: "Server", k: int):
        self.rounds_run += k
        for cid, (req, done) in list(self.live.items()):
            server.switches_run += k * (len(req.edges) // 2)
            if done + k == req.rounds:
                del self.live[cid]
                self.retire(server, cid, req)
            else:
                self.live[cid] = (req, done + k)

    def busy(self) -> bool:
        return bool(self.queue or self.live or self.running)


class Server:
    """Continuous batching over one pool, or over one pool per size class.

    size_classes = (b1, b2, ...) sends a request with at most b1 edges to
    the first pool, at most b2 to the second, and larger ones to the last.
    Each pool has its own CUDA stream and its own worker thread, and each
    admits, runs and retires on its own schedule: a small request waits for
    the rounds of its own class, not for those of the largest request
    admitted.  The class pools hold small_fraction of max_edges each (at
    least their bound), the last one max_edges.  Results are the same as
    with one pool (each chain's result depends only on its own inputs)."""

    def __init__(self, max_edges: int, max_chains: int, max_rounds_per_step: int = 8, size_classes=(),
                 small_fraction: float = 0.25, small_round_ctas: int = 0, small_round_max_edges: int = 1 << 17,
                 small_rounds_per_step: int | None = None, **pool_opts):
        # small_round_ctas >= 1: the pools of size classes bounded by at most
        # small_round_max_edges edges run each round as one cooperative launch
        # of that many CTAs (gesmc_pool_set_round_launch), at most
        # small_rounds_per_step rounds between admissions (default
        # max_rounds_per_step): their rounds are short, so a larger cap cuts
        # the host synchronisations per round at the same admission delay.
        # small_round_ctas = gesmc.ROUND_RESIDENT: the classes bounded by at
        # most gesmc.RESIDENT_MAX_EDGES edges run resident rounds (one CTA per
        # request, all rounds of a step in one launch); a request with more
        # than gesmc.RESIDENT_MAX_NODES nodes goes to the next class
        if small_rounds_per_step is None:
            small_rounds_per_step = max_rounds_per_step
        if max_rounds_per_step < 1 or small_rounds_per_step < 1:
            raise ValueError("max_rounds_per_step and small_rounds_per_step must be at least 1")
        self.bounds = tuple(int(b) for b in size_classes)
        if list(self.bounds) != sorted(set(self.bounds)) or any(b < 1 for b in self.bounds):
            raise ValueError("size_classes must be increasing positive edge counts")
        self.max_rounds_per_step = max_rounds_per_step
        self.lanes: list[_Lane] = []
        for b in self.bounds:
            opts = dict(pool_opts, stream=_new_stream())
            # a class of small requests runs each round as one launch (its rounds are launch-bound)
            if small_round_ctas == gesmc.ROUND_RESIDENT:
                ctas = small_round_ctas if b <= gesmc.RESIDENT_MAX_EDGES else 0
            else:
                ctas = small_round_ctas if b <= small_round_max_edges else 0
            cap = small_rounds_per_step if ctas else max_rounds_per_step
            self.lanes.append(_Lane(max(b, int(max_edges * small_fraction)), max_chains, opts, cap, ctas))
        opts = dict(pool_opts)
        if self.bounds and "stream" not in opts:
            opts["stream"] = _new_stream()
        self.lanes.append(_Lane(max_edges, max_chains, opts, max_rounds_per_step))
        self.pool = self.lanes[-1].pool  # the only pool without size classes
        self._workers = ThreadPoolExecutor(max_workers=len(self.lanes)) if len(self.lanes) > 1 else None
        self.done: list[Request] = []
        self.switches_run = 0

    @property
    def rounds_run(self) -> int:
        return max(lane.rounds_run for lane in self.lanes)

    def _lane_of(self, req: Request) -> _Lane:
        m = len(req.edges)
        for b, lane in zip(self.bounds, self.lanes):
            if m <= b and not (lane.resident and not 0 < req.n <= gesmc.RESIDENT_MAX_NODES):
                return lane
        return self.lanes[-1]

    def submit(self, req: Request, now: float | None = None):
        req.arrival = time.perf_counter() if now is None else now
        lane = self._lane_of(req)
        if len(req.edges) > lane.max_edges:
            raise ValueError(f"request {req.rid}: {len(req.edges)} edges exceed the pool's capacity")
        lane.queue.append(req)

    @property
    def pool_capacity(self) -> int:
        return self.lanes[-1].max_edges

    @property
    def live(self) -> dict:
        out = {}
        for t, lane in enumerate(self.lanes):
            out.update({(t, cid): v for cid, v in lane.live.items()})
        return out

    def step(self, timeout: float | None = None) -> list[Request]:
        """One pool: admit what fits, run the admitted requests for the same
        number of rounds, retire the finished ones.  Several pools: start
        every idle pool's next rounds on its worker, then wait (at most
        `timeout` seconds, if given) until some pool's rounds are done and
        retire its finished requests; a caller that polls with a short
        timeout admits new requests to an idle pool while another still
        runs.  Returns the requests finished in this step."""
        before = len(self.done)
        for lane in self.lanes:
            if lane.running is not None:
                continue
            lane.admit(self)
            k = lane.rounds_now()
            if k == 0:
                continue
            if self._workers is None:
                lane.pool.run(k)
                lane.advance(self, k)
            else:
                lane.running = (self._workers.submit(lane.pool.run, k), k)
        running = [lane.running[0] for lane in self.lanes if lane.running is not None]
        if running:
            wait(running, timeout=timeout, return_when=FIRST_COMPLETED)
            for lane in self.lanes:
                if lane.running is not None and lane.running[0].done():
                    future, k = lane.running
                    lane.running = None
                    future.result()
                    lane.advance(self, k)
        return self.done[before:]

    def idle(self) -> bool:
        return not any(lane.busy() for lane in self.lanes)

    def close(self):
        if self._workers is not None:
            self._workers.shutdown(wait=True)
        for lane in self.lanes:
            lane.pool.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def split_requests(requests, world: int) -> list[list]:
    """Requests split over `world` GPUs by work (edges x rounds; see
    ensemble.shard), each GPU serving its share of the stream with no
    exchange; every rank computes the same split."""
    from .ensemble import shard

    return [[requests[t] for t in part] for part in shard([len(r.edges) * r.rounds for r in requests], world)]


def serve_all(requests, **server_opts) -> dict:
    """Submit every request, serve until idle: {rid: result list}."""
    with Server(**server_opts) as srv:
        for r in requests:
            srv.submit(r)
        while not srv.idle():
            srv.step()
    return {r.rid: r.result for r in requests}


def _new_stream():
    import torch

    return torch.cuda.Stream()
