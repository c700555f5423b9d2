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

A request's result does not depend on what else is in the pool: each chain
draws its permutations from its own seed and round numbers and owns its own
index ranges, so the result equals a single-chain run with the same inputs.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque

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


class Server:
    def __init__(self, max_edges: int, max_chains: int, max_rounds_per_step: int = 8, **pool_opts):
        if max_rounds_per_step < 1:
            raise ValueError("max_rounds_per_step must be at least 1")
        self.pool = gesmc.Pool(max_edges=max_edges, max_chains=max_chains, **pool_opts)
        self._max_edges = max_edges
        self.max_rounds_per_step = max_rounds_per_step
        self.queue: deque[Request] = deque()
        self.live: dict[int, tuple[Request, int]] = {}  # chain id -> (request, rounds run)
        self.done: list[Request] = []
        self.rounds_run = 0
        self.switches_run = 0

    def submit(self, req: Request, now: float | None = None):
        req.arrival = time.perf_counter() if now is None else now
        if len(req.edges) > self.pool_capacity:
            raise ValueError(f"request {req.rid}: {len(req.edges)} edges exceed the pool's capacity")
        self.queue.append(req)

    @property
    def pool_capacity(self) -> int:
        return self._max_edges

    def _admit(self):
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
                self._retire(cid, req)
            else:
                self.live[cid] = (req, 0)

    def _retire(self, cid: int, req: Request):
        req.result = self.pool.edges(cid)
        req.accepted = self.pool.chain_info(cid)["accepted"]
        req.finished = time.perf_counter()
        self.pool.remove(cid)
        self.done.append(req)

    def step(self) -> list[Request]:
        """Admit what fits, run the same number of rounds (at least one) for
        every admitted request, retire the finished ones.  Returns the
        requests finished in this step."""
        before = len(self.done)
        self._admit()
        if self.live:
            k = min(self.max_rounds_per_step, min(req.rounds - done for req, done in self.live.values()))
            self.pool.run(k)
            self.rounds_run += k
            for cid, (req, done) in list(self.live.items()):
                self.switches_run += k * (len(req.edges) // 2)
                if done + k == req.rounds:
                    del self.live[cid]
                    self._retire(cid, req)
                else:
                    self.live[cid] = (req, done + k)
        return self.done[before:]

    def idle(self) -> bool:
        return not self.queue and not self.live

    def close(self):
        self.pool.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

