"""Autotuner for the layout choices of a pool of chains.

Two choices shape a round without changing its result:

* ``tuple_log2``: the mean number of dependency tuples per hash partition
  (log2).  Larger partitions mean fewer write frontiers for the tuple
  scatter, but more work per grouping CTA.
* ``group_log2``: the slots of the shared-memory grouping table (log2).
  Together with ``tuple_log2`` it fixes the table's load factor, and with it
  the grouping kernel's occupancy (20 bytes of shared memory per slot).

A third choice, for small problems only, is how a round is launched:
``round_ctas`` = 0 runs the round's kernels one after another (replayed from
a captured CUDA graph); ``round_ctas`` >= 1 runs the whole round in one
cooperative launch of that many CTAs (the block-count axis), which saves the
launch latency between stages that dominates the rounds of small graphs;
``round_ctas`` = ROUND_RESIDENT (when every chain is small enough) runs all
rounds of a call with one CTA per chain and the chain in shared memory.

Every chain's list after a round is the same under every setting (the
partitioning only decides where a tuple is grouped, never what is decided).
The tuner times a few rounds of the caller's own graphs (or a sample of
them) under each candidate, checks that all candidates agree on the result,
keeps the fastest, and caches the choice per device and problem class in a
JSON file (``$GESMC_TUNE_CACHE``, else ``~/.cache/gesmc/tune.json``).
"""
from __future__ import annotations

import json
import math
import os
import tempfile

import numpy as np

CANDIDATES = ((9, 10), (9, 11), (10, 11), (10, 12), (11, 11), (11, 12))
# round launches tried for problems of at most LAUNCH_TUNE_MAX_EDGES edges: the
# multi-kernel round, one-launch rounds of these CTA counts, and resident
# rounds (0xFFFFFFFF, gesmc.ROUND_RESIDENT; tried only if every chain qualifies)
ROUND_RESIDENT = 0xFFFFFFFF
RESIDENT_MAX_EDGES = 10240
RESIDENT_MAX_NODES = 65536
LAUNCH_CANDIDATES = (0, 8, 16, 32, 64, 152, ROUND_RESIDENT)
LAUNCH_TUNE_MAX_EDGES = 1 << 21


def problem_key(device: str, total_edges: int, chains: int) -> str:
    """Problem class: device name, total edges and chain count, each rounded to a power of two."""
    m2 = round(math.log2(max(total_edges, 1)))
    c2 = round(math.log2(max(chains, 1)))
    return f"{device}|edges~2^{m2}|chains~2^{c2}"


def pick(timings: dict) -> tuple:
    """The candidate with the smallest time; ties go to the earlier candidate."""
    if not timings:
        raise ValueError("no timings")
    order = list(timings)
    return min(order, key=lambda c: (timings[c], order.index(c)))


class TuneCache:
    """A JSON file mapping problem keys to the chosen setting."""

    def __init__(self, path: str | None = None):
        self.path = path or os.environ.get("GESMC_TUNE_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "gesmc", "tune.json")
        try:
            with open(self.path) as f:
                self.data = json.load(f)
        except (OSError, ValueError):
            self.data = {}

    def get(self, key: str):
        v = self.data.get(key)
        if not v:
            return None
        return int(v["tuple_log2"]), int(v["group_log2"]), int(v.get("round_ctas", 0))

    def put(self, key: str, best: tuple, timings: dict, round_ctas: int = 0, launch_timings: dict | None = None):
        self.data[key] = {"tuple_log2": best[0], "group_log2": best[1], "round_ctas": round_ctas,
                          "timings_ms": {f"{t},{g}": ms for (t, g), ms in timings.items()},
                          "launch_timings_ms": {str(c): ms for c, ms in (launch_timings or {}).items()}}
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d or ".", prefix=".tune", suffix=".json")
        with os.fdopen(fd, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def sample_graphs(graphs, seeds, max_chains: int, rng_seed: int = 0):
    """A uniform sample of at most max_chains (graph, seed) pairs, in their original order."""
    if len(graphs) <= max_chains:
        return list(graphs), list(seeds)
    idx = np.sort(np.random.default_rng(rng_seed).choice(len(graphs), size=max_chains, replace=False))
    return [graphs[i] for i in idx], [seeds[i] for i in idx]


def tune(graphs, seeds, rounds: int = 3, candidates=CANDIDATES, timer=None, cache: TuneCache | None = None,
         device: str | None = None, problem: tuple | None = None, sample_chains: int = 512,
         launch_candidates=LAUNCH_CANDIDATES) -> dict:
    """Choose (tuple_log2, group_log2) for running `graphs` (a list of
    (edges, n)) with `seeds` in one pool, and, for a problem of at most
    LAUNCH_TUNE_MAX_EDGES edges, the round launch (round_ctas).

    timer(graphs, seeds, rounds, candidate) -> (milliseconds per round, the
    first chain's list after the rounds); candidate is (tuple_log2,
    group_log2) for the layout and (tuple_log2, group_log2, round_ctas) for
    the launch.  The default runs a pool on the current CUDA device.
    problem = (total edges, chains) names the problem class for the cache
    (default: the graphs given); the timing itself uses at most
    sample_chains of the graphs.  Returns a dict with the choice, the
    timings and whether it came from the cache."""
    if timer is None:
        timer = gpu_timer
    if device is None:
        device = _device_name()
    total, chains = problem or (sum(len(e) for e, _ in graphs), len(graphs))
    key = problem_key(device, total, chains)
    if cache is not None:
        hit = cache.get(key)
        if hit is not None:
            return {"tuple_log2": hit[0], "group_log2": hit[1], "round_ctas": hit[2], "cached": True, "key": key}
    g_sample, s_sample = sample_graphs(graphs, seeds, sample_chains)
    timings, first = {}, None
    for cand in candidates:
        ms, out = timer(g_sample, s_sample, rounds, cand)
        if first is None:
            first = out
        elif not np.array_equal(first, out):
            raise RuntimeError(f"tuning candidate {cand} changed the result of a round")
        timings[cand] = ms
    best = pick(timings)
    # launch, with the chosen layout: one-launch rounds for small problems only
    # (one launch of at most a few hundred CTAs is too narrow for large
    # graphs); resident rounds whenever every chain qualifies (one CTA per
    # chain scales with the chains)
    launch_timings, round_ctas = {}, 0
    resident_ok = all(len(e) <= RESIDENT_MAX_EDGES and 0 < n <= RESIDENT_MAX_NODES for e, n in graphs)
    cands = [c for c in launch_candidates if c != ROUND_RESIDENT] if total <= LAUNCH_TUNE_MAX_EDGES else []
    if ROUND_RESIDENT in launch_candidates and resident_ok:
        cands += [0, ROUND_RESIDENT] if not cands else [ROUND_RESIDENT]
    if cands:
        for ctas in dict.fromkeys(cands):
            ms, out = timer(g_sample, s_sample, rounds, (best[0], best[1], ctas))
            if not np.array_equal(first, out):
                raise RuntimeError(f"round launch {ctas} changed the result of a round")
            launch_timings[ctas] = ms
        round_ctas = pick(launch_timings)
    if cache is not None:
        cache.put(key, best, timings, round_ctas, launch_timings)
    return {"tuple_log2": best[0], "group_log2": best[1], "round_ctas": round_ctas, "cached": False, "key": key,
            "timings_ms_per_round": {f"{t},{g}": ms for (t, g), ms in timings.items()},
            "launch_timings_ms_per_round": {str(c): ms for c, ms in launch_timings.items()},
            "sample_chains": len(g_sample)}


def _device_name() -> str:
    import torch

    return torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"


def gpu_timer(graphs, seeds, rounds: int, cand: tuple):
    """Time `rounds` rounds of all graphs in one pool with the candidate's
    layout (one warm-up round first), with CUDA events on the pool's stream."""
    import torch

    from . import gesmc

    total = sum(len(e) for e, _ in graphs)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), gesmc.Pool(max_edges=total, max_chains=len(graphs), tuple_log2=cand[0],
                                                group_log2=cand[1], stream=stream) as pool:
        ids = [pool.add(e, n=n, seed=s) for (e, n), s in zip(graphs, seeds)]
        if len(cand) > 2:
            pool.set_round_launch(cand[2])
        pool.run(1)
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        pool.run(rounds)
        stop.record(stream)
        stop.synchronize()
        out = pool.edges(ids[0])
    return start.elapsed_time(stop) / rounds, out
