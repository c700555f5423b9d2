"""Ensembles: many independent chains (e.g. a null-model ensemble of graphs of
uneven size) advanced together in one pool, one set of kernels per round for
all of them, against the plain alternative of one handle per graph."""
from __future__ import annotations

import numpy as np

from . import gesmc


def shard(sizes, world: int) -> list[list[int]]:
    """Split chains (their edge counts) over `world` GPUs by device
    footprint, which grows with the edges: largest first, each to the GPU
    with the fewest edges so far (ties to the lower rank).  Chains are
    independent, so the shards need no exchange; each keeps its chains in
    their original order.  Deterministic, so every rank computes the same
    split on its own."""
    if world < 1:
        raise ValueError("world must be at least 1")
    load = [0] * world
    owner = [0] * len(sizes)
    for t in sorted(range(len(sizes)), key=lambda t: (-int(sizes[t]), t)):
        r = min(range(world), key=lambda r: (load[r], r))
        owner[t] = r
        load[r] += int(sizes[t])
    return [[t for t in range(len(sizes)) if owner[t] == r] for r in range(world)]


def run_shard(graphs, seeds, rounds: int, rank: int, world: int, start_round: int = 0, **pool_opts) -> dict:
    """This GPU's share of an ensemble (shard() by edges), all in one pool
    for `rounds` rounds: {index of the chain in `graphs`: final list}."""
    mine = shard([len(e) for e, _ in graphs], world)[rank]
    if not mine:
        return {}
    lists = run_pool([graphs[t] for t in mine], [seeds[t] for t in mine], rounds, start_round, **pool_opts)
    return dict(zip(mine, lists))


def gather_shards(dist, local: dict) -> dict:
    """The union of every rank's {chain index: result}, on every rank; a chain
    reported by two ranks is an error (each chain runs on one GPU only)."""
    if dist is None:
        return dict(local)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, local)
    out = {}
    for part in parts:
        for t, v in part.items():
            if t in out:
                raise RuntimeError(f"chain {t} was run by two ranks")
            out[t] = v
    return out


def rate_over_ranks(dist, switches_local: float, seconds_local: float, device=None) -> float:
    """Whole-job rate: every rank's switches over the slowest rank's time
    (`device`: where the process group's backend takes its tensors)."""
    if dist is None:
        return switches_local / seconds_local
    import torch

    t = torch.tensor([switches_local, seconds_local], dtype=torch.float64, device=device)
    parts = [torch.zeros_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, t)
    return float(sum(p[0] for p in parts)) / float(max(p[1] for p in parts))


def run_pool(graphs, seeds, rounds: int, start_round: int = 0, **pool_opts):
    """All graphs in one pool for `rounds` rounds; returns the final lists."""
    total = sum(len(e) for e, _ in graphs)
    with gesmc.Pool(max_edges=total, max_chains=len(graphs), **pool_opts) as pool:
        ids = [pool.add(e, n=n, seed=s, start_round=start_round) for (e, n), s in zip(graphs, seeds)]
        pool.run(rounds)
        return [pool.edges(c) for c in ids]


def run_one_by_one(graphs, seeds, rounds: int, start_round: int = 0, **chain_opts):
    """The per-graph alternative: one single-chain handle per graph."""
    out = []
    for (e, n), s in zip(graphs, seeds):
        with gesmc.Chain(e, n=n, start_round=start_round, **chain_opts) as c:
            c.run(rounds, s)
            out.append(c.edges())
    return out


def same_results(a, b) -> bool:
    return len(a) == len(b) and all(np.array_equal(x, y) for x, y in zip(a, b))
