"""Write ensemble_4096_digests.json: for each of the 4096 graphs of the
null-model ensemble (inputs.ensemble_graphs(4096, seed=41); chain t has seed
5000 + t), the first 16 hex digits of the SHA-256 of its list (little-endian
uint64, position order) after 50 global switches (Algorithm 3) of the
sequential oracle, and its accepted count.  The chains run one per process
(the oracle itself is single-threaded).

    python tests/golden/make_ensemble_digests.py [--workers 6]

The digest of the inputs is stored too, so that a test can tell a generator
that gave other graphs on another machine from a mismatch of the rounds."""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

COUNT, GEN_SEED, SEED0, ROUNDS = 4096, 41, 5000, 50


def list_digest(edges: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(edges, dtype="<u8").tobytes()).hexdigest()[:16]


def inputs_digest(graphs) -> str:
    h = hashlib.sha256()
    for e, n in graphs:
        h.update(np.array([n, len(e)], dtype="<u8").tobytes())
        h.update(np.ascontiguousarray(e, dtype="<u8").tobytes())
    return h.hexdigest()


def _one(job):
    sys.path.insert(0, ROOT)
    import oracle

    t, edges, seed = job
    out, st = oracle.run(edges, seed=seed, rounds=ROUNDS)
    return t, list_digest(out), int(st["accepted"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 2))
    ap.add_argument("--out", default=os.path.join(HERE, "ensemble_4096_digests.json"))
    args = ap.parse_args()
    from paper_2111_03005_gb300 import inputs

    graphs = inputs.ensemble_graphs(COUNT, seed=GEN_SEED)
    digests, accepted = [None] * COUNT, [None] * COUNT
    # largest first, so that the last jobs are short
    order = sorted(range(COUNT), key=lambda t: -len(graphs[t][0]))
    jobs = [(t, graphs[t][0], SEED0 + t) for t in order]
    t0 = time.time()
    with mp.get_context("spawn").Pool(args.workers) as pool:
        for done, (t, d, acc) in enumerate(pool.imap_unordered(_one, jobs), 1):
            digests[t], accepted[t] = d, acc
            if done % 256 == 0:
                print(f"{done} chains, {time.time() - t0:.0f} s", flush=True)
    record = {"what": "inputs.ensemble_graphs(4096, seed=41), chain t seeded 5000 + t, 50 global switches each "
                      "by the sequential oracle: SHA-256 (first 16 hex digits) of each final list, "
                      "little-endian uint64 in position order",
              "count": COUNT, "gen_seed": GEN_SEED, "seed0": SEED0, "rounds": ROUNDS,
              "edges": int(sum(len(e) for e, _ in graphs)), "inputs_sha256": inputs_digest(graphs),
              "digests": digests, "accepted": accepted}
    with open(args.out, "w") as f:
        json.dump(record, f, separators=(",", ":"))


if __name__ == "__main__":
    main()
