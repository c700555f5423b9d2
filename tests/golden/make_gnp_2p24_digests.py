"""Write gnp_2p24_round_digests.json: SHA-256 digests of the edge list (in
position order, little-endian uint64) after each of 20 global switches
(Algorithm 3) on G(n = 2^24, p = 16/(n-1)), computed by the sequential oracle
alone.  One round of the oracle at this size takes a few minutes on one core,
so the GPU test compares its lists with these digests instead of running the
oracle.

    python tests/golden/make_gnp_2p24_digests.py [--rounds 20]

The input's own digest is stored too: the test checks it first, so that a
generator that gave a different graph on another machine is reported as such
rather than as a round mismatch."""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2111_03005_gb300 import inputs  # noqa: E402

GEN_SEED = 3
CHAIN_SEED = 7


def digest(edges: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(edges, dtype="<u8").tobytes()).hexdigest()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rounds", type=int, default=20)
    ap.add_argument("--out", default=os.path.join(HERE, "gnp_2p24_round_digests.json"))
    args = ap.parse_args()
    edges, n = inputs.workload_gnp_2p24(seed=GEN_SEED)
    record = {"what": "G(n=2^24, p=16/(n-1)) from inputs.workload_gnp_2p24; SHA-256 of the list "
                      "(little-endian uint64, position order) after each global switch of the sequential oracle",
              "n": n, "gen_seed": GEN_SEED, "m": int(len(edges)), "input_sha256": digest(edges),
              "chain_seed": CHAIN_SEED, "start_round": 0, "rounds": []}
    for r in range(args.rounds):
        t = time.time()
        edges, st = oracle.run(edges, seed=CHAIN_SEED, rounds=1, start_round=r)
        record["rounds"].append({"round": r, "sha256": digest(edges), "accepted": int(st["accepted"]),
                                 "rejected_exists": int(st["rejected_exists"])})
        print(f"round {r}: {time.time() - t:.0f} s, accepted {st['accepted']}", flush=True)
        with open(args.out + ".tmp", "w") as f:       # keep what is done if the run is cut short
            json.dump(record, f, indent=1)
    os.replace(args.out + ".tmp", args.out)


if __name__ == "__main__":
    main()
