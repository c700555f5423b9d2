#!/usr/bin/env python
"""Throughput of the G-ES-MC global switch round (arXiv 2111.03005) on GB300.

A step is one call of the public API's gesmc_run with R global switches
(Def. 2; Algorithm 3) on the workload below: R x floor(m/2) edge switches.
The metric is attempted edge switches per second.  The timed calls replay the
library's captured CUDA graph of a round (its default path); stage times come
from one more, untimed step with per-stage CUDA events.

Parity is checked on the run itself: the first warm-up step starts at round 0
with chain seed 7 and its list is compared with the sequential oracle's
(stored SHA-256 digests for G(2^24); the oracle run beside it for the small
workloads).  A mismatch ends the run with an error.

Workloads (seeded synthetic stand-ins for the paper's SynGnp / SynPld):
  gnp_2p24  (default) G(n = 2^24, p = 16/(n-1)), about 1.34e8 edges, 20 global
            switches per step; device state about 19 GB, far above the 129 MB L2
  gnp_small G(n = 1000, p = 0.01), 10 global switches per step
  pld_1m    Pld([1..1000], gamma = 2.5) on 10^6 nodes by Havel-Hakimi, 100 global
            switches per step
The two small ones fit in L2; L2 is flushed between their timed steps.

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gesmc|reference] [--workload NAME]
Under torchrun each rank runs an independent replica of the workload on its
own GPU (a single chain does not shard); value = all ranks' switches / the
slowest rank's time.  The ensemble and serving workloads split their chains
or requests over the ranks by footprint instead, with no exchange.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "edge switches/sec on 1 GB300 (bit-exact vs sequential oracle); % random-access HBM roofline"
UNIT = "edge switches/s"
CHAIN_SEED = 7
L2_FLUSH_BYTES = 512 << 20

WORKLOADS = {
    "gnp_2p24": dict(desc="G(n=2^24, p=16/(n-1)), seed 3; 20 global switches per step", n_log2=24, deg=16.0,
                     seed=3, rounds=20, digests="gnp_2p24_round_digests.json"),
    "gnp_small": dict(desc="G(n=1000, p=0.01), seed 1; 10 global switches per step", gen="gnp_small", seed=1,
                      rounds=10, oracle_rounds=10),
    "pld_1m": dict(desc="Pld([1..1000], gamma=2.5) on n=10^6 nodes, even-sum fix, Havel-Hakimi, seed 2; "
                        "100 global switches per step", gen="pld_1m", seed=2, rounds=100, oracle_rounds=20),
    "gnp_2p22": dict(desc="G(n=2^22, p=16/(n-1)), seed 4", n_log2=22, deg=16.0, seed=4, rounds=20),
    "gnp_2p20": dict(desc="G(n=2^20, p=16/(n-1)), seed 5", n_log2=20, deg=16.0, seed=5, rounds=20),
    "gnp_2p12": dict(desc="G(n=2^12, p=16/(n-1)), seed 7 (tests)", n_log2=12, deg=16.0, seed=7, rounds=20),
    "gnp_2p27": dict(desc="G(n=2^27, p=16/(n-1)), seed 6: about 1.07e9 edges, 155 GB of device state (near the "
                          "largest chain one GPU holds)", n_log2=27, deg=16.0, seed=6, rounds=20),
}
CPU_SAMPLE = "gnp_2p20"


def make_workload(name):
    from paper_2111_03005_gb300 import inputs

    w = WORKLOADS[name]
    if w.get("gen") == "gnp_small":
        return inputs.workload_gnp_small(seed=w["seed"])
    if w.get("gen") == "pld_1m":
        return inputs.workload_pld_1m(seed=w["seed"])
    n = 1 << w["n_log2"]
    return inputs.gnp(n, w["deg"] / (n - 1), w["seed"]), n


def list_digest(a) -> str:
    import hashlib

    import numpy as np

    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()


def stored_digests(name):
    w = WORKLOADS[name]
    if not w.get("digests"):
        return None
    with open(os.path.join(ROOT, "tests", "golden", w["digests"])) as f:
        return json.load(f)


# --------------------------------------------------------------------- ranks

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world, backend):
    import torch.distributed as dist

    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(value: float, dist, device=None) -> float:
    """Largest `value` over all ranks (the slowest rank's time)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self._t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------- roofline

def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def algorithmic_bytes(stage: str, m: int, L: int, nb: int, npart: int, accepted: float) -> float:
    """DRAM bytes a stage must move per round (streaming reads + writes).

    Per switch (two positions):
      permute:   read the list in slot order (2 x 12 B) and the status word (4 B),
                 write two 16-byte bucket records (their write frontiers stay in L2)
      sortpair:  read the two records (32 B); write the list in slot order (24 B),
                 the reject word (4 B), the dependency-entry pair (8 B) and append
                 the two target tuples to their hash partitions (32 B)
      sources:   read the two list edges (16 B) and the reject word (4 B); the
                 source tuples a target needs are rare in a sparse graph, and the
                 ones a filter collision lets through are not counted
      group:     read the two target tuples of the partition (32 B)
      wave1:     read the reject word, write the status word (8 B)
    The scans, the clear and the (normally empty) overflow pass move a few
    bytes per bucket or partition; the target filter stays in L2."""
    if stage == "permute":
        return 12.0 * m + 4.0 * L + 16.0 * m
    if stage == "sortpair":
        return 16.0 * m + 12.0 * m + L * (4.0 + 8.0 + 32.0)
    if stage == "sources":
        return 8.0 * m + 4.0 * L
    if stage == "group":
        return 32.0 * L
    if stage == "wave1":
        return 8.0 * L
    if stage in ("scan_perm", "clear"):
        return 12.0 * nb + 8.0 * npart
    return 0.0


def traffic_sources_sha256() -> str:
    """SHA-256 over what a round kernel's DRAM traffic depends on: the round
    kernels (round.cu), the structures and constants they share
    (gesmc_internal.cuh), and the layout code of api.cu (chain shapes,
    capacities, the target filter's size, the pieces of the allocation),
    each without its comments and blank lines."""
    import hashlib

    import re

    def code(text: str) -> bytes:  # comments and blank lines do not change a kernel
        lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.split("\n"))
        return "\n".join(ln for ln in lines if ln).encode()

    csrc = os.path.join(ROOT, "paper_2111_03005_gb300", "csrc")
    api = open(os.path.join(csrc, "api.cu")).read()
    layout = api[api.index("// Largest m:"):api.index("template <class T>\nT *at(")]
    h = hashlib.sha256()
    for part in (open(os.path.join(csrc, "round.cu")).read(), open(os.path.join(csrc, "gesmc_internal.cuh")).read(),
                 layout):
        h.update(hashlib.sha256(code(part)).digest())
    return h.hexdigest()


def traffic_from_profile(kernel: str, workload: str):
    """Measured DRAM bytes per launch of `kernel` from the committed ncu
    summary, if neither the kernels nor the layout have changed since it was
    taken (traffic_sources_sha256)."""
    path = os.path.join(ROOT, "profiles", f"traffic_{kernel}_{workload}.txt")
    try:
        kv = dict(line.split("=", 1) for line in open(path).read().split("\n") if "=" in line)
        if kv.get("sources_sha256", "").strip() != traffic_sources_sha256():
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def resident_sources_sha256() -> str:
    """SHA-256 over what the resident kernel's instruction count depends on
    (resident.cu, resident.cuh, device_util.cuh), without comments."""
    import hashlib
    import re

    def code(text: str) -> bytes:
        lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.split("\n"))
        return "\n".join(ln for ln in lines if ln).encode()

    csrc = os.path.join(ROOT, "paper_2111_03005_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("resident.cu", "resident.cuh", "device_util.cuh"):
        h.update(hashlib.sha256(code(open(os.path.join(csrc, name)).read())).digest())
    return h.hexdigest()


def resident_inst_from_profile(workload: str):
    """Warp instructions one resident round of the workload's chain executes
    (ncu, committed summary), if the kernel has not changed since."""
    path = os.path.join(ROOT, "profiles", f"inst_k_round_resident_{workload}.txt")
    try:
        kv = dict(line.split("=", 1) for line in open(path).read().split("\n") if "=" in line)
        if kv.get("sources_sha256", "").strip() != resident_sources_sha256():
            return None
        return float(kv["warp_inst_per_round"])
    except (OSError, KeyError, ValueError):
        return None


# one SM issues at most 4 warp instructions per clock (4 schedulers) at the
# maximum SM clock of 2070 MHz: the issue-rate peak of a kernel that runs a
# chain on one CTA
SM_ISSUE_PEAK_GINST = 4 * 2.070


# --------------------------------------------------------------------- CPU legs

def cpu_sample_switches_per_s():
    """The oracle, as it stands, on one host core: one global switch of the
    2^20-node sample (same degree profile as the default workload)."""
    import oracle

    edges, _ = make_workload(CPU_SAMPLE)
    oracle.build()
    t0 = time.perf_counter()
    _, st = oracle.run(edges, seed=11, rounds=1)
    dt = time.perf_counter() - t0
    return st["switches"] / dt, st["switches"], dt


def run_reference(args):
    """The reference arm: the sequential oracle, as it stands, on one host
    core, on a bounded sample of the workload per step (the default
    workload: one global switch of the 2^20-node sample with the same degree
    profile; the small workloads: their own graph, 10 rounds of G(1000, 0.01)
    or 1 round of the power law per step)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    wl = WORKLOADS[args.workload]
    if wl.get("oracle_rounds"):
        edges, n = make_workload(args.workload)
        per_step = wl["rounds"] if len(edges) < 100_000 else 1
        sample = (f"{per_step} global switch(es) per step on {wl['desc'].split(';')[0]} (m={len(edges)}), "
                  f"sequential oracle, 1 thread")
        sample_desc = wl["desc"]
    else:
        edges, n = make_workload(CPU_SAMPLE)
        per_step = 1
        sample = (f"1 global switch per step on {WORKLOADS[CPU_SAMPLE]['desc']} (m={len(edges)}), "
                  f"sequential oracle, 1 thread")
        sample_desc = WORKLOADS[CPU_SAMPLE]["desc"]
    times, done = [], 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, st = oracle.run(edges, seed=11 + step, rounds=per_step)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            done += st["switches"]
    total = sum(times)
    value = done / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl["desc"], "sample": sample_desc, "parallelism": "none (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- GPU arm

def check_parity(chain, name, edges, rounds, seed, world_rank):
    """Run the first warm-up step and compare its list with the sequential
    oracle's.  Returns the parity record and, for the small workloads, the
    oracle's time and switch count (its cpu_baseline)."""
    import numpy as np

    gold = stored_digests(name)
    w = WORKLOADS[name]
    if gold is not None:
        assert gold["chain_seed"] == seed and gold["start_round"] == 0
        assert list_digest(edges) == gold["input_sha256"], "the generator gave another graph on this machine"
        k = min(rounds, len(gold["rounds"]))
        chain.run(k, seed)
        got = list_digest(chain.edges())
        want = gold["rounds"][k - 1]["sha256"]
        if got != want:
            raise SystemExit(f"parity FAILED on rank {world_rank}: {name}, list after {k} rounds has SHA-256 {got}, "
                             f"the sequential oracle's is {want}")
        acc = sum(r["accepted"] for r in gold["rounds"][:k])
        if chain.stats()["accepted"] != acc:
            raise SystemExit(f"parity FAILED on rank {world_rank}: {name}, accepted counts differ")
        return {"checked": True, "rounds": k, "chain_seed": seed,
                "against": "stored SHA-256 of the sequential oracle's list after each round "
                           f"(tests/golden/{w['digests']})"}, None
    if w.get("oracle_rounds"):
        import oracle

        oracle.build()
        k = w["oracle_rounds"]
        t0 = time.perf_counter()
        want, st = oracle.run(edges, seed=seed, rounds=k)
        dt = time.perf_counter() - t0
        chain.run(k, seed)
        got = chain.edges()
        if not np.array_equal(got, want):
            bad = int(np.flatnonzero(got != want)[0])
            raise SystemExit(f"parity FAILED on rank {world_rank}: {name}, list after {k} rounds differs from the "
                             f"sequential oracle's at position {bad}")
        if chain.stats()["accepted"] != st["accepted"]:
            raise SystemExit(f"parity FAILED on rank {world_rank}: {name}, accepted counts differ")
        return ({"checked": True, "rounds": k, "chain_seed": seed,
                 "against": "the sequential oracle run beside it, whole list compared"},
                {"seconds": dt, "switches": st["switches"], "rounds": k})
    return {"checked": False, "why": "no stored oracle result for this workload (the parity tests cover its kernels)"}, \
        None


def run_gesmc(args):
    import numpy as np
    import torch

    from paper_2111_03005_gb300 import gesmc

    world, rank, local = dist_env()
    if world != args.gpus:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE {world}", file=sys.stderr)
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    wl = WORKLOADS[args.workload]
    rounds = wl["rounds"]
    edges, n = make_workload(args.workload)
    m, L = len(edges), len(edges) // 2
    seed = CHAIN_SEED
    state_bytes = gesmc.gesmc_device_bytes(m)
    flush_l2 = state_bytes < 4 * L2_FLUSH_BYTES
    layout = {"tuple_log2": args.tuple_log2, "group_log2": args.group_log2}
    tuning = None
    if not args.no_autotune and not (args.tuple_log2 or args.group_log2):
        # partition size and table load factor timed on this graph (3 rounds per candidate, untimed here)
        from paper_2111_03005_gb300 import autotune

        t_tune = time.perf_counter()
        tuning = autotune.tune([(edges, n)], [seed + 1], rounds=3, cache=autotune.TuneCache(args.tune_cache))
        tuning["tuning_s"] = time.perf_counter() - t_tune
        layout = {"tuple_log2": tuning["tuple_log2"], "group_log2": tuning["group_log2"]}
    # create time (the paper's timings include initialisation): validation, edge set and first layout from a
    # device-resident list; the second of two creates (the first also pays one-time driver work)
    d_edges = torch.from_numpy(edges.view(np.int64)).to(dev)
    create_ms = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with gesmc.Chain(d_edges, n=n, **layout):
            torch.cuda.synchronize()
            create_ms.append(1e3 * (time.perf_counter() - t0))
    del d_edges
    chain = gesmc.Chain(edges, n=n, **layout)
    if args.round_launch == "auto":
        want = tuning["round_ctas"] if tuning and tuning.get("round_ctas") else 0
    else:
        want = gesmc.ROUND_RESIDENT if args.round_launch == "resident" else int(args.round_launch)
    round_ctas = chain.set_round_launch(want) if want else 0
    resident = round_ctas == gesmc.ROUND_RESIDENT
    # the first warm-up step (from round 0, chain seed 7) is checked against the sequential oracle
    parity, oracle_time = check_parity(chain, args.workload, edges, rounds, seed, rank)
    for _ in range(args.warmup - 1):
        chain.run(rounds, seed)
    chain.reset_stats()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev) if flush_l2 else None
    barrier(dist)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        if flush is None:   # device state far above L2: one event pair around all steps
            start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            start.record(stream)
            for _ in range(args.steps):
                chain.run(rounds, seed)
            stop.record(stream)
            torch.cuda.synchronize()
            ms_local = start.elapsed_time(stop)
        else:               # L2-resident state: L2 flushed between steps, each step timed on its own
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            for a0, a1 in evs:
                flush.add_(1)
                a0.record(stream)
                chain.run(rounds, seed)
                a1.record(stream)
            torch.cuda.synchronize()
            ms_local = sum(a0.elapsed_time(a1) for a0, a1 in evs)
    barrier(dist)
    ms = max_over_ranks(ms_local, dist, dev)
    st = chain.stats()
    # one more step, untimed, with CUDA events between the stages of every round
    # (resident rounds have no separate stages: the step's time is the kernel's)
    chain.reset_stats()
    if resident:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        chain.run(rounds, seed)
        e1.record(stream)
        torch.cuda.synchronize()
        stage_ms, prof_rounds = {"resident": e0.elapsed_time(e1)}, rounds
    else:
        chain.set_profiling(True)
        chain.run(rounds, seed)
        chain.set_profiling(False)
        stage_ms, prof_rounds = chain.stage_times()
    chain.close()

    switches_rank = args.steps * rounds * L
    value = world * switches_rank / (ms / 1e3)

    # roofline of the dominant kernel, from its live CUDA-event time
    nb, npart = st["perm_buckets"], st["tuple_partitions"]
    acc_per_round = st["accepted"] / max(st["rounds"], 1)
    peak, peak_kind = read_peaks()
    per_stage = {k: v / max(prof_rounds, 1) for k, v in stage_ms.items()}
    dom = max(per_stage, key=per_stage.get)
    if resident:
        # the chain never leaves shared memory between rounds: the kernel is
        # bound by its SM's instruction issue, not by HBM
        ipr = resident_inst_from_profile(args.workload)
        rounds_per_s = args.steps * rounds / (ms_local / 1e3)
        achieved = ipr * rounds_per_s / 1e9 if ipr else None
        roofline = {"bound": "alu", "kernel": "k_round_resident", "achieved": achieved,
                    "peak": SM_ISSUE_PEAK_GINST, "unit": "G warp instructions/s (one SM)",
                    "frac": achieved / SM_ISSUE_PEAK_GINST if achieved else None,
                    "peak_kind": "one SM's issue rate (4 schedulers x 1 warp instruction per clock x 2070 MHz): "
                                 "the chain runs on one CTA",
                    "warp_inst_per_round": ipr, "traffic": None,
                    "timing": "the timed steps (one launch of the resident kernel per step)"}
    else:
        abytes = algorithmic_bytes(dom, m, L, nb, npart, acc_per_round)
        achieved = abytes / (per_stage[dom] / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": f"k_{dom}", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": abytes,
                    "traffic": traffic_from_profile(f"k_{dom}", args.workload),
                    "timing": "stage events of one extra untimed step (direct launches)"}
    # whole-round view: all stages' algorithmic bytes over the round time
    round_bytes = sum(algorithmic_bytes(s, m, L, nb, npart, acc_per_round) for s in per_stage)
    round_ms = sum(per_stage.values())
    hist = st["wave_hist"]
    top = max((w for w, c in enumerate(hist) if c), default=0)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl["desc"], "n": n, "m": m,
                   "global_switches_per_step": rounds, "switches_per_step": rounds * L,
                   "l2": ("L2 flushed between timed steps (%d MB written; device state %.2f GB)"
                          % (L2_FLUSH_BYTES >> 20, state_bytes / 1e9)) if flush_l2 else
                         "inputs larger than L2 (device state ~%.1f GB)" % (state_bytes / 1e9),
                   "path": ("resident rounds: one CTA keeps the chain in shared memory, all rounds of a step "
                            "in one launch" if resident else
                            f"one cooperative launch per round ({round_ctas} CTAs)" if round_ctas
                            else "captured CUDA graph of a round, replayed (the library's default)")
                           + (" (the tuner's choice)" if args.round_launch == "auto" and round_ctas else ""),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "parity": parity,
        "roofline": roofline,
        "round": {"ms": round_ms, "algorithmic_GBps": round_bytes / (round_ms / 1e3) / 1e9,
                  "stages_ms": {k: round(v, 4) for k, v in per_stage.items()}},
        "tuning": dict(layout, autotune=tuning),
        "waves": {"max": st["waves_max"], "mean": st["waves_total"] / max(st["rounds"], 1),
                  "hist": {str(w): hist[w] for w in range(1, top + 1) if hist[w]},
                  "accept_rate": st["accepted"] / max(st["switches"], 1)},
        "gpu_launches": st["kernel_launches"],
        "create_ms": {"from_device": create_ms[-1]},
    }
    clk = clocks.summary()
    line["clocks"] = clk

    if not resident:
        line["round"]["bytes_per_switch"] = round_bytes / max(L, 1)
        line["round"]["frac_of_peak"] = line["round"]["algorithmic_GBps"] / peak
        line["round"]["streaming_bound_switches_per_s"] = peak * 1e9 / (round_bytes / max(L, 1))
    if not args.no_probe:
        # random-access ceiling of this GPU (8-byte accesses over a 4 GB buffer), for context: the round is
        # laid out so that no step depends on it
        rates = {name: gesmc.gesmc_probe_random_access(4 << 30, kind, 1 << 29)
                 for name, kind in (("load", gesmc.RANDOM_LOAD), ("store", gesmc.RANDOM_STORE),
                                    ("cas", gesmc.RANDOM_CAS))}
        line["random_access"] = {
            "ceiling_per_s": {k: v for k, v in rates.items()},
            "ceiling_sector_GBps": {k: 32 * v / 1e9 for k, v in rates.items()},
        }
        # the random-access roofline of a global switch: what one round costs a design that
        # gathers the sources and probes an edge hash set at random, per switch 8 random loads
        # (2 source gathers, 2 set probes, 2 slot reads, 2 table reads), 2 table atomics,
        # 6a random writes for an accepted switch (2 set erases, 2 set inserts, 2 list writes)
        # and about 130 streaming bytes, at this GPU's measured rates
        a = line["waves"]["accept_rate"]
        t_switch = (8 / rates["load"] + 2 / rates["cas"] + 6 * a / rates["store"] + 130.0 / (peak * 1e9))
        line["random_access_roofline"] = {
            "switches_per_s": 1.0 / t_switch, "frac": value * t_switch,
            "model": "per switch: 8 random loads + 2 random atomics + 6a random writes + 130 streaming bytes",
        }
        # the L2-operation roofline of the permutation scatter: per position one cursor atomic
        # with its result and one 16-byte record store, at the rates of L2-resident random
        # atomics and stores (64 MB buffer); the kernel's live duration against that time
        l2 = {name: gesmc.gesmc_probe_random_access(64 << 20, kind, 1 << 29)
              for name, kind in (("atomic_add", gesmc.RANDOM_ATOMIC_ADD), ("store", gesmc.RANDOM_STORE),
                                 ("red", gesmc.RANDOM_RED))}
        t_perm = m * (1.0 / l2["atomic_add"] + 1.0 / l2["store"])
        if "permute" in per_stage:
            line["l2_op_roofline"] = {
                "kernel": "k_permute", "ops_per_launch": 2 * m, "bound_ms": 1e3 * t_perm,
                "achieved_ms": per_stage.get("permute"), "frac": 1e3 * t_perm / per_stage["permute"],
                "rates_per_s": l2,
                "model": "per position: one cursor atomic with return + one record store, L2-resident rates",
            }
        if "sortpair" in per_stage:
            # the sort kernel's emission: per switch two tuple-cursor atomics with return, two 16-byte
            # tuple stores and two target-filter reductions, at the same rates
            t_sort = L * (2.0 / l2["atomic_add"] + 2.0 / l2["store"] + 2.0 / l2["red"])
            line["l2_op_roofline_sortpair"] = {
                "kernel": "k_sortpair", "ops_per_launch": 6 * L, "bound_ms": 1e3 * t_sort,
                "achieved_ms": per_stage["sortpair"], "frac": 1e3 * t_sort / per_stage["sortpair"],
                "model": "per switch: two cursor atomics with return + two tuple stores + two filter reductions, "
                         "L2-resident rates (the sort in shared memory and the list's streaming stores come on top)",
            }

    # end to end through the public API from pinned host memory
    if not args.no_e2e:
        host_in = torch.from_numpy(edges.view(np.int64)).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        e2e_times, host_create, phases = [], [], []
        for step in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with gesmc.Chain(host_in, n=n, **layout) as c:
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                host_create.append(1e3 * (t1 - t0))
                if round_ctas:
                    c.set_round_launch(round_ctas)
                c.run(rounds, seed + 7)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                c.edges(host_out)
                torch.cuda.synchronize()
                t3 = time.perf_counter()
            torch.cuda.synchronize()
            e2e_times.append(time.perf_counter() - t0)
            phases.append((1e3 * (t1 - t0), 1e3 * (t2 - t1), 1e3 * (t3 - t2), 1e3 * (time.perf_counter() - t3)))
        e2e_t = max_over_ranks(statistics.median(e2e_times), dist, dev)
        line["e2e"] = {"value": world * rounds * L / e2e_t, "unit": UNIT,
                       "h2d_bytes_per_step": 8 * m, "d2h_bytes_per_step": 8 * m,
                       "includes": f"gesmc_create (H2D copy, validation) + gesmc_run({rounds}) + gesmc_edges (D2H) "
                                   "+ destroy",
                       "phases_ms": dict(zip(("create", "run", "edges", "destroy"),
                                             (round(statistics.median(x), 2) for x in zip(*phases)))),
                       "layout": layout}
        line["create_ms"]["from_pinned_host"] = statistics.median(host_create)
    if rank == 0 and world == 1 and not args.no_cpu:
        if oracle_time is not None:   # the oracle's run on this workload, done for the parity check
            line["cpu_baseline"] = {
                "value": oracle_time["switches"] / oracle_time["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"the first {oracle_time['rounds']} global switches ({oracle_time['switches']} switches) of "
                          f"this workload, {oracle_time['seconds']:.1f} s, sequential oracle, 1 thread"}
        else:
            v, sw, dt = cpu_sample_switches_per_s()
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"1 global switch ({sw} switches) on {WORKLOADS[CPU_SAMPLE]['desc']}, "
                                              f"{dt:.1f} s, sequential oracle, 1 thread"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------- ensemble and serving

def run_ensemble(args):
    """4096 chains on graphs of uneven size in one pool, 50 rounds per step,
    against one single-chain handle per graph (a sample) on the same GPU."""
    import numpy as np
    import torch

    from paper_2111_03005_gb300 import autotune, ensemble, gesmc, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    count, rounds = args.chains, 50
    all_graphs = inputs.ensemble_graphs(count, seed=41, n_hi=args.n_hi)
    # several GPUs: the chains are split by footprint, each GPU runs its share in its own pool (no exchange)
    mine = ensemble.shard([len(e) for e, _ in all_graphs], world)[rank]
    graphs = [all_graphs[t] for t in mine]
    seeds = [5000 + t for t in mine]
    count_mine = len(graphs)
    total = sum(len(e) for e, _ in graphs)
    layout, tuning = {}, None
    if args.tuple_log2 or args.group_log2:
        layout = {"tuple_log2": args.tuple_log2, "group_log2": args.group_log2}
    elif not args.no_autotune and count_mine:
        # partition size and table load factor timed on a sample of the ensemble itself
        t_tune = time.perf_counter()
        tuning = autotune.tune(graphs, seeds, rounds=3, cache=autotune.TuneCache(args.tune_cache),
                               problem=(total, count_mine), sample_chains=512)
        tuning["tuning_s"] = time.perf_counter() - t_tune
        layout = {"tuple_log2": tuning["tuple_log2"], "group_log2": tuning["group_log2"]}
    stream = torch.cuda.Stream()
    gold = None
    gold_path = os.path.join(ROOT, "tests", "golden", "ensemble_4096_digests.json")
    if count == 4096 and args.n_hi == 100_000 and os.path.exists(gold_path):
        with open(gold_path) as f:
            gold = json.load(f)
        if gold["rounds"] != rounds or gold["seed0"] != 5000 or gold["gen_seed"] != 41:
            gold = None
    with torch.cuda.stream(stream), gesmc.Pool(max_edges=max(total, 1), max_chains=max(count_mine, 1),
                                                   stream=stream, **layout) as pool:
        t0 = time.perf_counter()
        ids = [pool.add(e, n=n, seed=s) for (e, n), s in zip(graphs, seeds)]
        add_s = time.perf_counter() - t0
        if args.round_launch == "auto":
            launch = tuning["round_ctas"] if tuning and tuning.get("round_ctas") else 0
        else:
            launch = gesmc.ROUND_RESIDENT if args.round_launch == "resident" else int(args.round_launch)
        launch = pool.set_round_launch(launch) if launch else 0
        # the first warm-up step (rounds 0..49 of every chain) against the sequential oracle's stored digests
        pool.run(rounds)
        parity = {"checked": False, "why": "stored oracle digests cover the 4096-chain ensemble only"}
        if gold is None and count_mine:
            # other recipes: the sequential oracle, run here, on a sample of the chains
            import oracle

            pick = sorted(np.random.default_rng(7).choice(count_mine, size=min(6, count_mine),
                                                          replace=False).tolist())
            bad = [t for t in pick
                   if not np.array_equal(pool.edges(ids[t]), oracle.run(graphs[t][0], seed=seeds[t], rounds=rounds)[0])]
            if bad:
                raise SystemExit(f"parity FAILED: ensemble chain {mine[bad[0]]} differs from the sequential oracle")
            parity = {"checked": True, "rounds": rounds, "chains": len(pick),
                      "against": "the sequential oracle run beside it on a sample of the chains, whole lists compared"}
        if gold is not None:
            bad = [t for t, c in zip(mine, ids) if list_digest(pool.edges(c))[:16] != gold["digests"][t]]
            bad = sorted(ensemble.gather_shards(dist, {t: 1 for t in bad}))
            if bad:
                raise SystemExit(f"parity FAILED: {len(bad)} ensemble chains differ from the sequential oracle "
                                 f"after {rounds} rounds (first: chain {bad[0]})")
            parity = {"checked": True, "rounds": rounds, "chains": count,
                      "against": "stored SHA-256 of each chain's list after 50 rounds of the sequential oracle "
                                 "(tests/golden/ensemble_4096_digests.json)"}
        for _ in range(args.warmup - 1):
            pool.run(rounds)
        pool.reset_stats()
        barrier(dist)
        torch.cuda.synchronize()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clocks:
            start.record(stream)
            for _ in range(args.steps):
                pool.run(rounds)
            stop.record(stream)
            torch.cuda.synchronize()
        barrier(dist)
        ms_local = start.elapsed_time(stop)
        ms = max_over_ranks(ms_local, dist, dev)
        st = pool.stats()
        # one more step, untimed, with CUDA events between the stages of every round
        # (resident rounds have no separate stages)
        stage_ms, prof_rounds = {}, 0
        if launch != gesmc.ROUND_RESIDENT:
            pool.set_profiling(True)
            pool.run(rounds)
            stage_ms, prof_rounds = pool.stage_times()
            pool.set_profiling(False)
        del ids
    # all ranks' switches over the slowest rank's time (the shards cover every chain once)
    value = ensemble.rate_over_ranks(dist, args.steps * rounds * sum(len(e) // 2 for e, _ in graphs), ms_local / 1e3,
                                     device=dev)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    # the per-graph alternative on a sample of this GPU's chains, and bit-exactness of the two
    rng = np.random.default_rng(3)
    sample = sorted(rng.choice(count_mine, size=min(args.sample, count_mine), replace=False).tolist())
    sub = [graphs[t] for t in sample]
    sub_seeds = [seeds[t] for t in sample]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    alone = ensemble.run_one_by_one(sub, sub_seeds, rounds)
    torch.cuda.synchronize()
    one_by_one_s = time.perf_counter() - t0
    pooled = ensemble.run_pool(sub, sub_seeds, rounds, **layout)
    L_sub = sum(len(e) // 2 for e, _ in sub)
    per_graph = rounds * L_sub / one_by_one_s
    line = {
        "metric": "edge switches/sec, batched ensemble of chains (one pool, bit-exact per chain)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"{count} chains, n log-uniform in [100, {'1e5' if args.n_hi == 100_000 else args.n_hi}], "
                               f"half G(n, 8/(n-1)), half "
                               f"Pld([1..n^(1/(gamma-1))], gamma ~ U[2.2, 3.0]) by Havel-Hakimi; "
                               f"{rounds} global switches per step", "chains": count,
                   "edges": sum(len(e) for e, _ in all_graphs),
                   "round_launch": ("resident rounds (one CTA per chain, all rounds of a step in one launch)"
                                    if launch == gesmc.ROUND_RESIDENT else
                                    f"one cooperative launch per round ({launch} CTAs)" if launch else
                                    "captured CUDA graph of the multi-kernel round, replayed"),
                   "parallelism": "single GPU" if world == 1 else
                   f"chains split by footprint over {world} GPUs (rank 0: {count_mine} chains, {total} edges)"},
        "parity": parity,
        "per_graph_handles": {"value": per_graph, "unit": UNIT, "sample_chains": len(sample),
                              "includes": "create + run + edges per graph, one after another"},
        "autotune": tuning,
        "stages_ms_per_round": {k: round(v / max(prof_rounds, 1), 4) for k, v in stage_ms.items()},
        "speedup_vs_per_graph": value / per_graph,
        "identical_results_on_sample": ensemble.same_results(pooled, alone),
        "pool_add_s": add_s,
        "gpu_launches": st["kernel_launches"],
        "waves": {"max": st["waves_max"], "mean": st["waves_total"] / max(st["rounds"], 1)},
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_serve(args):
    """A Poisson stream of sampling requests served by continuous batching,
    at each arrival rate of --rates (requests/s), one JSON line per rate.
    The mean request is about 1.9e7 switches, so about 95 requests/s
    saturate one GPU; the defaults are 0.5x and 0.8x of that and an
    overload burst.  On several GPUs each serves the requests the footprint
    split gives it (edges x rounds), with no exchange."""
    import numpy as np
    import torch

    from paper_2111_03005_gb300 import ensemble, gesmc, inputs, serve

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    rng = np.random.default_rng(17)
    base = []
    for rid in range(args.requests):
        m_target = int(np.exp(rng.uniform(np.log(1e3), np.log(1e7))))
        e, n = inputs.request_graph(m_target, seed=rid)
        base.append((e, n, 100 + rid, int(rng.integers(10, 101))))
    unit_gaps = rng.exponential(1.0, size=len(base))
    work = sum(r * (len(e) // 2) for e, _, _, r in base)
    cap = max(args.pool_edges, max(len(e) for e, _, _, _ in base))
    mine = [r.rid for r in serve.split_requests(
        [serve.Request(rid=rid, edges=e, n=n, seed=sd, rounds=r) for rid, (e, n, sd, r) in enumerate(base)],
        world)[rank]]
    # the plain alternative: one handle per request, first come first served on this GPU (service times
    # do not depend on the arrival rate)
    svc, alone = {}, {}
    for rid in mine:
        e, n, seed, rounds = base[rid]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        with gesmc.Chain(e, n=n) as c:
            c.run(rounds, seed)
            alone[rid] = c.edges()
        svc[rid] = time.perf_counter() - t1
    stream = torch.cuda.Stream()
    classes = tuple(int(float(x)) for x in args.size_classes.split(",") if x.strip())
    small_ctas = gesmc.ROUND_RESIDENT if args.small_round_ctas == "resident" else int(args.small_round_ctas)
    poll = 2e-4 if classes else None   # with several pools, admit to an idle one while another runs
    for rate in [float(x) for x in args.rates.split(",")]:
        offsets_all = (np.cumsum(unit_gaps) - unit_gaps[0]) / rate
        reqs = [serve.Request(rid=rid, edges=base[rid][0], n=base[rid][1], seed=base[rid][2], rounds=base[rid][3])
                for rid in mine]
        offsets = [offsets_all[rid] for rid in mine]
        with torch.cuda.stream(stream), serve.Server(max_edges=cap, max_chains=args.pool_chains,
                                                     max_rounds_per_step=args.rounds_per_step,
                                                     size_classes=classes, small_round_ctas=small_ctas,
                                                     small_rounds_per_step=args.small_rounds_per_step or None,
                                                     stream=stream) as srv:
            # warm the kernels of every pool once (one request each, not counted)
            warmed = set()
            for r in reqs:
                lane = id(srv._lane_of(r))
                if lane not in warmed:
                    warmed.add(lane)
                    srv.submit(serve.Request(rid=-1, edges=r.edges, n=r.n, seed=1, rounds=3))
            while not srv.idle():
                srv.step()
            srv.done.clear()
            barrier(dist)
            t0 = time.perf_counter()
            nxt = 0
            while nxt < len(reqs) or not srv.idle():
                now = time.perf_counter() - t0
                while nxt < len(reqs) and offsets[nxt] <= now:
                    srv.submit(reqs[nxt], now=t0 + offsets[nxt])
                    nxt += 1
                if srv.idle():
                    time.sleep(max(0.0, min(0.01, offsets[nxt] - now)) if nxt < len(reqs) else 0)
                    continue
                srv.step(poll)
            wall = time.perf_counter() - t0
            rounds_run = srv.rounds_run
        for r in reqs:
            assert np.array_equal(alone[r.rid], r.result), f"request {r.rid}: served result differs from its single run"
        wall = max_over_ranks(wall, dist, torch.device("cuda", local))
        # this GPU's first-come-first-served queue of single handles over its requests
        fifo_mine, free_at = [], 0.0
        for rid, off in zip(mine, offsets):
            free_at = max(free_at, off) + svc[rid]
            fifo_mine.append((rid, free_at - off, free_at))
        mine_lat = [(r.rid, r.finished - r.arrival) for r in reqs]
        if dist is not None:   # gathered for the report only
            got_lat, got_fifo = [None] * world, [None] * world
            dist.all_gather_object(got_lat, mine_lat)
            dist.all_gather_object(got_fifo, fifo_mine)
            mine_lat = [x for part in got_lat for x in part]
            fifo_mine = [x for part in got_fifo for x in part]
        if rank != 0:
            continue
        lat_by = dict(mine_lat)
        fifo_by = {rid: f for rid, f, _ in fifo_mine}
        order = sorted(lat_by)
        lat = np.array([lat_by[rid] for rid in order])
        fifo = np.array([fifo_by[rid] for rid in order])
        small = np.array([len(base[rid][0]) <= 100_000 for rid in order])
        fifo_wall = max(end for _, _, end in fifo_mine)
        line = {
            "metric": "sampling service: aggregate edge switches/sec with continuous batching",
            "value": work / wall, "unit": UNIT, "n_gpus": world, "steps": len(base), "warmup": 1,
            "ms_per_step": 1e3 * wall / len(base), "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"{len(base)} requests, Poisson arrivals at {rate}/s, power-law graphs with "
                                   f"m log-uniform in [1e3, 1e7], 10-100 global switches each",
                       "pool_edges": cap, "pool_chains": args.pool_chains, "total_switches": work,
                       "max_rounds_per_step": args.rounds_per_step,
                       "size_classes": list(classes),
                       "small_round_ctas": args.small_round_ctas,
                       "small_rounds_per_step": args.small_rounds_per_step or args.rounds_per_step,
                       "parallelism": "single GPU" if world == 1 else
                       f"requests split by edges x rounds over {world} GPUs"},
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max()),
                          "p50_small_requests": float(np.percentile(lat[small], 50)) if small.any() else None},
            "per_request_handles_fifo": {
                "value": work / fifo_wall,
                "latency_s": {"p50": float(np.percentile(fifo, 50)), "p99": float(np.percentile(fifo, 99)),
                              "p50_small_requests": float(np.percentile(fifo[small], 50)) if small.any() else None}},
            "identical_to_single_runs": True,
            "rounds_run": rounds_run,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _launch_name(k: str) -> str:
    if k == "0":
        return "multi-kernel (graph replay)"
    if k == "resident":
        return "resident (one CTA, all rounds of a call in one launch)"
    return f"one launch, {k} CTAs"


def run_round_latency(args):
    """Time of one round of a small chain alone (G(2500, 8/(n-1)), about 1e4
    edges), 200 rounds per step: the multi-kernel round (replayed graph)
    against the one-launch round at several CTA counts, bit-exact against
    each other and the oracle."""
    import numpy as np
    import torch

    import oracle
    from paper_2111_03005_gb300 import gesmc, inputs

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = 2500
    edges = inputs.gnp(n, 8.0 / (n - 1), 21)
    rounds = 200
    results, lists = {}, {}
    want, _ = oracle.run(edges, seed=CHAIN_SEED, rounds=rounds)
    modes = [gesmc.ROUND_RESIDENT if x.strip() == "resident" else int(x) for x in args.launch_modes.split(",")]
    for ctas in modes:
        with gesmc.Chain(edges, n=n) as c:
            used = c.set_round_launch(ctas)
            c.run(rounds, CHAIN_SEED)          # checked against the oracle
            lists[ctas] = c.edges()
            for _ in range(args.warmup - 1):
                c.run(rounds, CHAIN_SEED)
            torch.cuda.synchronize()
            start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            start.record(stream)
            for _ in range(args.steps):
                c.run(rounds, CHAIN_SEED)
            stop.record(stream)
            torch.cuda.synchronize()
            results["resident" if used == gesmc.ROUND_RESIDENT else str(used)] = \
                1e3 * start.elapsed_time(stop) / (args.steps * rounds)
    exact = all(np.array_equal(v, want) for v in lists.values())
    if not exact:
        raise SystemExit("parity FAILED: a round launch differs from the sequential oracle")
    best = min(results, key=results.get)
    line = {
        "metric": "time of one global switch of a small chain alone on the GPU", "value": results[best],
        "unit": "us per round", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": results[best] * rounds / 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"G(n={n}, p=8/(n-1)), seed 21, m={len(edges)}; {rounds} global switches per step"},
        "us_per_round": {_launch_name(k): v for k, v in results.items()},
        "best": _launch_name(best),
        "parity": {"checked": True, "rounds": rounds, "against": "the sequential oracle, every launch mode"},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_es(args):
    """ParES (Algorithm 2): ES-MC switches with the sequential outcome, on one
    chain (one CTA) and on a pool of chains (one CTA each), next to the
    sequential oracle on one host core."""
    import numpy as np
    import torch

    import oracle
    from paper_2111_03005_gb300 import gesmc, inputs

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    # one chain: G(2^20, 16/(n-1)), m switches per step
    edges, n = make_workload("gnp_2p20")
    m = len(edges)
    per_step = m
    with gesmc.Chain(edges, n=n) as c:
        for _ in range(args.warmup):
            c.es_run(per_step // 16, 3)
        c.reset_stats()
        torch.cuda.synchronize()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clocks:
            start.record(stream)
            for _ in range(args.steps):
                c.es_run(per_step, 3)
            stop.record(stream)
            torch.cuda.synchronize()
        ms = start.elapsed_time(stop)
        st = c.stats()
    single = args.steps * per_step / (ms / 1e3)
    # a pool: 4096 chains of the ensemble recipe, m_t switches each per step
    graphs = inputs.ensemble_graphs(args.chains, seed=41)
    total = sum(len(e) for e, _ in graphs)
    sw = 20_000
    with gesmc.Pool(max_edges=total, max_chains=len(graphs)) as pool:
        for t, (e, nn) in enumerate(graphs):
            pool.add(e, n=nn, seed=9000 + t)
        pool.es_run(1000)
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(args.steps):
            pool.es_run(sw)
        stop.record(stream)
        torch.cuda.synchronize()
        pms = start.elapsed_time(stop)
        pst = pool.stats()
    pooled = args.steps * sw * len(graphs) / (pms / 1e3)
    # the sequential oracle on a sample
    oracle.build()
    t0 = time.perf_counter()
    _, ost = oracle.es_run(edges, seed=3, switches=2_000_000)
    cpu = ost["switches"] / (time.perf_counter() - t0)
    line = {
        "metric": "ES-MC edge switches/sec (ParES, bit-exact vs sequential ES-MC)",
        "value": single, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"{WORKLOADS['gnp_2p20']['desc']}, m switches per step, one chain",
                   "m": m, "switches_per_step": per_step},
        "accept_rate": st["accepted"] / max(st["switches"], 1),
        "pool": {"value": pooled, "unit": UNIT, "chains": len(graphs), "edges": total,
                 "switches_per_chain_per_step": sw, "ms_per_step": pms / args.steps,
                 "accept_rate": pst["accepted"] / max(pst["switches"], 1)},
        "cpu_baseline": {"value": cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"2e6 sequential ES-MC switches on {WORKLOADS['gnp_2p20']['desc']}"},
        "clocks": clocks.summary(),
        "gpu_launches": st["kernel_launches"],
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    global CPU_SAMPLE
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gesmc", "reference"], default="gesmc")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["ensemble", "serve", "es", "round_latency"],
                    default="gnp_2p24")
    ap.add_argument("--chains", type=int, default=4096, help="ensemble: chains")
    ap.add_argument("--n-hi", type=int, default=100_000, help="ensemble: largest n of the log-uniform node counts")
    ap.add_argument("--sample", type=int, default=256, help="ensemble: chains run one by one for comparison")
    ap.add_argument("--requests", type=int, default=128, help="serve: requests")
    ap.add_argument("--rates", default="48,76,400", help="serve: arrival rates (requests/s), comma-separated")
    ap.add_argument("--pool-edges", type=int, default=40_000_000, help="serve: pool capacity in edges")
    ap.add_argument("--pool-chains", type=int, default=256, help="serve: pool capacity in chains")
    ap.add_argument("--rounds-per-step", type=int, default=8, help="serve: most rounds between admissions")
    ap.add_argument("--size-classes", default="",
                    help="serve: edge-count bounds of the size classes (one pool each), comma-separated")
    ap.add_argument("--launch-modes", default="0,1,4,8,16,32,64,152,resident",
                    help="round_latency: round launches to time (0: multi-kernel; k: one launch of k CTAs; "
                         "resident: one CTA per chain for all rounds of a call)")
    ap.add_argument("--round-launch", default="auto",
                    help="chain workloads: how a round is launched (auto: the tuner's choice; 0: multi-kernel; "
                         "k: one launch of k CTAs; resident: one CTA per chain for all rounds of a step)")
    ap.add_argument("--small-round-ctas", default="0",
                    help="serve: one-launch rounds with this many CTAs for size classes of at most 2^17 edges, "
                         "or 'resident': resident rounds for size classes of at most 10,240 edges")
    ap.add_argument("--small-rounds-per-step", type=int, default=0,
                    help="serve: most rounds between admissions in the one-launch size classes (0: --rounds-per-step)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-probe", action="store_true", help="skip the random-access ceiling probe")
    ap.add_argument("--tuple-log2", type=int, default=0, help="tuning: mean tuples per partition (log2)")
    ap.add_argument("--no-autotune", action="store_true", help="default layout, no tuning")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache file")
    ap.add_argument("--group-log2", type=int, default=0, help="tuning: grouping table slots (log2)")
    ap.add_argument("--cpu-sample", choices=sorted(WORKLOADS), default=CPU_SAMPLE,
                    help="workload of the CPU (oracle) legs")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    CPU_SAMPLE = args.cpu_sample
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "es":
        return run_es(args)
    if args.workload == "round_latency":
        return run_round_latency(args)
    return run_gesmc(args)


if __name__ == "__main__":
    sys.exit(main())
