"""Seeded synthetic starting graphs (inputs only; none of the method's arithmetic).

These stand in for the paper's SynGnp and SynPld datasets (arXiv 2111.03005,
Sec. 6: G(n, p) graphs, and Pld([1..Delta], gamma) degree sequences realised
by Havel-Hakimi).  The paper's NetRep graphs are not available here.  Both the
CUDA library (through its tests and ``bench.py``) and the CPU oracle receive
exactly the arrays produced here.

Edges are ``numpy.uint64`` packed canonically as ``(min << 32) | max``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    u32, u64, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
    u64p, u32p = ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32)
    lib.gen_gnp.argtypes = [u32, dbl, u64, u64p, u64]
    lib.gen_gnp.restype = u64
    lib.gen_pld_degrees.argtypes = [u32, u32, u32, dbl, u64, u32p]
    lib.gen_pld_degrees.restype = ctypes.c_int
    lib.gen_is_graphical.argtypes = [u32p, u32]
    lib.gen_is_graphical.restype = ctypes.c_int
    lib.gen_havel_hakimi.argtypes = [u32p, u32, u64p]
    lib.gen_havel_hakimi.restype = ctypes.c_int64
    _lib = lib
    return lib


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def gnp(n: int, p: float, seed: int) -> np.ndarray:
    """G(n, p): each pair independently with probability p (SynGnp)."""
    lib = _load()
    guess = int(p * n * (n - 1) / 2 * 1.01 + 64 * (p * n * n) ** 0.5 + 1024)
    out = np.empty(guess, dtype=np.uint64)
    m = int(lib.gen_gnp(n, p, seed, _p64(out), guess))
    if m > guess:
        out = np.empty(m, dtype=np.uint64)
        m2 = int(lib.gen_gnp(n, p, seed, _p64(out), m))
        assert m2 == m
    return out[:m].copy()


def pld_degrees(n: int, gamma: float, dmin: int, dmax: int, seed: int) -> np.ndarray:
    """n i.i.d. degrees from Pld([dmin..dmax], gamma)."""
    deg = np.empty(n, dtype=np.uint32)
    rc = _load().gen_pld_degrees(n, dmin, dmax, gamma, seed, _p32(deg))
    if rc != 0:
        raise ValueError(f"gen_pld_degrees failed: {rc}")
    return deg


def make_even(deg: np.ndarray) -> np.ndarray:
    """Fix an odd degree sum by decrementing the first node of maximum degree."""
    deg = deg.copy()
    if int(deg.sum(dtype=np.uint64)) % 2 == 1:
        deg[int(np.argmax(deg))] -= 1
    return deg


def is_graphical(deg: np.ndarray) -> bool:
    d = np.ascontiguousarray(deg, dtype=np.uint32)
    rc = _load().gen_is_graphical(_p32(d), len(d))
    if rc < 0:
        raise MemoryError("gen_is_graphical")
    return bool(rc)


def havel_hakimi(deg: np.ndarray) -> np.ndarray:
    """A simple graph with exactly this degree sequence (Havel-Hakimi)."""
    d = np.ascontiguousarray(deg, dtype=np.uint32)
    total = int(d.sum(dtype=np.uint64))
    out = np.empty(max(total // 2, 1), dtype=np.uint64)
    m = int(_load().gen_havel_hakimi(_p32(d), len(d), _p64(out)))
    if m < 0:
        raise ValueError("degree sequence is not graphical" if m == -1 else "allocation failure")
    return out[:m].copy()


def pld_graph(n: int, gamma: float, dmin: int, dmax: int, seed: int) -> np.ndarray:
    """SynPld: Pld degrees, even-sum fix, Erdos-Gallai check, Havel-Hakimi."""
    deg = make_even(pld_degrees(n, gamma, dmin, dmax, seed))
    if not is_graphical(deg):
        raise ValueError("sampled degree sequence is not graphical")
    return havel_hakimi(deg)


def random_simple_graph(n: int, m: int, seed: int) -> np.ndarray:
    """m distinct uniformly random edges on n nodes, in random list order (small tests)."""
    if m > n * (n - 1) // 2:
        raise ValueError("too many edges")
    rng = np.random.Generator(np.random.Philox(seed))
    seen: set[int] = set()
    out = []
    while len(out) < m:
        u, v = (int(x) for x in rng.integers(0, n, size=2))
        if u == v:
            continue
        key = (min(u, v) << 32) | max(u, v)
        if key in seen:
            continue
        seen.add(key)
        out.append(key)
    return np.array(out, dtype=np.uint64)


def shuffle_edges(edges: np.ndarray, seed: int) -> np.ndarray:
    """The same edge set in a seeded random list order."""
    rng = np.random.Generator(np.random.Philox(seed))
    return edges[rng.permutation(len(edges))].copy()


# --- the workloads the benchmark and the full-size parity tests use ---------

def workload_gnp_small(seed: int = 1) -> tuple[np.ndarray, int]:
    """G(n=1000, p=0.01): about 5k edges."""
    n = 1000
    return gnp(n, 0.01, seed), n


def workload_pld_1m(seed: int = 2) -> tuple[np.ndarray, int]:
    """Pld([1..1000], gamma=2.5) on n=1e6 nodes, realised by Havel-Hakimi."""
    n = 1_000_000
    return pld_graph(n, 2.5, 1, 1000, seed), n


def workload_gnp_2p24(seed: int = 3) -> tuple[np.ndarray, int]:
    """G(n=2^24, p=16/(n-1)): about 1.34e8 edges."""
    n = 1 << 24
    return gnp(n, 16.0 / (n - 1), seed), n


def pld_mean_degree(gamma: float, dmin: int, dmax: int) -> float:
    k = np.arange(dmin, dmax + 1, dtype=np.float64)
    w = k ** -gamma
    return float((k * w).sum() / w.sum())


def graphical_pld_graph(n: int, gamma: float, dmax: int, seed: int, tries: int = 8) -> np.ndarray:
    """pld_graph, redrawing the degrees (seed + 1, ...) until they are graphical."""
    for t in range(tries):
        try:
            return pld_graph(n, gamma, 1, dmax, seed + t)
        except ValueError:
            continue
    raise ValueError("no graphical power-law sequence drawn")


def ensemble_graphs(count: int, seed: int, n_lo: int = 100, n_hi: int = 100_000) -> list[tuple[np.ndarray, int]]:
    """A null-model ensemble of graphs of uneven size: n log-uniform in
    [n_lo, n_hi]; half G(n, 8/(n-1)), half Pld([1..Delta], gamma) with gamma
    uniform in [2.2, 3.0] and Delta = n^(1/(gamma-1)) (the paper's SynPld
    choice, Sec. 6), realised by Havel-Hakimi."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for t in range(count):
        n = int(round(float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))))
        s = int(rng.integers(0, 2**62))
        if t % 2 == 0:
            out.append((gnp(n, 8.0 / (n - 1), s), n))
        else:
            gamma = float(rng.uniform(2.2, 3.0))
            dmax = max(1, min(n - 1, int(n ** (1.0 / (gamma - 1.0)))))
            out.append((graphical_pld_graph(n, gamma, dmax, s), n))
    return out


def request_graph(m_target: int, seed: int) -> tuple[np.ndarray, int]:
    """A sampling request's starting graph: a power-law degree sequence
    (gamma uniform in [2.2, 3.0], Delta = n^(1/(gamma-1))) with n chosen so
    that the graph has about m_target edges, realised by Havel-Hakimi."""
    rng = np.random.Generator(np.random.Philox(seed))
    gamma = float(rng.uniform(2.2, 3.0))
    n = max(16, int(m_target))
    for _ in range(4):  # Delta depends on n: settle n by fixed-point steps
        dmax = max(1, min(n - 1, int(n ** (1.0 / (gamma - 1.0)))))
        n = max(16, int(round(2.0 * m_target / pld_mean_degree(gamma, 1, dmax))))
    dmax = max(1, min(n - 1, int(n ** (1.0 / (gamma - 1.0)))))
    return graphical_pld_graph(n, gamma, dmax, int(rng.integers(0, 2**62))), n


def double_star(k: int, seed: int) -> tuple[np.ndarray, int]:
    """Hubs 0 and 1 with k leaves each (leaves 2..k+1 on hub 0, k+2..2k+1 on
    hub 1), in a seeded random list order.  About a quarter of the switches
    of a round pair a hub-0 edge with a hub-1 edge in the orientation that
    proposes the edge {0, 1}, so that one edge id collects thousands of
    insert tuples: the case that fills a dependency partition."""
    a = np.concatenate([np.zeros(k, np.uint64), np.ones(k, np.uint64)])
    b = np.arange(2, 2 + 2 * k, dtype=np.uint64)
    return shuffle_edges((a << np.uint64(32)) | b, seed), 2 + 2 * k
