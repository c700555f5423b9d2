"""ORACLE -- test infrastructure only, never part of the product path.

ctypes front end of ``gesmc_oracle.cpp``, the plain sequential CPU statement
of the Global Edge Switching Markov Chain (arXiv 2111.03005, Def. 1, Def. 2,
Algorithm 3).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs
of ``bench.py`` import this package.  It never imports the CUDA library and
the CUDA library never imports it.

Every function takes and returns numpy arrays; edges are packed canonically
as ``(min << 32) | max`` in ``uint64``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gesmc_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# outcome codes of orc_edge_switch
ACCEPTED, REJECTED_LOOP, REJECTED_EXISTS = 0, 1, 2
# error codes of orc_validate / orc_run
OK, E_INVALID, E_LOOP, E_MULTI, E_RANGE, E_INVARIANT = 0, -1, -2, -3, -4, -20


class Stats(ctypes.Structure):
    _fields_ = [
        ("switches", ctypes.c_uint64),
        ("lazy", ctypes.c_uint64),
        ("accepted", ctypes.c_uint64),
        ("rejected_loop", ctypes.c_uint64),
        ("rejected_exists", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (portable, -O2)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    u64, u64p, u32p = ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32)
    lib.orc_philox4x64_10.argtypes = [u64p, u64p, u64p]
    lib.orc_philox4x64_10.restype = None
    lib.orc_perm_key.argtypes = [u64, u64, u64]
    lib.orc_perm_key.restype = u64
    lib.orc_lazy_word.argtypes = [u64, u64, u64]
    lib.orc_lazy_word.restype = u64
    lib.orc_permutation.argtypes = [u64, u64, u64, u32p]
    lib.orc_permutation.restype = None
    lib.orc_validate.argtypes = [u64p, u64, u64]
    lib.orc_validate.restype = ctypes.c_int
    lib.orc_edge_switch.argtypes = [u64p, u64, u64, u64, ctypes.c_int]
    lib.orc_edge_switch.restype = ctypes.c_int
    lib.orc_global_switch.argtypes = [u64p, u64, u32p, u64, ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(Stats)]
    lib.orc_global_switch.restype = ctypes.c_int
    lib.orc_run.argtypes = [u64p, u64, u64, u64, u64, u64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Stats), u64p]
    lib.orc_run.restype = ctypes.c_int
    lib.orc_run_rounds.argtypes = [u64p, u64, u64, u64, u64, u64, ctypes.c_int, u64p, u64p, u64]
    lib.orc_run_rounds.restype = ctypes.c_int
    lib.orc_global_switch_rounds.argtypes = [u64p, u64, u32p, u64, ctypes.POINTER(ctypes.c_uint8), u64p, u64p, u64]
    lib.orc_global_switch_rounds.restype = ctypes.c_int
    lib.orc_es_sample.argtypes = [u64, u64, u64, u64p]
    lib.orc_es_sample.restype = None
    lib.orc_es_run.argtypes = [u64p, u64, u64, u64, u64, ctypes.c_int, ctypes.POINTER(Stats)]
    lib.orc_es_run.restype = ctypes.c_int
    _lib = lib
    return lib


def _p64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _u64(edges) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(edges, dtype=np.uint64)).copy()


def pack(u, v) -> np.ndarray:
    """Canonical packed ids of the undirected edges {u, v} (Sec. 5.2)."""
    u = np.asarray(u, dtype=np.uint64)
    v = np.asarray(v, dtype=np.uint64)
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    return (lo << np.uint64(32)) | hi


def unpack(edges) -> tuple[np.ndarray, np.ndarray]:
    e = np.asarray(edges, dtype=np.uint64)
    return (e >> np.uint64(32)).astype(np.uint32), (e & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def philox4x64_10(counter, key) -> np.ndarray:
    lib = _load()
    c = np.asarray(counter, dtype=np.uint64).copy()
    k = np.asarray(key, dtype=np.uint64).copy()
    out = np.zeros(4, dtype=np.uint64)
    lib.orc_philox4x64_10(_p64(c), _p64(k), _p64(out))
    return out


def perm_key(seed: int, rnd: int, i: int) -> int:
    return int(_load().orc_perm_key(seed, rnd, i))


def lazy_word(seed: int, rnd: int, k: int) -> int:
    return int(_load().orc_lazy_word(seed, rnd, k))


def permutation(seed: int, rnd: int, m: int) -> np.ndarray:
    out = np.zeros(m, dtype=np.uint32)
    _load().orc_permutation(seed, rnd, m, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out


def validate(edges, n: int = 0) -> tuple[int, np.ndarray]:
    """Return (code, canonical copy of the list)."""
    e = _u64(edges)
    code = _load().orc_validate(_p64(e), len(e), n)
    return int(code), e


def edge_switch(edges, i: int, j: int, g: int) -> tuple[int, np.ndarray]:
    """Def. 1 on a copy of the list; returns (outcome, new list)."""
    e = _u64(edges)
    code = _load().orc_edge_switch(_p64(e), len(e), i, j, g)
    return int(code), e


def global_switch(edges, pi, ell: int | None = None, skip=None) -> tuple[np.ndarray, dict]:
    """Def. 2 with an explicit permutation (0-based) on a copy of the list."""
    e = _u64(edges)
    m = len(e)
    p = np.ascontiguousarray(np.asarray(pi, dtype=np.uint32))
    if len(p) != m:
        raise ValueError("pi must have length m")
    ell = m // 2 if ell is None else ell
    sk = None
    if skip is not None:
        sk_arr = np.ascontiguousarray(np.asarray(skip, dtype=np.uint8))
        sk = sk_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    st = Stats()
    code = _load().orc_global_switch(_p64(e), m, p.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), ell, sk,
                                     ctypes.byref(st))
    if code != 0:
        raise ValueError(f"orc_global_switch failed: {code}")
    return e, st.as_dict()


def run(edges, seed: int, rounds: int, start_round: int = 0, lazy_threshold: int = 0,
        check_every_switch: bool = False, snapshots: bool = False, exact_ell: bool = False):
    """Algorithm 3, sequentially.  Returns (final list, stats[, per-round lists])."""
    e = _u64(edges)
    m = len(e)
    st = Stats()
    snap = np.zeros((rounds, m), dtype=np.uint64) if snapshots else None
    code = _load().orc_run(_p64(e), m, seed, start_round, rounds, lazy_threshold, int(exact_ell),
                           int(check_every_switch),
                           ctypes.byref(st), _p64(snap) if snap is not None else None)
    if code != 0:
        raise ValueError(f"orc_run failed: {code}")
    if snapshots:
        return e, st.as_dict(), snap
    return e, st.as_dict()


MAX_ROUNDS_RECORDED = 64


def run_rounds(edges, seed: int, rounds: int, start_round: int = 0, lazy_threshold: int = 0,
               exact_ell: bool = False):
    """Algorithm 3 with every global switch performed by Algorithm 1's
    decide / delay rounds in Jacobi order (Sec. 4, Thm. 2's worst-case
    scheduler).  Returns (final list, rounds of each global switch,
    entering) with entering[t, w] = undecided switches entering round w of
    global switch t (w >= 1; w < MAX_ROUNDS_RECORDED)."""
    e = _u64(edges)
    w = np.zeros(rounds, dtype=np.uint64)
    ent = np.zeros((rounds, MAX_ROUNDS_RECORDED), dtype=np.uint64)
    code = _load().orc_run_rounds(_p64(e), len(e), seed, start_round, rounds, lazy_threshold, int(exact_ell),
                                  _p64(w), _p64(ent), MAX_ROUNDS_RECORDED)
    if code != 0:
        raise ValueError(f"orc_run_rounds failed: {code}")
    return e, w.astype(np.int64), ent.astype(np.int64)


def global_switch_rounds(edges, pi, ell: int | None = None, skip=None):
    """One global switch with an explicit permutation, performed by Algorithm
    1's rounds in Jacobi order.  Returns (new list, rounds, entering)."""
    e = _u64(edges)
    m = len(e)
    p = np.ascontiguousarray(np.asarray(pi, dtype=np.uint32))
    if len(p) != m:
        raise ValueError("pi must have length m")
    ell = m // 2 if ell is None else ell
    sk = None
    if skip is not None:
        sk_arr = np.ascontiguousarray(np.asarray(skip, dtype=np.uint8))
        sk = sk_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    w = np.zeros(1, dtype=np.uint64)
    ent = np.zeros(MAX_ROUNDS_RECORDED, dtype=np.uint64)
    code = _load().orc_global_switch_rounds(_p64(e), m, p.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), ell, sk,
                                            _p64(w), _p64(ent), MAX_ROUNDS_RECORDED)
    if code != 0:
        raise ValueError(f"orc_global_switch_rounds failed: {code}")
    return e, int(w[0]), ent.astype(np.int64)


def es_sample(seed: int, k: int, m: int) -> tuple[int, int, int]:
    """ES-MC switch k of a list of m >= 2 edges: (i, j, g)."""
    out = np.zeros(3, dtype=np.uint64)
    _load().orc_es_sample(seed, k, m, _p64(out))
    return int(out[0]), int(out[1]), int(out[2])


def es_run(edges, seed: int, switches: int, start_switch: int = 0, check_every_switch: bool = False):
    """ES-MC sequentially (the chain ParES parallelises).  Returns (final list, stats)."""
    e = _u64(edges)
    st = Stats()
    code = _load().orc_es_run(_p64(e), len(e), seed, start_switch, switches, int(check_every_switch),
                              ctypes.byref(st))
    if code != 0:
        raise ValueError(f"orc_es_run failed: {code}")
    return e, st.as_dict()

