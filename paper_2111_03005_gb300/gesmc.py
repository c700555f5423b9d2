"""Thin ctypes binding of libgesmc (include/gesmc.h).

The functions ``gesmc_create``, ``gesmc_run``, ``gesmc_edges``,
``gesmc_stats``, ``gesmc_reset_stats``, ``gesmc_destroy`` and
``gesmc_strerror`` mirror the C entry points one to one; ``Chain`` wraps a
handle.  Every step of a round runs in the library's CUDA kernels; this
module only marshals arguments.  PyTorch supplies the device memory (its
caching allocator, through the library's allocation hooks) and the stream
(the current torch stream).  There is no CPU fallback: if the library cannot
be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

GESMC_OK = 0
GESMC_E_INVALID = -1
GESMC_E_LOOP = -2
GESMC_E_MULTI = -3
GESMC_E_RANGE = -4
GESMC_E_NOMEM = -5
GESMC_E_CUDA = -6
GESMC_E_TABLE_FULL = -7
GESMC_E_WAVE_CAP = -8
GESMC_E_INTERNAL = -9
GESMC_E_CAPACITY = -10
GESMC_E_TOO_LARGE = -11
GESMC_E_INVARIANT = -12
FLAG_NO_GRAPHS = 1
FLAG_EXACT_ELL = 2
FLAG_TINY_OVERFLOW = 4  # fault injection for tests (see include/gesmc.h)
FLAG_VERIFY_ROUNDS = 8  # debugging: check the invariants on the device after every round
CHAIN_EXACT_ELL = 1
NOALLOC_MAX_EDGES = 65536
# round launch: every round of a call in one CTA per chain, the list in shared
# memory (chains with m <= RESIDENT_MAX_EDGES, n <= RESIDENT_MAX_NODES)
ROUND_RESIDENT = 0xFFFFFFFF
RESIDENT_MAX_EDGES = 10240
RESIDENT_MAX_NODES = 65536
WAVE_HIST = 64

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class GesmcOpts(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("lazy_threshold", ctypes.c_uint64),
        ("start_round", ctypes.c_uint64),
        ("max_waves", ctypes.c_uint32),
        ("tuple_log2", ctypes.c_uint32),
        ("group_log2", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
    ]


class GesmcStats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_uint64),
        ("switches", ctypes.c_uint64),
        ("lazy", ctypes.c_uint64),
        ("accepted", ctypes.c_uint64),
        ("rejected_loop", ctypes.c_uint64),
        ("rejected_exists", ctypes.c_uint64),
        ("kernel_launches", ctypes.c_uint64),
        ("perm_buckets", ctypes.c_uint64),
        ("tuple_partitions", ctypes.c_uint64),
        ("waves_total", ctypes.c_uint64),
        ("waves_max", ctypes.c_uint64),
        ("wave_hist", ctypes.c_uint64 * WAVE_HIST),
        ("last_round_pending", ctypes.c_uint64 * WAVE_HIST),
        ("overflow_tuples", ctypes.c_uint64),
        ("subpass_partitions", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        d = {f: int(getattr(self, f)) for f, _ in self._fields_[:11]}
        d["wave_hist"] = [int(x) for x in self.wave_hist]
        d["last_round_pending"] = [int(x) for x in self.last_round_pending]
        d["overflow_tuples"] = int(self.overflow_tuples)
        d["subpass_partitions"] = int(self.subpass_partitions)
        return d


class GesmcPoolOpts(ctypes.Structure):
    _fields_ = [
        ("max_edges", ctypes.c_uint64),
        ("max_chains", ctypes.c_uint32),
        ("max_waves", ctypes.c_uint32),
        ("tuple_log2", ctypes.c_uint32),
        ("group_log2", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
    ]


class GesmcChainInfo(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in ("m", "n", "seed", "rounds", "next_round", "switches",
                                                      "accepted", "es_switches")]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class GesmcError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {gesmc_strerror(code)} ({code})")


_lib = None
_lib_lock = threading.Lock()

# C symbols of include/gesmc.h: (name, restype, argtypes)
_SIGNATURES = [
    ("gesmc_opts_default", None, [ctypes.POINTER(GesmcOpts)]),
    ("gesmc_create", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(GesmcOpts),
                                    ctypes.POINTER(ctypes.c_void_p)]),
    ("gesmc_run", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]),
    ("gesmc_es_run", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]),
    ("gesmc_edges", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_uint64)]),
    ("gesmc_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(GesmcStats)]),
    ("gesmc_reset_stats", ctypes.c_int, [ctypes.c_void_p]),
    ("gesmc_set_profiling", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("gesmc_stage_times", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_uint64)]),
    ("gesmc_stage_name", ctypes.c_char_p, [ctypes.c_int]),
    ("gesmc_next_round", ctypes.c_uint64, [ctypes.c_void_p]),
    ("gesmc_num_edges", ctypes.c_uint64, [ctypes.c_void_p]),
    ("gesmc_num_nodes", ctypes.c_uint64, [ctypes.c_void_p]),
    ("gesmc_device_bytes", ctypes.c_size_t, [ctypes.c_uint64]),
    ("gesmc_destroy", None, [ctypes.c_void_p]),
    ("gesmc_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("gesmc_run_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]),
    ("gesmc_pool_opts_default", None, [ctypes.POINTER(GesmcPoolOpts)]),
    ("gesmc_pool_device_bytes", ctypes.c_size_t, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]),
    ("gesmc_pool_create", ctypes.c_int, [ctypes.POINTER(GesmcPoolOpts), ctypes.POINTER(ctypes.c_void_p)]),
    ("gesmc_pool_destroy", None, [ctypes.c_void_p]),
    ("gesmc_pool_add", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                      ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    ("gesmc_pool_remove", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    ("gesmc_pool_run", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    ("gesmc_pool_es_run", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    ("gesmc_generate_gnp", ctypes.c_int, [ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p,
                                          ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p]),
    ("gesmc_pool_edges", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
    ("gesmc_pool_chain_info", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(GesmcChainInfo)]),
    ("gesmc_pool_num_chains", ctypes.c_uint32, [ctypes.c_void_p]),
    ("gesmc_pool_free_edges", ctypes.c_uint64, [ctypes.c_void_p]),
    ("gesmc_pool_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(GesmcStats)]),
    ("gesmc_pool_reset_stats", ctypes.c_int, [ctypes.c_void_p]),
    ("gesmc_pool_set_profiling", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("gesmc_pool_set_round_launch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32,
                                                   ctypes.POINTER(ctypes.c_uint32)]),
    ("gesmc_set_round_launch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    ("gesmc_verify", ctypes.c_int, [ctypes.c_void_p]),
    ("gesmc_pool_verify", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    ("gesmc_verify_list", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.c_uint64]),
    ("gesmc_pool_stage_times", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_uint64)]),
    # include/gesmc_microbench.h
    ("gesmc_probe_random_access", ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                                 ctypes.POINTER(ctypes.c_double)]),
]


def library_path() -> str:
    return _build.LIB


def load_library():
    """Load (building first if needed) libgesmc.so; raises if that fails."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        path = _build.build_library()
        lib = ctypes.CDLL(path)
        for name, res, args in _SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def gesmc_strerror(code: int) -> str:
    return load_library().gesmc_strerror(int(code)).decode()


def gesmc_device_bytes(m: int) -> int:
    return int(load_library().gesmc_device_bytes(m))


def _check(code: int, where: str):
    if code != GESMC_OK:
        raise GesmcError(code, where)


class _TorchAllocator:
    """Allocation hooks that route the library's device memory through torch."""

    def __init__(self, device_index: int):
        import torch

        self._torch = torch
        self._device = device_index
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, stream, _ctx):
        try:
            return int(self._torch.cuda.caching_allocator_alloc(int(nbytes), self._device, int(stream or 0)))
        except Exception:  # noqa: BLE001 -- a NULL return is the library's OOM signal
            return None

    def _free(self, ptr, _ctx):
        if ptr:
            self._torch.cuda.caching_allocator_delete(int(ptr))


def _as_edge_buffer(edges):
    """(pointer, m, on_device, keepalive) for a numpy array or torch tensor of packed ids."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(edges, torch.Tensor):
        if edges.dtype not in (torch.int64, torch.uint64):
            raise TypeError("edge tensor must be int64 or uint64 (packed ids)")
        t = edges.contiguous()
        return t.data_ptr(), t.numel(), int(t.is_cuda), t
    a = np.ascontiguousarray(np.asarray(edges, dtype=np.uint64))
    return a.ctypes.data, a.size, 0, a


def gesmc_create(edges, n: int = 0, lazy_threshold: int = 0, start_round: int = 0, max_waves: int = 0, stream=None,
                 torch_allocator: bool = True, tuple_log2: int = 0, group_log2: int = 0, graphs: bool = True,
                 exact_ell: bool = False, tiny_overflow: bool = False, verify_rounds: bool = False):
    """Create a chain handle; returns (handle, keepalive).  Raises GesmcError."""
    import torch

    lib = load_library()
    if not torch.cuda.is_available():
        raise RuntimeError("libgesmc needs a CUDA device")
    opts = GesmcOpts()
    lib.gesmc_opts_default(ctypes.byref(opts))
    opts.n = n
    opts.lazy_threshold = lazy_threshold
    opts.start_round = start_round
    opts.max_waves = max_waves
    opts.tuple_log2 = tuple_log2
    opts.group_log2 = group_log2
    opts.flags = ((0 if graphs else FLAG_NO_GRAPHS) | (FLAG_EXACT_ELL if exact_ell else 0)
                  | (FLAG_TINY_OVERFLOW if tiny_overflow else 0) | (FLAG_VERIFY_ROUNDS if verify_rounds else 0))
    if stream is None:
        stream = torch.cuda.current_stream()
    opts.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream) or 0))
    hooks = None
    if torch_allocator:
        hooks = _TorchAllocator(torch.cuda.current_device())
        opts.alloc = hooks.alloc
        opts.free = hooks.free
    ptr, m, on_dev, keep = _as_edge_buffer(edges)
    h = ctypes.c_void_p()
    _check(lib.gesmc_create(ctypes.c_void_p(ptr), m, on_dev, ctypes.byref(opts), ctypes.byref(h)), "gesmc_create")
    return h, (hooks, keep)


def gesmc_run(h, global_switches: int, seed: int):
    _check(load_library().gesmc_run(h, global_switches, seed), "gesmc_run")


def gesmc_edges(h, out=None):
    """Copy E (position order) into `out` (numpy uint64 or torch int64/uint64 on any device) or a new numpy array."""
    lib = load_library()
    m = int(lib.gesmc_num_edges(h))
    if out is None:
        out = np.empty(m, dtype=np.uint64)
    ptr, cap, on_dev, _keep = _as_edge_buffer(out)
    if isinstance(out, np.ndarray) and not out.flags.c_contiguous:
        raise ValueError("out must be contiguous")
    m_out = ctypes.c_uint64()
    _check(lib.gesmc_edges(h, ctypes.c_void_p(ptr), cap, on_dev, ctypes.byref(m_out)), "gesmc_edges")
    return out


def gesmc_stats(h) -> dict:
    st = GesmcStats()
    _check(load_library().gesmc_stats(h, ctypes.byref(st)), "gesmc_stats")
    return st.as_dict()


def gesmc_reset_stats(h):
    _check(load_library().gesmc_reset_stats(h), "gesmc_reset_stats")


NUM_STAGES = 11


def gesmc_set_profiling(h, enable: bool):
    _check(load_library().gesmc_set_profiling(h, int(enable)), "gesmc_set_profiling")


def gesmc_stage_name(stage: int) -> str:
    return load_library().gesmc_stage_name(stage).decode()


def gesmc_stage_times(h) -> tuple[dict, int]:
    """({stage name: accumulated ms}, profiled rounds)."""
    ms = (ctypes.c_double * NUM_STAGES)()
    rounds = ctypes.c_uint64()
    _check(load_library().gesmc_stage_times(h, ms, NUM_STAGES, ctypes.byref(rounds)), "gesmc_stage_times")
    return {gesmc_stage_name(i): float(ms[i]) for i in range(NUM_STAGES)}, int(rounds.value)


def gesmc_verify_list(edges, reference, n: int = 0) -> int:
    """Device check of a list (CUDA tensor of packed ids) against the degree
    sequence of `reference`: GESMC_OK or GESMC_E_INVARIANT."""
    return int(load_library().gesmc_verify_list(ctypes.c_void_p(edges.data_ptr()), edges.numel(),
                                                ctypes.c_void_p(reference.data_ptr()), reference.numel(), n))


def gesmc_destroy(h):
    if h:
        load_library().gesmc_destroy(h)


def noalloc_stream(edges_device, stream=None):
    """The stream an allocation-free call on a tensor of `edges_device` runs
    on: the given torch stream, which must belong to that device, or that
    device's current stream.  (A raw stream handle is taken as is.)"""
    import torch

    if stream is None:
        return torch.cuda.current_stream(edges_device)
    dev = getattr(stream, "device", None)
    if dev is not None and torch.device(dev) != torch.device(edges_device):
        raise ValueError(f"stream is on {dev}, but the edge list is on {edges_device}")
    return stream


def gesmc_run_noalloc(edges, n: int, global_switches: int, seed: int, start_round: int = 0, stream=None):
    """Allocation-free rounds in place on a CUDA tensor of packed ids (int64/uint64).

    For callers that may not allocate device memory; m <= NOALLOC_MAX_EDGES.
    The library's fixed scratch array is shared by all calls on a device, so
    calls whose device work may overlap must be serialised by the caller.
    The call runs on the tensor's device (made current for the call) and on
    `stream`, which must belong to that device (default: its current stream)."""
    import torch

    if not (isinstance(edges, torch.Tensor) and edges.is_cuda and edges.is_contiguous()
            and edges.dtype in (torch.int64, torch.uint64)):
        raise TypeError("edges must be a contiguous int64/uint64 CUDA tensor")
    stream = noalloc_stream(edges.device, stream)
    s = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream) or 0))
    with torch.cuda.device(edges.device):
        _check(load_library().gesmc_run_noalloc(ctypes.c_void_p(edges.data_ptr()), edges.numel(), n,
                                                global_switches, seed, start_round, s), "gesmc_run_noalloc")
    return edges


RANDOM_LOAD, RANDOM_STORE, RANDOM_CAS, RANDOM_ATOMIC_ADD, RANDOM_RED = 0, 1, 2, 3, 4


def gesmc_probe_random_access(nbytes: int, kind: int, accesses: int) -> float:
    """Uniformly random 8-byte accesses per second over an nbytes device buffer."""
    rate = ctypes.c_double()
    _check(load_library().gesmc_probe_random_access(nbytes, kind, accesses, ctypes.byref(rate)),
           "gesmc_probe_random_access")
    return float(rate.value)


class Chain:
    """One G-ES-MC chain resident on the current CUDA device."""

    def __init__(self, edges, **opts):
        self._h, self._keep = gesmc_create(edges, **opts)

    @property
    def handle(self):
        return self._h

    @property
    def m(self) -> int:
        return int(load_library().gesmc_num_edges(self._h))

    @property
    def n(self) -> int:
        return int(load_library().gesmc_num_nodes(self._h))

    @property
    def next_round(self) -> int:
        return int(load_library().gesmc_next_round(self._h))

    def run(self, global_switches: int, seed: int):
        gesmc_run(self._h, global_switches, seed)
        return self

    def es_run(self, switches: int, seed: int):
        """ParES: `switches` ES-MC switches with the sequential outcome (Algorithm 2)."""
        _check(load_library().gesmc_es_run(self._h, switches, seed), "gesmc_es_run")
        return self

    def edges(self, out=None):
        return gesmc_edges(self._h, out)

    def stats(self) -> dict:
        return gesmc_stats(self._h)

    def reset_stats(self):
        gesmc_reset_stats(self._h)

    def set_profiling(self, enable: bool = True):
        gesmc_set_profiling(self._h, enable)

    def set_round_launch(self, ctas: int) -> int:
        """0: the round's kernels one after another; >= 1: the whole round in
        one cooperative launch of that many CTAs; ROUND_RESIDENT: all rounds
        of a call in one CTA per chain (small chains).  Returns the count used
        (ROUND_RESIDENT for resident rounds)."""
        eff = ctypes.c_uint32()
        _check(load_library().gesmc_set_round_launch(self._h, ctas, ctypes.byref(eff)), "gesmc_set_round_launch")
        return int(eff.value)

    def verify(self) -> int:
        """Device check of the invariants (simple graph, starting degrees): GESMC_OK or GESMC_E_INVARIANT."""
        return int(load_library().gesmc_verify(self._h))

    def stage_times(self) -> tuple[dict, int]:
        return gesmc_stage_times(self._h)

    def close(self):
        if self._h:
            gesmc_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class Pool:
    """Many independent chains on the current CUDA device, advanced together.

    Each chain's result equals what a single-chain ``Chain`` with the same
    list, seed and start round gives; chains join and leave between rounds."""

    def __init__(self, max_edges: int, max_chains: int, max_waves: int = 0, tuple_log2: int = 0,
                 group_log2: int = 0, stream=None, torch_allocator: bool = True, graphs: bool = True):
        import torch

        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("libgesmc needs a CUDA device")
        o = GesmcPoolOpts()
        lib.gesmc_pool_opts_default(ctypes.byref(o))
        o.max_edges, o.max_chains, o.max_waves = max_edges, max_chains, max_waves
        o.tuple_log2, o.group_log2 = tuple_log2, group_log2
        o.flags = 0 if graphs else FLAG_NO_GRAPHS
        if stream is None:
            stream = torch.cuda.current_stream()
        o.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream) or 0))
        self._hooks = None
        if torch_allocator:
            self._hooks = _TorchAllocator(torch.cuda.current_device())
            o.alloc, o.free = self._hooks.alloc, self._hooks.free
        self._p = ctypes.c_void_p()
        _check(lib.gesmc_pool_create(ctypes.byref(o), ctypes.byref(self._p)), "gesmc_pool_create")

    @staticmethod
    def device_bytes(max_edges: int, max_chains: int, tuple_log2: int = 0) -> int:
        return int(load_library().gesmc_pool_device_bytes(max_edges, max_chains, tuple_log2))

    def add(self, edges, n: int = 0, seed: int = 0, start_round: int = 0, lazy_threshold: int = 0,
            exact_ell: bool = False) -> int:
        ptr, m, on_dev, _keep = _as_edge_buffer(edges)
        cid = ctypes.c_uint32()
        _check(load_library().gesmc_pool_add(self._p, ctypes.c_void_p(ptr), m, on_dev, n, seed, start_round,
                                             lazy_threshold, CHAIN_EXACT_ELL if exact_ell else 0,
                                             ctypes.byref(cid)), "gesmc_pool_add")
        return int(cid.value)

    def remove(self, chain: int):
        _check(load_library().gesmc_pool_remove(self._p, chain), "gesmc_pool_remove")

    def run(self, global_switches: int):
        _check(load_library().gesmc_pool_run(self._p, global_switches), "gesmc_pool_run")
        return self

    def es_run(self, switches: int):
        """ParES on every chain: `switches` ES-MC switches each, with its own seed."""
        _check(load_library().gesmc_pool_es_run(self._p, switches), "gesmc_pool_es_run")
        return self

    def edges(self, chain: int, out=None):
        lib = load_library()
        if out is None:
            out = np.empty(self.chain_info(chain)["m"], dtype=np.uint64)
        ptr, cap, on_dev, _keep = _as_edge_buffer(out)
        m_out = ctypes.c_uint64()
        _check(lib.gesmc_pool_edges(self._p, chain, ctypes.c_void_p(ptr), cap, on_dev, ctypes.byref(m_out)),
               "gesmc_pool_edges")
        return out

    def chain_info(self, chain: int) -> dict:
        info = GesmcChainInfo()
        _check(load_library().gesmc_pool_chain_info(self._p, chain, ctypes.byref(info)), "gesmc_pool_chain_info")
        return info.as_dict()

    @property
    def num_chains(self) -> int:
        return int(load_library().gesmc_pool_num_chains(self._p))

    @property
    def free_edges(self) -> int:
        return int(load_library().gesmc_pool_free_edges(self._p))

    def stats(self) -> dict:
        st = GesmcStats()
        _check(load_library().gesmc_pool_stats(self._p, ctypes.byref(st)), "gesmc_pool_stats")
        return st.as_dict()

    def reset_stats(self):
        _check(load_library().gesmc_pool_reset_stats(self._p), "gesmc_pool_reset_stats")

    def set_profiling(self, enable: bool = True):
        _check(load_library().gesmc_pool_set_profiling(self._p, int(enable)), "gesmc_pool_set_profiling")

    def set_round_launch(self, ctas: int) -> int:
        """0: the round's kernels one after another; >= 1: the whole round in
        one cooperative launch of that many CTAs; ROUND_RESIDENT: all rounds
        of a call in one CTA per chain (small chains).  Returns the count used
        (ROUND_RESIDENT for resident rounds)."""
        eff = ctypes.c_uint32()
        _check(load_library().gesmc_pool_set_round_launch(self._p, ctas, ctypes.byref(eff)),
               "gesmc_pool_set_round_launch")
        return int(eff.value)

    def verify(self, chain: int) -> int:
        """Device check of one chain's invariants: GESMC_OK or GESMC_E_INVARIANT."""
        return int(load_library().gesmc_pool_verify(self._p, chain))

    def stage_times(self) -> tuple[dict, int]:
        ms = (ctypes.c_double * NUM_STAGES)()
        rounds = ctypes.c_uint64()
        _check(load_library().gesmc_pool_stage_times(self._p, ms, NUM_STAGES, ctypes.byref(rounds)),
               "gesmc_pool_stage_times")
        return {gesmc_stage_name(i): float(ms[i]) for i in range(NUM_STAGES)}, int(rounds.value)

    def close(self):
        if self._p:
            load_library().gesmc_pool_destroy(self._p)
            self._p = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def generate_gnp(n: int, p: float, seed: int, stream=None):
    """G(n, p) generated on the current CUDA device: a device tensor (int64
    view of the packed uint64 edge ids, canonical, in pair order)."""
    import torch

    lib = load_library()
    if stream is None:
        stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream) or 0))
    m = ctypes.c_uint64()
    rc = lib.gesmc_generate_gnp(n, p, seed, None, 0, ctypes.byref(m), sp)
    if rc not in (0, -5):
        raise GesmcError(rc, "gesmc_generate_gnp")
    out = torch.empty(int(m.value), dtype=torch.int64, device=torch.device("cuda", torch.cuda.current_device()))
    if m.value:
        m2 = ctypes.c_uint64()
        _check(lib.gesmc_generate_gnp(n, p, seed, ctypes.c_void_p(out.data_ptr()), int(m.value), ctypes.byref(m2), sp),
               "gesmc_generate_gnp")
        assert m2.value == m.value
    return out

