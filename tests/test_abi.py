"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/gesmc.h declares.  No device work is started here."""
import ctypes
import os
import re

import pytest

from paper_2111_03005_gb300 import build as libbuild
from paper_2111_03005_gb300 import gesmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(gesmc_[a-z_]+)\s*\(", text))
    names -= {"gesmc_alloc_fn", "gesmc_free_fn"}
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return ctypes.CDLL(libbuild.build_library())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gesmc_create", "gesmc_run", "gesmc_edges", "gesmc_stats", "gesmc_destroy", "gesmc_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    bound = {name for name, _, _ in gesmc._SIGNATURES}
    assert set(declared_functions()) <= bound


def test_host_only_entry_points():
    lib = gesmc.load_library()
    assert gesmc.gesmc_strerror(0) == "ok"
    assert "loop" in gesmc.gesmc_strerror(gesmc.GESMC_E_LOOP)
    opts = gesmc.GesmcOpts()
    lib.gesmc_opts_default(ctypes.byref(opts))
    assert opts.lazy_threshold == 0 and opts.n == 0 and opts.max_waves == 0
    # memory plan: about 145 bytes per edge for one chain (permutation buckets with room for twice their
    # mean, tuple partitions with room for their mean plus a margin, the overflow list for every tuple)
    m = 1 << 20
    b = gesmc.gesmc_device_bytes(m)
    assert 120 * m <= b < 180 * m
    # the bucket room doubles (and the bucket count halves) above 2^27 edges: the plan stays per edge
    for m in ((1 << 27) - 1, (1 << 27) + 1):
        assert 120 * m <= gesmc.gesmc_device_bytes(m) < 180 * m, m
    assert gesmc.gesmc_device_bytes(1 << 31) == 0
    # a 1.2e9-edge chain (the paper's largest graph) fits in 280 GB; near 2^31 edges the tuple storage
    # would need more than 32-bit indices, and such a pool is refused
    assert 0 < gesmc.gesmc_device_bytes(1_200_000_000) < 280e9
    assert gesmc.Pool.device_bytes((1 << 31) - 1, 1, 9) == 0
    assert gesmc.Pool.device_bytes(1 << 26, 4096, 0) > 0
    assert gesmc.gesmc_stage_name(0) == "clear" and gesmc.gesmc_stage_name(99) == ""


def test_create_rejects_bad_arguments_before_touching_a_device():
    lib = gesmc.load_library()
    h = ctypes.c_void_p()
    assert lib.gesmc_create(None, 5, 0, None, ctypes.byref(h)) == gesmc.GESMC_E_INVALID
    opts = gesmc.GesmcOpts()
    lib.gesmc_opts_default(ctypes.byref(opts))
    opts.n = (1 << 32) + 1
    assert lib.gesmc_create(None, 0, 0, ctypes.byref(opts), ctypes.byref(h)) == gesmc.GESMC_E_INVALID
    assert lib.gesmc_create(None, 1 << 31, 0, None, ctypes.byref(h)) == gesmc.GESMC_E_INVALID
    assert lib.gesmc_create(None, 0, 0, None, None) == gesmc.GESMC_E_INVALID


def test_sources_are_free_of_x86_only_code():
    # the GPU hosts are aarch64: no x86 intrinsics in anything compiled there
    for d in ("paper_2111_03005_gb300/csrc", "paper_2111_03005_gb300/inputs", "oracle"):
        for f in os.listdir(os.path.join(ROOT, d)):
            if f.endswith((".cu", ".cuh", ".c", ".cpp", ".h")):
                src = open(os.path.join(ROOT, d, f)).read()
                assert "immintrin" not in src and "__builtin_ia32" not in src and "march=native" not in src


def test_noalloc_binding_refuses_a_stream_of_another_device():
    # the allocation-free call runs on the edge list's device; a torch stream
    # that belongs to another device is refused before anything is launched
    import types

    torch = pytest.importorskip("torch")
    other = types.SimpleNamespace(device=torch.device("cuda", 1), cuda_stream=0)
    with pytest.raises(ValueError):
        gesmc.noalloc_stream(torch.device("cuda", 0), other)
    same = types.SimpleNamespace(device=torch.device("cuda", 0), cuda_stream=0)
    assert gesmc.noalloc_stream(torch.device("cuda", 0), same) is same
    assert gesmc.noalloc_stream(torch.device("cuda", 0), 12345) == 12345  # a raw handle is taken as is
