"""Error paths, driven from the host only (nothing faults, traps or hangs the
GPU): an allocator that returns NULL, and capacities shrunk by the
fault-injection flag until a round runs out of them.  Each must end in its
error code, leave the handle destroyable, and leave the library usable."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2111_03005_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_03005_gb300 import gesmc  # noqa: E402


def test_allocator_returning_null_gives_nomem_and_no_leak():
    lib = gesmc.load_library()
    calls = {"alloc": 0, "free": 0}

    def alloc(nbytes, stream, ctx):
        calls["alloc"] += 1
        return None   # out of memory

    def free(ptr, ctx):
        calls["free"] += 1

    alloc_fn, free_fn = gesmc.ALLOC_FN(alloc), gesmc.FREE_FN(free)
    edges, n = inputs.workload_gnp_small(seed=1)
    e = np.ascontiguousarray(edges, dtype=np.uint64)
    opts = gesmc.GesmcOpts()
    lib.gesmc_opts_default(ctypes.byref(opts))
    opts.alloc, opts.free = alloc_fn, free_fn
    h = ctypes.c_void_p()
    rc = lib.gesmc_create(ctypes.c_void_p(e.ctypes.data), len(e), 0, ctypes.byref(opts), ctypes.byref(h))
    assert rc == gesmc.GESMC_E_NOMEM and not h.value
    assert calls["alloc"] == 1 and calls["free"] == 0   # nothing was allocated, nothing freed
    # a pool the same way
    po = gesmc.GesmcPoolOpts()
    lib.gesmc_pool_opts_default(ctypes.byref(po))
    po.max_edges, po.max_chains = 10_000, 4
    po.alloc, po.free = alloc_fn, free_fn
    p = ctypes.c_void_p()
    assert lib.gesmc_pool_create(ctypes.byref(po), ctypes.byref(p)) == gesmc.GESMC_E_NOMEM and not p.value
    # the next handle, with the default allocator, works and is exact
    with gesmc.Chain(edges, n=n) as c:
        c.run(3, 5)
        assert np.array_equal(c.edges(), oracle.run(edges, seed=5, rounds=3)[0])


def test_tiny_overflow_capacity_reports_internal_error_and_stays_destroyable():
    # the double star's edge {0, 1} is proposed by about L/4 switches a round:
    # its partition overflows, and the overflow list holds only 16 tuples here
    edges, n = inputs.double_star(4000, seed=5)
    c = gesmc.Chain(edges, n=n, tiny_overflow=True)
    with pytest.raises(gesmc.GesmcError) as ei:
        c.run(2, 9)
    assert ei.value.code == gesmc.GESMC_E_INTERNAL
    # after the error: stats and edges still answer, further runs report the error, destroy works
    assert c.stats()["rounds"] >= 0
    assert len(c.edges()) == len(edges)
    with pytest.raises(gesmc.GesmcError):
        c.run(1, 9)
    c.close()
    # without the flag the same graph runs exactly
    with gesmc.Chain(edges, n=n) as ok:
        ok.run(2, 9)
        assert np.array_equal(ok.edges(), oracle.run(edges, seed=9, rounds=2)[0])


def test_tiny_overflow_on_a_graph_that_needs_no_room_is_exact():
    # a perfect matching stays one (every degree is 1), so no two switches
    # ever share a target and no target is in E: no dependency entry, no
    # overflow, and the shrunk capacities change nothing
    n = 4000
    edges = inputs.shuffle_edges(oracle.pack(list(range(0, n, 2)), list(range(1, n, 2))), 3)
    with gesmc.Chain(edges, n=n, tiny_overflow=True) as c:
        c.run(4, 3)
        assert np.array_equal(c.edges(), oracle.run(edges, seed=3, rounds=4)[0])
    # a G(n, p) graph needs more than 16 dependency entries a round: the error is reported
    edges, n = inputs.workload_gnp_small(seed=1)
    c = gesmc.Chain(edges, n=n, tiny_overflow=True)
    with pytest.raises(gesmc.GesmcError) as ei:
        c.run(4, 3)
    assert ei.value.code == gesmc.GESMC_E_INTERNAL
    c.close()


def test_wave_cap_error_leaves_the_library_usable():
    edges = inputs.pld_graph(5000, 2.01, 1, 500, seed=17)
    c = gesmc.Chain(edges, n=5000, max_waves=1)
    with pytest.raises(gesmc.GesmcError) as ei:
        c.run(3, 123)
    assert ei.value.code == gesmc.GESMC_E_WAVE_CAP
    c.close()
    with gesmc.Chain(edges, n=5000) as ok:
        ok.run(1, 123)
        assert np.array_equal(ok.edges(), oracle.run(edges, seed=123, rounds=1)[0])
