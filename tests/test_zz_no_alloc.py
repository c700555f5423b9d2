"""gesmc_run_noalloc: the allocation-free entry point, for callers that may not
allocate device memory (a framework that owns all device memory through its
own pool, a process with a fixed memory budget).  Its output must equal the
allocating path (gesmc_create + gesmc_run + gesmc_edges) bit for bit, on two
calls in a row that share the library's one scratch array.

This file is collected last on purpose, so that a run that stops at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2111_03005_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_03005_gb300 import gesmc  # noqa: E402


def allocating_path(edges, n, rounds, seed, start_round=0):
    with gesmc.Chain(edges, n=n, start_round=start_round) as c:
        c.run(rounds, seed)
        return c.edges()


def noalloc_call(dev_edges, n, rounds, seed, start_round):
    """Call the C entry point through ctypes on a device buffer."""
    lib = gesmc.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.gesmc_run_noalloc(ctypes.c_void_p(dev_edges.data_ptr()), dev_edges.numel(), n, rounds, seed,
                               start_round, stream)
    return rc


@pytest.mark.parametrize("which", ["gnp_small", "near_max"])
def test_noalloc_matches_allocating_path_on_two_calls(which):
    if which == "gnp_small":
        edges, n = inputs.workload_gnp_small(seed=1)
    else:
        n = 3000
        edges = inputs.random_simple_graph(n, gesmc.NOALLOC_MAX_EDGES - 3, seed=12)
    seed, rounds = 77, 3
    dev = torch.from_numpy(edges.view(np.int64).copy()).cuda()
    # first call: rounds 0..2
    assert noalloc_call(dev, n, rounds, seed, 0) == gesmc.GESMC_OK
    first = dev.cpu().numpy().view(np.uint64).copy()
    assert np.array_equal(first, allocating_path(edges, n, rounds, seed))
    # second call on the first call's output: rounds 3..5, same shared scratch
    assert noalloc_call(dev, n, rounds, seed, rounds) == gesmc.GESMC_OK
    second = dev.cpu().numpy().view(np.uint64).copy()
    assert np.array_equal(second, allocating_path(edges, n, 2 * rounds, seed))
    assert not np.array_equal(first, second)


def test_noalloc_rejects_too_many_edges_and_bad_input():
    big = torch.zeros(gesmc.NOALLOC_MAX_EDGES + 1, dtype=torch.int64, device="cuda")
    assert noalloc_call(big, 0, 1, 1, 0) == gesmc.GESMC_E_TOO_LARGE
    loop = torch.tensor([(2 << 32) | 2, 1], dtype=torch.int64, device="cuda")
    assert noalloc_call(loop, 10, 1, 1, 0) == gesmc.GESMC_E_LOOP
    # a rejected list may come back in canonical form (min << 32 | max), at the same positions
    multi = torch.tensor([(5 << 32) | 1, (1 << 32) | 5, (2 << 32) | 3], dtype=torch.int64, device="cuda")
    assert noalloc_call(multi, 10, 1, 1, 0) == gesmc.GESMC_E_MULTI
    assert multi.cpu().tolist() == [(1 << 32) | 5, (1 << 32) | 5, (2 << 32) | 3]
    with pytest.raises(gesmc.GesmcError) as ei:
        gesmc.gesmc_run_noalloc(big, 0, 1, 1)
    assert ei.value.code == gesmc.GESMC_E_TOO_LARGE


def test_noalloc_binding_runs_on_the_tensor_device_and_stream():
    # the binding makes the tensor's device current and runs on a stream of that device
    edges, n = inputs.workload_gnp_small(seed=1)
    dev = torch.from_numpy(edges.view(np.int64).copy()).cuda()
    s = torch.cuda.Stream(device=dev.device)
    gesmc.gesmc_run_noalloc(dev, n, 2, 9, stream=s)
    s.synchronize()
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), allocating_path(edges, n, 2, 9))
