"""On-GPU G(n, p) generator: valid simple graphs in pair order, the right
edge-count and degree distributions, deterministic per seed, and usable as a
chain's input without leaving the device."""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_03005_gb300 import gesmc  # noqa: E402


def host(t):
    return t.cpu().numpy().view(np.uint64)


def test_complete_graph_and_empty_graph():
    n = 300
    e = host(gesmc.generate_gnp(n, 1.0, seed=1))
    assert len(e) == n * (n - 1) // 2
    u, v = oracle.unpack(e)
    assert np.array_equal(u, np.repeat(np.arange(n - 1), np.arange(n - 1, 0, -1)))
    assert len(gesmc.generate_gnp(n, 0.0, seed=1)) == 0


@pytest.mark.parametrize("n,p", [(1000, 0.01), (50_000, 2e-4), (1 << 20, 16.0 / ((1 << 20) - 1)), (70, 0.5),
                                 (10_000, 1e-9)])
def test_valid_sorted_and_binomial_count(n, p):
    e = host(gesmc.generate_gnp(n, p, seed=7))
    N = n * (n - 1) // 2
    mean, sd = N * p, math.sqrt(N * p * (1 - p))
    assert abs(len(e) - mean) <= 5 * sd + 1
    if len(e):
        assert oracle.validate(e, n)[0] == oracle.OK
        assert (np.diff(e.astype(np.uint64)) > 0).all()       # canonical ids in pair order


def test_degree_distribution_is_binomial():
    from scipy.stats import binom, chisquare
    n, p = 40_000, 2.5e-4
    e = host(gesmc.generate_gnp(n, p, seed=3))
    u, v = oracle.unpack(e)
    deg = np.bincount(np.concatenate([u, v]).astype(np.int64), minlength=n)
    k = np.arange(deg.max() + 1)
    obs = np.bincount(deg, minlength=len(k)).astype(float)
    exp = binom.pmf(k, n - 1, p) * n
    keep = exp >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    x = np.append(exp[keep], n - exp[keep].sum())
    assert chisquare(o, x * o.sum() / x.sum()).pvalue > 1e-4


def test_deterministic_per_seed():
    a = host(gesmc.generate_gnp(20_000, 1e-3, seed=11))
    b = host(gesmc.generate_gnp(20_000, 1e-3, seed=11))
    c = host(gesmc.generate_gnp(20_000, 1e-3, seed=12))
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_generated_graph_runs_on_the_device():
    n = 1 << 16
    dev = gesmc.generate_gnp(n, 8.0 / (n - 1), seed=5)
    with gesmc.Chain(dev, n=n) as c:
        c.run(2, 9)
        got = c.edges()
    expect, _ = oracle.run(host(dev), seed=9, rounds=2)
    assert np.array_equal(got, expect)
