"""Pins for the seeded input generators (psigen): the counter-based generator matches the
published SplitMix64 known answers, and each graph/rate recipe has the structure it claims."""
import numpy as np
import pytest

import psigen


def test_splitmix64_known_answers():
    # Vigna's splitmix64.c: state 0 gives 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f;
    # state 1234567 gives 6457827717110365317, 3203168211198807973, 9817491932198370423
    assert [psigen.splitmix64_at(0, i) for i in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                             0x06C45D188009454F]
    assert [psigen.splitmix64_at(1234567, i) for i in range(3)] == [6457827717110365317, 3203168211198807973,
                                                                    9817491932198370423]


def test_uniform_moments_and_determinism():
    u = psigen.uniform(5, 9, 200_000)
    assert u.min() >= 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    np.testing.assert_array_equal(u, psigen.uniform(5, 9, 200_000))
    assert not np.array_equal(u[:1000], psigen.uniform(6, 9, 1000))


def test_poisson_uniform_graph():
    n = 1000
    f, l = psigen.poisson_uniform_graph(n, 10.0, 0)
    assert (f != l).all()
    deg = np.bincount(f, minlength=n)
    assert abs(deg.mean() - 10) < 0.4 and abs(deg.var() - 10) < 2.0  # Poisson: mean = variance
    pairs = f.astype(np.int64) * n + l
    assert np.unique(pairs).size == pairs.size  # leaders drawn without replacement
    w = psigen.workload("poisson1000", seed=0)
    assert w["lam"].min() >= 0.1 and w["lam"].max() <= 1.0


def test_rmat_quadrants_and_relabel():
    sc = 16
    f, l = psigen.rmat_graph(sc, 8, 0.57, 0.19, 0.19, 3, relabel=False)
    assert f.size == 8 << sc and (f != l).all()
    top = 1 << (sc - 1)
    q = np.array([np.mean((f < top) & (l < top)), np.mean((f < top) & (l >= top)),
                  np.mean((f >= top) & (l < top)), np.mean((f >= top) & (l >= top))])
    np.testing.assert_allclose(q, [0.57, 0.19, 0.19, 0.05], atol=0.01)
    fr, lr = psigen.rmat_graph(sc, 8, 0.57, 0.19, 0.19, 3, relabel=True)
    perm = psigen.permutation(1 << sc, 3, 4)
    np.testing.assert_array_equal(fr, perm[f])
    np.testing.assert_array_equal(lr, perm[l])


def test_chung_lu_degree_law():
    n = 1 << 14
    f, l = psigen.chung_lu_graph(n, 2.1, 300_000, 1)
    assert (f != l).all()
    deg = np.sort(np.bincount(l, minlength=n))[::-1]
    # expected-degree weights (r+1)^(-1/(gamma-1)): the top user holds about 1/H of the draws
    w = np.arange(1, n + 1) ** (-1 / 1.1)
    assert abs(deg[0] / 300_000 - w[0] / w.sum()) < 0.01


def test_lognormal_rates():
    x = psigen.lognormal_rates(400_000, 0.0, 1.5, 1e-3, 1e3, 0, psigen.STREAM_LAMBDA)
    assert x.min() >= 1e-3 and x.max() <= 1e3
    assert abs(np.median(np.log(x))) < 0.02 and abs(np.std(np.log(x)) - 1.5) < 0.03


@pytest.mark.parametrize("name", ["poisson1000", "chunglu", "rmat"])
def test_workloads_small(name):
    w = psigen.workload(name, seed=0, scale=None if name == "poisson1000" else 12)
    assert w["follower"].dtype == np.int32 and w["lam"].dtype == np.float64
    assert w["follower"].min() >= 0 and w["leader"].max() < w["n"]
