"""The leader sums sigma_j, beta_j of Sec. II in the single-graph build: exact integer sums
taken half-way through the edge sort with repeated edges subtracted afterwards (rates whose
exponents span at most 40 binades), else the follower-grouped product.  Both against the FP64
oracle (relative L1 of psi <= 1e-12 in FP64 mode), with many repeated edges, and bit-identical
results for any order of the same edges."""
import numpy as np
import pytest

import oracle
import psigen

pytestmark = pytest.mark.gpu


def _solve(n, f, l, lam, mu, precision="fp64", eps=1e-13):
    import torch
    from paper_2206_09960_gb300 import Graph

    args = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
            for a in (np.asarray(f, np.int32), np.asarray(l, np.int32), np.asarray(lam, np.float64),
                      np.asarray(mu, np.float64))]
    with Graph(n, *args, precision=precision, tol_mode="s_abs") as g:
        info = g.solve(eps, 20000)
        psi = g.scores().cpu().numpy()
        st = g.stats()
    return psi, info, st


def _log_uniform(n, lo, hi, seed, stream):
    u = psigen.uniform(seed, stream, n)
    return np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u)


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


@pytest.mark.parametrize("lo,hi", [(1e-5, 1e5), (1e-10, 1e10)])  # exact sums; the product (wider range)
def test_leader_sums_wide_rates(lo, hi):
    w = psigen.workload("rmat", seed=21, scale=13)
    n = w["n"]
    lam = _log_uniform(n, lo, hi, 21, psigen.STREAM_LAMBDA)
    mu = _log_uniform(n, lo, hi, 21, psigen.STREAM_MU)
    lam[::7] = 0.0  # zero posting rates are allowed
    ref = oracle.solve(n, w["follower"], w["leader"], lam, mu, eps=0.0, to_floor=True)
    psi, info, st = _solve(n, w["follower"], w["leader"], lam, mu)
    assert info["converged"]
    assert st["m_unique"] == ref["m_unique"]
    assert rel_l1(psi, ref["psi"]) <= 1e-12


def test_leader_sums_with_many_repeated_edges():
    w = psigen.workload("chunglu", seed=22, scale=14)
    n = w["n"]
    reps = 1 + (psigen.uniform(22, 7, w["follower"].size) * 5).astype(np.int64)  # each edge 1..5 times
    f = np.repeat(w["follower"], reps)
    l = np.repeat(w["leader"], reps)
    order = psigen.permutation(f.size, 22, 8)
    f, l = f[order], l[order]
    ref = oracle.solve(n, f, l, w["lam"], w["mu"], eps=0.0, to_floor=True)
    psi, info, st = _solve(n, f, l, w["lam"], w["mu"])
    assert st["m_unique"] == ref["m_unique"] and st["m_input"] == f.size
    assert rel_l1(psi, ref["psi"]) <= 1e-12


@pytest.mark.parametrize("precision", ["fp32_refine", "fp64"])
def test_edge_order_does_not_change_results(precision):
    w = psigen.workload("rmat", seed=23, scale=14)
    n = w["n"]
    f, l = w["follower"], w["leader"]
    order = psigen.permutation(f.size, 23, 9)
    a, ia, _ = _solve(n, f, l, w["lam"], w["mu"], precision, 1e-10)
    b, ib, _ = _solve(n, f[order], l[order], w["lam"], w["mu"], precision, 1e-10)
    c, ic, _ = _solve(n, f[::-1], l[::-1], w["lam"], w["mu"], precision, 1e-10)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    assert ia["iters"] == ib["iters"] == ic["iters"]


@pytest.mark.parametrize("top,tiny", [(2.0 ** 40, 0.0), (2.0 ** 41, 0.0), (1.0, 1e-310)])
def test_leader_sums_at_the_edges_of_the_exact_range(top, tiny):
    """Rates whose binary exponents span exactly 40 (exact sums), 41 (the product), and a
    subnormal rate (the product): each against the oracle."""
    w = psigen.workload("chunglu", seed=24, scale=13)
    n = w["n"]
    u = psigen.uniform(24, 11, n)
    lam = np.where(u < 0.5, 1.0, top)   # exponents 0 and log2(top)
    mu = np.where(u < 0.25, top, 1.0)
    if tiny:
        lam[::97] = tiny  # subnormal posting rates
    ref = oracle.solve(n, w["follower"], w["leader"], lam, mu, eps=0.0, to_floor=True)
    psi, info, st = _solve(n, w["follower"], w["leader"], lam, mu)
    assert info["converged"]
    assert st["m_unique"] == ref["m_unique"]
    assert rel_l1(psi, ref["psi"]) <= 1e-12


@pytest.mark.parametrize("lo,hi", [(1e-3, 1e3), (1e-10, 1e10)])
def test_one_edge_repeated_many_times(lo, hi):
    """200,000 copies of one follow edge beside a sparse graph: the repeats span whole warps
    and blocks of the duplicate merge and are subtracted from the exact sums in one run per
    warp (exact path), or merged before the follower sort (product path)."""
    w = psigen.workload("poisson1000", seed=25, scale=3000)
    n = w["n"]
    f = np.concatenate([w["follower"], np.full(200_000, 7, np.int32), w["follower"][:50]])
    l = np.concatenate([w["leader"], np.full(200_000, 11, np.int32), w["leader"][:50]])
    lam = _log_uniform(n, lo, hi, 25, psigen.STREAM_LAMBDA)
    mu = _log_uniform(n, lo, hi, 25, psigen.STREAM_MU)
    ref = oracle.solve(n, f, l, lam, mu, eps=0.0, to_floor=True)
    psi, info, st = _solve(n, f, l, lam, mu)
    assert info["converged"]
    assert st["m_unique"] == ref["m_unique"] and st["m_input"] == f.size
    assert rel_l1(psi, ref["psi"]) <= 1e-12
