"""Pins for the FP64 CPU oracle: it is checked against facts fixed by the paper and by
mathematics, never against itself.

* hand-derived closed forms (tests/golden/closed_forms.json, Eqs. 1-5) and exact
  rational solutions of the balance equations;
* brute force over every directed 4-user graph: five independent routes agree;
* homogeneous activity reduces psi to PageRank (Sec. III-D, Eqs. 20-22);
* the sum identity, residual certificates and the truncation bound (Eqs. 13-19);
* the L1 gap and the stop rule of Algorithm 2 on a case with a known gap sequence.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _cases():
    with open(GOLDEN) as fh:
        return json.load(fh)["cases"]


def _frac(xs):
    return np.array([float(Fraction(x)) for x in xs])


def _edges(case):
    e = np.array(case["edges"], np.int32).reshape(-1, 2)
    return e[:, 0].copy(), e[:, 1].copy()


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_closed_form_cases(case):
    n = case["n"]
    f, l = _edges(case)
    lam, mu = _frac(case["lambda"]), _frac(case["mu"])
    want_psi, want_s = _frac(case["psi"]), _frac(case["s"])
    with oracle.Model(n, f, l, lam, mu) as g:
        out = g.power_psi(max_iter=200, to_floor=True, history=True)
    np.testing.assert_allclose(out["psi"], want_psi, rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["s"], want_s, rtol=0, atol=1e-14)
    gaps = _frac(case["gaps_s_l1"])
    np.testing.assert_allclose(out["gaps"][: gaps.size], gaps, rtol=0, atol=1e-15)
    for route in (dense.direct_psi, dense.one_system_psi, dense.balance_psi):
        np.testing.assert_allclose(route(n, f, l, lam, mu), want_psi, rtol=0, atol=1e-14)


def _exact_balance(n, f, l, lam, mu):
    """psi in exact rationals from Eqs. 1-5 (sympy), for the stored fractions."""
    sympy = pytest.importorskip("sympy")
    L = dense.leader_sets(n, f, l)
    psi = []
    for i in range(n):
        p = sympy.symbols(f"p0:{n}")
        q = sympy.symbols(f"q0:{n}")
        eqs = []
        for j in range(n):
            if L[j]:
                eqs.append(sympy.Eq(sum(lam[k] + mu[k] for k in L[j]) * p[j],
                                    (lam[i] if i in L[j] else 0) + sum(mu[k] * p[k] for k in L[j])))
            else:
                eqs.append(sympy.Eq(p[j], 0))
            eqs.append(sympy.Eq((lam[j] + mu[j]) * q[j], mu[j] * p[j] + (lam[i] if j == i else 0)))
        sol = sympy.solve(eqs, list(p) + list(q), dict=True)[0]
        psi.append(sympy.Rational(sum(sol[x] for x in q), n))
    return psi


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_golden_fractions_are_exact(case):
    sympy = pytest.importorskip("sympy")
    f, l = _edges(case)
    lam = [sympy.Rational(x) for x in case["lambda"]]
    mu = [sympy.Rational(x) for x in case["mu"]]
    got = _exact_balance(case["n"], f, l, lam, mu)
    assert got == [sympy.Rational(x) for x in case["psi"]]


def test_two_cycle_closed_form_random_rates():
    rng = np.random.default_rng(7)
    for _ in range(50):
        lam, mu = rng.uniform(0.01, 5, 2), rng.uniform(0.01, 5, 2)
        c, d = mu / (lam + mu), lam / (lam + mu)
        want = np.array([d[0] * (1 + c[1]) / (2 * (1 - c[0] * c[1])),
                         d[1] * (1 + c[0]) / (2 * (1 - c[0] * c[1]))])
        out = oracle.solve(2, [0, 1], [1, 0], lam, mu, to_floor=True, max_iter=10000)
        np.testing.assert_allclose(out["psi"], want, rtol=1e-13)
        assert abs(out["psi"].sum() - 1) < 1e-13


def test_star_closed_form_random_rates():
    rng = np.random.default_rng(8)
    n = 7
    lam, mu = rng.uniform(0.01, 3, n), rng.uniform(0.01, 3, n)
    c, d = mu / (lam + mu), lam / (lam + mu)
    f = np.arange(1, n, dtype=np.int32)
    l = np.zeros(n - 1, np.int32)
    want = d / n
    want[0] = d[0] * (1 + c[1:].sum()) / n
    out = oracle.solve(n, f, l, lam, mu, to_floor=True)
    np.testing.assert_allclose(out["psi"], want, rtol=1e-14)


def test_brute_force_all_four_user_graphs():
    """All 2^12 directed graphs without self-loops on N=4: five routes agree."""
    n = 4
    pairs = [(j, i) for j in range(n) for i in range(n) if i != j]
    rng = np.random.default_rng(2022)
    worst = 0.0
    for mask in range(1 << len(pairs)):
        sel = [pairs[k] for k in range(len(pairs)) if mask >> k & 1]
        f = np.array([p[0] for p in sel], np.int32)
        l = np.array([p[1] for p in sel], np.int32)
        lam, mu = rng.uniform(0.05, 2.0, n), rng.uniform(0.05, 2.0, n)
        ref = dense.direct_psi(n, f, l, lam, mu)
        routes = [dense.one_system_psi(n, f, l, lam, mu)]
        if mask % 8 == 0:  # the slow scalar route on a regular subset
            routes.append(dense.balance_psi(n, f, l, lam, mu))
        with oracle.Model(n, f, l, lam, mu) as g:
            routes.append(g.power_psi(max_iter=5000, to_floor=True)["psi"])
            if mask % 4 == 0:
                routes.append(g.power_nf(1e-15, max_iter=5000)[0])
        for r in routes:
            worst = max(worst, float(np.abs(r - ref).max()))
    assert worst < 1e-12, worst


def test_balance_route_on_random_graph():
    rng = np.random.default_rng(3)
    n = 9
    f = rng.integers(0, n, 30).astype(np.int32)
    l = rng.integers(0, n, 30).astype(np.int32)
    keep = f != l
    f, l = f[keep], l[keep]
    lam, mu = rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    want = dense.balance_psi(n, f, l, lam, mu)
    out = oracle.solve(n, f, l, lam, mu, to_floor=True)
    np.testing.assert_allclose(out["psi"], want, rtol=1e-12, atol=1e-15)


def _random_graph(n, m, seed, every_user_follows=False):
    rng = np.random.default_rng(seed)
    f = rng.integers(0, n, m)
    l = rng.integers(0, n, m)
    if every_user_follows:
        f = np.concatenate([f, np.arange(n)])
        l = np.concatenate([l, (np.arange(n) + 1 + rng.integers(0, n - 1, n)) % n])
    keep = f != l
    return f[keep].astype(np.int32), l[keep].astype(np.int32)


@pytest.mark.parametrize("every", [True, False])
def test_homogeneous_activity_is_pagerank(every):
    """lambda_n = 0.15, mu_n = 0.85 for all n: psi = PageRank with alpha = 0.85 (Eqs. 20-22);
    W has zero rows for users without leaders (the model has no dangling patch)."""
    n = 80
    f, l = _random_graph(n, 300, 11, every)
    lam, mu = np.full(n, 0.15), np.full(n, 0.85)
    out = oracle.solve(n, f, l, lam, mu, to_floor=True)
    pr_dense = dense.pagerank_dense(n, f, l, 0.85)
    pr_iter = oracle.pagerank(n, f, l, 0.85)
    np.testing.assert_allclose(out["psi"], pr_dense, rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(pr_iter, pr_dense, rtol=1e-12, atol=1e-16)
    if every:
        assert abs(out["psi"].sum() - 1) < 1e-13


def test_equal_ratio_activity_is_weighted_pagerank():
    """lambda_n = k_n lam, mu_n = k_n mu: psi is PageRank on the walk that picks leader i of
    j with probability k_i / sum_{l in L(j)} k_l (not the unweighted one)."""
    n = 60
    f, l = _random_graph(n, 250, 12, True)
    k = np.random.default_rng(5).uniform(0.2, 5.0, n)
    out = oracle.solve(n, f, l, 0.3 * k, 0.7 * k, to_floor=True)
    np.testing.assert_allclose(out["psi"], dense.pagerank_dense(n, f, l, 0.7, weights=k), rtol=1e-12)
    unweighted = dense.pagerank_dense(n, f, l, 0.7)
    assert np.abs(out["psi"] - unweighted).max() > 1e-4


def test_sum_identity():
    """sum psi = (sum_n d_n + c^T m)/N with m = (I-A)^{-1} B 1 the newsfeed mass; m = 1
    exactly when every user has a leader (then sum psi = 1)."""
    n = 200
    rng = np.random.default_rng(14)
    lam, mu = rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    for every in (False, True):
        f, l = _random_graph(n, 500, 13, every)
        with oracle.Model(n, f, l, lam, mu) as g:
            out = g.power_psi(to_floor=True, max_iter=10000)
            c, d, sigma = g.vectors()
            m = g.newsfeed_mass()
        A, B, _, _ = dense.matrices(n, f, l, lam, mu)
        np.testing.assert_allclose(m, np.linalg.solve(np.eye(n) - A, B.sum(axis=1)), atol=1e-13)
        want = (d.sum() + c @ m) / n
        assert abs(out["psi"].sum() - want) < 1e-13
        if every:
            np.testing.assert_allclose(m, 1.0, atol=1e-13)
            assert abs(out["psi"].sum() - 1) < 1e-13
        else:
            assert (sigma == 0).any() and out["psi"].sum() < 1


def test_residual_certificate_and_truncation_bound():
    n = 300
    f, l = _random_graph(n, 1500, 15)
    rng = np.random.default_rng(16)
    lam, mu = rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    with oracle.Model(n, f, l, lam, mu) as g:
        exact = g.power_psi(to_floor=True, max_iter=10000)
        out = g.power_psi(eps=1e-6, tol_mode=oracle.TOL_S_ABS, max_iter=10000)
        c, d, sigma = g.vectors()
        # residual of the exact fixed point: s = s A + c
        sA, _ = g.apply(exact["s"])
        assert np.abs(sA + c - exact["s"]).sum() < 1e-12 * exact["s"].sum()
        # rho_inf = max_j sum_{l in L(j)} mu_l / sigma_j ; bound ||s* - s_t|| <= rho/(1-rho) eps_t
        fe, le = g.edges()
        rows = np.zeros(n)
        np.add.at(rows, fe, mu[le] / sigma[fe])
        rho = rows.max()
    assert out["converged"] and out["gap_s"] <= 1e-6
    err = np.abs(exact["s"] - out["s"]).sum()
    assert err <= rho / (1 - rho) * out["gap_s"] * (1 + 1e-9)
    # psi gap bound (Eq. 19 with the induced infinity norm of B): ||psi* - psi_t|| <= err ||B|| / N
    assert np.abs(exact["psi"] - out["psi"]).sum() <= err / n * (1 + 1e-9)


def test_gap_norm_and_stop_rule_two_cycle():
    """Gaps of the 2-cycle are 3/8, 3/16, 9/128 (golden); ||B||_inf = 3/4."""
    f, l, lam, mu = [0, 1], [1, 0], [1.0, 3.0], [3.0, 1.0]
    with oracle.Model(2, f, l, lam, mu) as g:
        assert abs(g.bnorm_inf - 0.75) < 1e-15
        # absolute s-tolerance, B_norm = 1: 3/8 > 0.3 >= 3/16 -> t = 2
        assert g.power_psi(0.3, oracle.TOL_S_ABS, oracle.BNORM_NONE)["iters"] == 2
        # with B_norm = 3/4: 9/32 <= 0.3 -> t = 1
        assert g.power_psi(0.3, oracle.TOL_S_ABS, oracle.BNORM_INF)["iters"] == 1
        # psi-tolerance divides by N = 2: 3/16 <= 0.2 -> t = 1; 3/32 > 0.05 >= 9/256 -> t = 3
        assert g.power_psi(0.2, oracle.TOL_PSI, oracle.BNORM_NONE)["iters"] == 1
        assert g.power_psi(0.05, oracle.TOL_PSI, oracle.BNORM_NONE)["iters"] == 3
        # Algorithm 2 starts with gap = 1: eps >= 1 performs no iteration (psi from s = c)
        out = g.power_psi(1.0, oracle.TOL_S_ABS, oracle.BNORM_NONE)
        assert out["iters"] == 0 and np.allclose(out["s"], [0.75, 0.25])
        # max_iter bound
        out = g.power_psi(1e-30, oracle.TOL_S_ABS, oracle.BNORM_NONE, max_iter=4)
        assert out["iters"] == 4 and not out["converged"]


def test_duplicates_merged_and_self_loops():
    n = 5
    f = np.array([0, 1, 2, 3, 4, 0], np.int32)
    l = np.array([1, 2, 3, 4, 0, 2], np.int32)
    lam, mu = np.linspace(0.2, 1, n), np.linspace(1, 0.3, n)
    base = oracle.solve(n, f, l, lam, mu, to_floor=True)
    dup = oracle.solve(n, np.concatenate([f, f[:3]]), np.concatenate([l, l[:3]]), lam, mu, to_floor=True)
    np.testing.assert_array_equal(base["psi"], dup["psi"])
    assert dup["m_unique"] == 6
    with pytest.raises(oracle.OracleError) as e:
        oracle.solve(n, np.append(f, 2), np.append(l, 2), lam, mu)
    assert e.value.code == oracle.ERR_SELF_LOOP
    dropped = oracle.solve(n, np.append(f, 2), np.append(l, 2), lam, mu, to_floor=True, drop_self_loops=True)
    np.testing.assert_array_equal(base["psi"], dropped["psi"])
    with pytest.raises(oracle.OracleError) as e:
        oracle.solve(n, np.append(f, 5), np.append(l, 0), lam, mu)
    assert e.value.code == oracle.ERR_ID
    for bad in (np.nan, -0.1, np.inf):
        lb = lam.copy()
        lb[2] = bad
        with pytest.raises(oracle.OracleError) as e:
            oracle.solve(n, f, l, lb, mu)
        assert e.value.code == oracle.ERR_RATE
    z = lam.copy(), mu.copy()
    z[0][1], z[1][1] = 0.0, 0.0
    with pytest.raises(oracle.OracleError):
        oracle.solve(n, f, l, z[0], z[1])
    # lambda = 0 or mu = 0 alone is allowed
    lz = lam.copy()
    lz[0] = 0.0
    oracle.solve(n, f, l, lz, mu, to_floor=True)


def test_ranking_ties_by_id():
    psi = np.array([0.1, 0.3, 0.3, 0.05, 0.3, 0.2])
    ids, vals = oracle.topk(psi, 4)
    assert ids.tolist() == [1, 2, 4, 5]
    assert vals.tolist() == [0.3, 0.3, 0.3, 0.2]
    rng = np.random.default_rng(1)
    psi = rng.integers(0, 20, 1000) / 7.0
    ids, _ = oracle.topk(psi, 100)
    want = sorted(range(1000), key=lambda i: (-psi[i], i))[:100]
    assert ids.tolist() == want


def test_power_nf_matches_power_psi_and_costs_more():
    rng = np.random.default_rng(17)
    n = 120
    f, l = _random_graph(n, 600, 18)
    lam, mu = rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    with oracle.Model(n, f, l, lam, mu) as g:
        nf, mv = g.power_nf(1e-14)
        ps = g.power_psi(1e-14, oracle.TOL_S_ABS)
    np.testing.assert_allclose(nf, ps["psi"], rtol=1e-11, atol=1e-15)
    assert mv > 20 * ps["iters"]


def test_power_nf_on_listed_origins_is_the_full_run():
    """Algorithm 1 treats each origin on its own: the oracle's origin-list form gives the full
    run's values for those origins, in the listed order (repeats allowed), and the step
    counts add up; an origin outside [0, n) is refused."""
    rng = np.random.default_rng(19)
    n = 150
    f, l = _random_graph(n, 700, 20)
    lam, mu = rng.uniform(0.0, 1, n), rng.uniform(0.1, 1, n)
    with oracle.Model(n, f, l, lam, mu) as g:
        full, mv = g.power_nf(1e-13)
        ids = np.array([149, 0, 7, 7, 63])
        sub, mv_sub = g.power_nf(1e-13, origins=ids)
        halves = [g.power_nf(1e-13, origins=np.arange(a, b))[1] for a, b in ((0, 75), (75, n))]
        with pytest.raises(oracle.OracleError):
            g.power_nf(1e-13, origins=np.array([n]))
    np.testing.assert_array_equal(sub, full[ids])
    assert sum(halves) == mv and 0 < mv_sub < mv


def test_poisson1000_direct_solve_agrees_with_power_psi():
    """The small FP64 workload: the direct solve of all N wall systems (one LU with N
    right-hand sides) and Algorithm 2 at eps = 1e-12 agree."""
    import psigen

    w = psigen.workload("poisson1000", seed=0)
    n = w["n"]
    direct = dense.direct_psi(n, w["follower"], w["leader"], w["lam"], w["mu"])
    out = oracle.solve(n, w["follower"], w["leader"], w["lam"], w["mu"], eps=1e-12,
                       tol_mode=oracle.TOL_S_ABS)
    assert out["converged"]
    rel_l1 = np.abs(out["psi"] - direct).sum() / np.abs(direct).sum()
    assert rel_l1 < 1e-12, rel_l1


def test_planted_transpose_is_caught():
    """A transposed A (a plausible slip) fails the asymmetric 2-cycle pin."""
    lam, mu = np.array([1.0, 3.0]), np.array([3.0, 1.0])
    A, B, c, d = dense.matrices(2, [0, 1], [1, 0], lam, mu)
    s_bad = np.linalg.solve(np.eye(2) - A, c)  # should be (I - A)^T
    psi_bad = (s_bad @ B + d) / 2
    assert np.abs(psi_bad - np.array([5 / 26, 21 / 26])).max() > 1e-3
