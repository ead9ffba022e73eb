"""Scenario batches (psi_batch_*): S activity scenarios on one graph in one product per step.
Each scenario must match the FP64 oracle run on that scenario alone (relative L1 <= 1e-6,
top-k identical up to near-ties) and the single-graph GPU path."""
import numpy as np
import pytest

import oracle
import psigen

pytestmark = pytest.mark.gpu


def _rates(n, S, seed, sigma=1.0):
    lam = np.stack([psigen.lognormal_rates(n, 0.0, sigma, 1e-3, 1e3, seed * 1000 + q, 201) for q in range(S)])
    mu = np.stack([psigen.lognormal_rates(n, 0.0, sigma, 1e-3, 1e3, seed * 1000 + q, 202) for q in range(S)])
    return lam, mu


def batch_solve(n, f, l, lam, mu, eps, k=50, on_device=True, **kw):
    import torch
    from paper_2206_09960_gb300 import Batch

    arrs = [np.ascontiguousarray(f, np.int32), np.ascontiguousarray(l, np.int32), np.ascontiguousarray(lam),
            np.ascontiguousarray(mu)]
    if on_device:
        arrs = [torch.from_numpy(x).cuda() for x in arrs]
    with Batch(n, *arrs, **kw) as b:
        status, infos = b.solve(eps, 20000)
        psi = b.scores().cpu().numpy()
        ids, vals = b.topk(min(k, n))
        stats = b.stats()
    return dict(status=status, infos=infos, psi=psi, ids=ids.cpu().numpy(), vals=vals.cpu().numpy(), stats=stats)


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def assert_same_ranking(gpu_ids, psi_ref, tol):
    ref_ids, _ = oracle.topk(psi_ref, len(gpu_ids))
    for pos in np.nonzero(gpu_ids != ref_ids)[0]:
        a, b = psi_ref[gpu_ids[pos]], psi_ref[ref_ids[pos]]
        assert abs(a - b) <= tol * max(abs(a), abs(b)), (pos, a, b)


@pytest.mark.parametrize("S,scale", [(8, 13), (64, 11), (1, 12), (33, 10)])
def test_batch_matches_oracle_per_scenario(S, scale):
    w = psigen.workload("rmat", seed=4, scale=scale)
    n = w["n"]
    lam, mu = _rates(n, S, scale)
    out = batch_solve(n, w["follower"], w["leader"], lam, mu, 1e-8)
    assert out["status"] == "PSI_OK"
    with oracle.Model(n, w["follower"], w["leader"], lam[0], mu[0]) as g0:
        m_unique = g0.m
    assert out["stats"]["m_unique"] == m_unique
    for q in range(S):
        ref = oracle.solve(n, w["follower"], w["leader"], lam[q], mu[q], to_floor=True, max_iter=5000)
        assert out["infos"][q]["converged"]
        assert out["infos"][q]["gap_scaled"] <= 1e-8
        assert rel_l1(out["psi"][q], ref["psi"]) <= 1e-6, q
        assert_same_ranking(out["ids"][q], ref["psi"], 1e-6)
        assert abs(out["infos"][q]["psi_sum"] - ref["psi"].sum()) <= 1e-6


def test_batch_matches_single_graph_path():
    from test_gpu_parity import gpu_solve

    w = psigen.workload("chunglu", seed=5, scale=14)
    n, S = w["n"], 6
    lam, mu = _rates(n, S, 7)
    out = batch_solve(n, w["follower"], w["leader"], lam, mu, 1e-9, on_device=False)
    for q in range(S):
        one = gpu_solve(n, w["follower"], w["leader"], lam[q], mu[q], 1e-9)
        assert rel_l1(out["psi"][q], one["psi"]) <= 1e-8
        # FP32 term sums round differently in the two kernels (chunk order vs tile tree): a
        # scenario whose first FP64 check narrowly fails takes one more series step and one
        # more FP64 step
        assert abs(out["infos"][q]["iters"] - one["info"]["iters"]) <= 2


def test_batch_homogeneous_scenario_is_pagerank_and_modes():
    w = psigen.workload("rmat", seed=6, scale=11)
    n = w["n"]
    lam, mu = _rates(n, 3, 8)
    lam[1], mu[1] = 0.15, 0.85
    for bn in ("none", "inf"):
        out = batch_solve(n, w["follower"], w["leader"], lam, mu, 1e-11, bnorm_mode=bn)
        pr = oracle.pagerank(n, w["follower"], w["leader"], 0.85)
        assert rel_l1(out["psi"][1], pr) <= 1e-9
        for q in (0, 2):
            ref = oracle.solve(n, w["follower"], w["leader"], lam[q], mu[q], to_floor=True)
            assert rel_l1(out["psi"][q], ref["psi"]) <= 1e-8


def test_batch_deterministic_and_empty_graph():
    w = psigen.workload("rmat", seed=7, scale=12)
    n = w["n"]
    lam, mu = _rates(n, 5, 9)
    a = batch_solve(n, w["follower"], w["leader"], lam, mu, 1e-8)
    b = batch_solve(n, w["follower"], w["leader"], lam, mu, 1e-8)
    np.testing.assert_array_equal(a["psi"], b["psi"])
    np.testing.assert_array_equal(a["ids"], b["ids"])
    e = batch_solve(n, np.zeros(0, np.int32), np.zeros(0, np.int32), lam, mu, 1e-8)
    np.testing.assert_allclose(e["psi"], lam / (lam + mu) / n, rtol=1e-15)


def test_batch_errors():
    from paper_2206_09960_gb300 import PsiError, _binding as B

    n = 20
    f = np.array([0, 1], np.int32)
    l = np.array([1, 2], np.int32)
    lam, mu = _rates(n, 4, 1)
    bad = lam.copy()
    bad[3, 5] = -1.0
    with pytest.raises(PsiError) as e:
        batch_solve(n, f, l, bad, mu, 1e-8)
    assert e.value.status == B.PSI_ERR_BAD_RATE
    big_l, big_m = _rates(n, 65, 2)
    with pytest.raises(PsiError) as e:
        batch_solve(n, f, l, big_l, big_m, 1e-8)
    assert e.value.status == B.PSI_ERR_INVALID_ARG


def test_batch_tight_absolute_tolerance():
    w = psigen.workload("rmat", seed=42, scale=12)
    n = w["n"]
    lam, mu = _rates(n, 4, 11)
    out = batch_solve(n, w["follower"], w["leader"], lam, mu, 1e-10, tol_mode="s_abs")
    assert out["status"] == "PSI_OK"
    for q in range(4):
        ref = oracle.solve(n, w["follower"], w["leader"], lam[q], mu[q], eps=1e-10, tol_mode=oracle.TOL_S_ABS)
        # refinement rounds of the FP32 series: more steps than plain FP64, but boundedly
        assert out["infos"][q]["iters"] <= 2 * ref["iters"] + 10
        assert rel_l1(out["psi"][q], ref["psi"]) <= 1e-9


def test_batch_at_the_benchmark_size_four_of_64_scenarios():
    """The batched benchmark's configuration (64 scenarios, LogNormal(0, 1) rates, R-MAT
    scale 22, edge factor 16); four scenarios spread over the batch against the oracle."""
    scale, S = 22, 64
    w = psigen.workload("rmat", seed=0, scale=scale)
    n = w["n"]
    lam, mu = _rates(n, S, 22)
    out = batch_solve(n, w["follower"], w["leader"], lam, mu, 1e-8, k=100)
    assert out["status"] == "PSI_OK"
    for q in (0, 21, 42, 63):
        ref = oracle.solve(n, w["follower"], w["leader"], lam[q], mu[q], eps=1e-11)
        assert out["stats"]["m_unique"] == ref["m_unique"]
        assert out["infos"][q]["converged"] and out["infos"][q]["gap_scaled"] <= 1e-8
        assert rel_l1(out["psi"][q], ref["psi"]) <= 1e-6, q
        assert_same_ranking(out["ids"][q], ref["psi"], 1e-6)
