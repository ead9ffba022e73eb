"""PageRank power method (Eq. 22) on the Power-psi kernels (psi_pagerank): against the FP64
oracle's PageRank (relative L1 <= 1e-6 in the default precision, <= 1e-12 in FP64, same top-100
up to near-ties), closed forms (a star, a two-cycle, no edges), the homogeneous-activity
identity psi = pi of Sec. III, and the handle's psi scores left as they were."""
import numpy as np
import pytest

import oracle
import psigen

pytestmark = pytest.mark.gpu


def _graph(n, f, l, lam=None, mu=None, precision="fp32_refine", **kw):
    import torch
    from paper_2206_09960_gb300 import Graph

    lam = np.full(n, 0.5) if lam is None else lam
    mu = np.full(n, 0.5) if mu is None else mu
    args = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
            for a in (np.asarray(f, np.int32), np.asarray(l, np.int32), np.asarray(lam, np.float64),
                      np.asarray(mu, np.float64))]
    return Graph(n, *args, precision=precision, **kw)


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


@pytest.mark.parametrize("name,scale,alpha", [("rmat", 12, 0.85), ("chunglu", 14, 0.85), ("rmat", 13, 0.5)])
def test_pagerank_matches_oracle(name, scale, alpha):
    w = psigen.workload(name, seed=11, scale=scale)
    n = w["n"]
    ref = oracle.pagerank(n, w["follower"], w["leader"], alpha)
    with _graph(n, w["follower"], w["leader"], w["lam"], w["mu"]) as g:
        pi, info = g.pagerank(alpha, 1e-10, 10000)
        pi = pi.cpu().numpy()
    assert info["status"] == "PSI_OK" and info["converged"]
    assert info["gap_s_l1"] <= 1e-10
    assert rel_l1(pi, ref) <= 1e-6
    assert abs(info["psi_sum"] - ref.sum()) <= 1e-9
    ids = np.argsort(-pi, kind="stable")[:100]
    ref_ids, _ = oracle.topk(ref, 100)
    for pos in np.nonzero(ids != ref_ids)[0]:
        a, b = ref[ids[pos]], ref[ref_ids[pos]]
        assert abs(a - b) <= 1e-6 * max(a, b)


def test_pagerank_fp64_mode_and_host_output():
    w = psigen.workload("rmat", seed=12, scale=11)
    n = w["n"]
    ref = oracle.pagerank(n, w["follower"], w["leader"], 0.85)
    out = np.zeros(n)
    with _graph(n, w["follower"], w["leader"], precision="fp64") as g:
        _, info = g.pagerank(0.85, 1e-14, 10000, out=out)
    assert info["converged"]
    assert rel_l1(out, ref) <= 1e-12


def test_pagerank_closed_forms():
    alpha = 0.85
    # star: users 1..k follow user 0; pi_j = (1-a)/N, pi_0 = (1-a)/N (1 + a k)
    k = 9
    n = k + 1
    f = np.arange(1, n)
    l = np.zeros(k)
    with _graph(n, f, l, precision="fp64") as g:
        pi, _ = g.pagerank(alpha, 1e-15, 1000)
        pi = pi.cpu().numpy()
    base = (1 - alpha) / n
    np.testing.assert_allclose(pi[1:], base, rtol=1e-14)
    np.testing.assert_allclose(pi[0], base * (1 + alpha * k), rtol=1e-14)
    # two-cycle: the fixed point is the start 1/N
    with _graph(2, [0, 1], [1, 0]) as g:
        pi, info = g.pagerank(alpha, 1e-12, 1000)
    np.testing.assert_allclose(pi.cpu().numpy(), [0.5, 0.5], rtol=1e-15)
    # no edges: pi = (1 - alpha)/N everywhere after one step
    with _graph(5, np.zeros(0), np.zeros(0)) as g:
        pi, info = g.pagerank(alpha, 1e-12, 1000)
    np.testing.assert_allclose(pi.cpu().numpy(), (1 - alpha) / 5, rtol=1e-15)
    assert info["converged"]


def test_homogeneous_psi_equals_pagerank_and_scores_untouched():
    w = psigen.workload("rmat", seed=13, scale=12)
    n = w["n"]
    lam, mu = np.full(n, 0.15), np.full(n, 0.85)
    with _graph(n, w["follower"], w["leader"], lam, mu) as g:
        g.solve(1e-12, 10000)
        psi = g.scores().cpu().numpy()
        pi, _ = g.pagerank(0.85, 1e-12, 10000)
        pi = pi.cpu().numpy()
        again = g.scores().cpu().numpy()
    np.testing.assert_array_equal(psi, again)
    assert rel_l1(psi, pi) <= 1e-8


def test_pagerank_errors_and_step_cap():
    from paper_2206_09960_gb300 import PsiError, _binding as B

    w = psigen.workload("rmat", seed=14, scale=10)
    with _graph(w["n"], w["follower"], w["leader"]) as g:
        for a in (1.0, -0.1, float("nan")):
            with pytest.raises(PsiError) as e:
                g.pagerank(a)
            assert e.value.status == B.PSI_ERR_INVALID_ARG
        _, info = g.pagerank(0.85, 1e-12, 3)
        assert info["status"] == "PSI_ERR_NOT_CONVERGED" and info["iters"] == 3
