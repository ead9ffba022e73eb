"""Power-NF (Algorithm 1) on the GPU (psi_power_nf): against the FP64 oracle's Power-NF (psi
within 1e-11 of each value's size, the same matrix-vector count up to origins whose last gap
sits at eps), against Power-psi's psi (the two methods reach the same scores, Sec. IV), the
no-step case (eps >= 1: psi from the first newsfeed vectors b_i), the step cap, host output,
the size limit and the handle's psi scores left as they were."""
import numpy as np
import pytest

import oracle
import psigen
from paper_2206_09960_gb300 import PsiError

pytestmark = pytest.mark.gpu


def _graph(n, f, l, lam, mu, precision="fp64", **kw):
    import torch
    from paper_2206_09960_gb300 import Graph

    args = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
            for a in (np.asarray(f, np.int32), np.asarray(l, np.int32), np.asarray(lam, np.float64),
                      np.asarray(mu, np.float64))]
    return Graph(n, *args, precision=precision, tol_mode="s_abs", **kw)


def _cases():
    w = psigen.workload("poisson1000", seed=3)
    yield "poisson1000", w
    w = psigen.workload("chunglu", seed=4, scale=11)
    yield "chunglu2048", w
    w = psigen.workload("poisson1000", seed=10, scale=4096)  # the size limit
    yield "poisson4096", w
    w = psigen.workload("rmat", seed=5, scale=11)
    yield "rmat2048", w
    w = psigen.workload("poisson1000", seed=6, scale=777)  # a ragged size
    yield "poisson777", w


@pytest.mark.parametrize("name", ["poisson1000", "chunglu2048", "rmat2048", "poisson777", "poisson4096"])
def test_power_nf_matches_oracle(name):
    w = dict(_cases())[name]
    n = w["n"]
    eps = 1e-12
    with oracle.Model(n, w["follower"], w["leader"], w["lam"], w["mu"]) as m:
        ref, ref_mv = m.power_nf(eps)
        ps = m.power_psi(0.0, to_floor=True)["psi"]
    with _graph(n, w["follower"], w["leader"], w["lam"], w["mu"]) as g:
        psi, info = g.power_nf(eps)
        psi = psi.cpu().numpy()
    assert info["status"] == "PSI_OK" and info["converged"]
    scale = np.maximum(np.abs(ref), 1.0 / n)
    assert np.max(np.abs(psi - ref) / scale) <= 1e-11
    # per-origin stop tests in a different summation order: an origin whose gap lands
    # within rounding of eps may take one step more or less
    assert abs(info["spmv_launches"] - ref_mv) <= max(2, ref_mv // 1000)
    assert info["gap_s_l1"] <= eps
    # Power-NF and Power-psi reach the same psi (the per-origin error is at most eps-sized)
    assert np.max(np.abs(psi - ps) / scale) <= 1e-9


def test_power_nf_no_step_and_cap():
    w = psigen.workload("poisson1000", seed=7, scale=300)
    n = w["n"]
    with oracle.Model(n, w["follower"], w["leader"], w["lam"], w["mu"]) as m:
        ref0, mv0 = m.power_nf(2.0)  # gap 1 <= eps: psi from b_i itself
        ref3, mv3 = m.power_nf(1e-300, max_iter=3)
    assert mv0 == 0 and mv3 == 3 * n
    with _graph(n, w["follower"], w["leader"], w["lam"], w["mu"]) as g:
        psi0, i0 = g.power_nf(2.0)
        out = np.zeros(n)
        _, i3 = g.power_nf(1e-300, max_iter=3, out=out)
        _, iz = g.power_nf(0.5, max_iter=0)
    assert i0["status"] == "PSI_OK" and i0["spmv_launches"] == 0 and i0["iters"] == 0
    np.testing.assert_allclose(psi0.cpu().numpy(), ref0, rtol=1e-13, atol=1e-16)
    assert i3["status"] == "PSI_ERR_NOT_CONVERGED" and i3["iters"] == 3 and i3["spmv_launches"] == 3 * n
    np.testing.assert_allclose(out, ref3, rtol=1e-12, atol=1e-16)
    assert iz["status"] == "PSI_ERR_NOT_CONVERGED" and iz["spmv_launches"] == 0


def test_power_nf_leaves_scores_and_limits_size():
    import torch

    w = psigen.workload("poisson1000", seed=8, scale=500)
    n = w["n"]
    with _graph(n, w["follower"], w["leader"], w["lam"], w["mu"]) as g:
        g.solve(1e-13)
        before = g.scores().clone()
        g.power_nf(1e-12)
        assert torch.equal(before, g.scores())
    big = psigen.workload("poisson1000", seed=9, scale=4097)
    with _graph(big["n"], big["follower"], big["leader"], big["lam"], big["mu"]) as g:
        with pytest.raises(PsiError):
            g.power_nf(1e-12)
