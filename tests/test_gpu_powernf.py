"""Power-NF (Algorithm 1) on the GPU (psi_power_nf): against the FP64 oracle's Power-NF (psi
within 1e-11 of each value's size, the same matrix-vector count up to origins whose last gap
sits at eps), against Power-psi's psi (the two methods reach the same scores, Sec. IV), the
no-step case (eps >= 1: psi from the first newsfeed vectors b_i), the step cap, host output,
the handle's psi scores left as they were; origins stepped in passes of any width give
bit-identical results; at the node and edge counts of the paper's Table III graphs
(Chung-Lu stand-ins, rates U(0, 1) as in Sec. V) against the oracle's Power-NF on sampled
origins, one by one; and the size limit (2^20 users with leaders)."""
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
    # passes of 256 origins (several passes, a ragged last one): the same bits
    with _graph(n, w["follower"], w["leader"], w["lam"], w["mu"]) as g:
        psi2, info2 = g.power_nf(eps, origins_per_pass=256)
    np.testing.assert_array_equal(psi2.cpu().numpy(), psi)
    assert info2["spmv_launches"] == info["spmv_launches"] and info2["iters"] == info["iters"]


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
        with pytest.raises(PsiError):
            g.power_nf(1e-12, origins_per_pass=-1)
    # 2^20 + 1 users in a ring, each following the next: every user has a leader
    n = (1 << 20) + 1
    f = np.arange(n, dtype=np.int32)
    l = np.roll(f, -1)
    u = psigen.uniform(9, 1, n)
    with _graph(n, f, l, 0.1 + u, 1.1 - u) as g:
        with pytest.raises(PsiError) as e:
            g.power_nf(1e-12)
    assert "2^20" in str(e.value)


@pytest.mark.parametrize("per_pass", [1, 7, 100, 255, 256, 257, 777, 5000])
def test_power_nf_pass_width_does_not_change_results(per_pass):
    """Each origin's arithmetic is the same in any pass: widths below, at and above the block
    of 256 origins, one origin per pass, and wider than the graph."""
    w = psigen.workload("poisson1000", seed=11, scale=777)
    n = w["n"]
    with _graph(n, w["follower"], w["leader"], w["lam"], w["mu"]) as g:
        ref, iref = g.power_nf(1e-12)
        got, info = g.power_nf(1e-12, origins_per_pass=per_pass)
    np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())
    assert info["spmv_launches"] == iref["spmv_launches"] and info["iters"] == iref["iters"]


def test_power_nf_long_leader_lists():
    """Users with more leaders than one segment holds (256): one with 2000 leaders (7 full
    segments and a partial one), one with exactly 512, one with 257, beside a sparse graph;
    every origin against the oracle's Algorithm 1, and pass widths that cut through them."""
    n = 2600
    w = psigen.workload("poisson1000", seed=12, scale=n)
    f, l = [w["follower"]], [w["leader"]]
    for user, k in ((0, 2000), (7, 512), (1999, 257)):
        lead = np.array([v for v in range(n) if v != user][:k], np.int32)
        f.append(np.full(k, user, np.int32))
        l.append(lead)
    f, l = np.concatenate(f), np.concatenate(l)
    eps = 1e-12
    with oracle.Model(n, f, l, w["lam"], w["mu"]) as m:
        ref, ref_mv = m.power_nf(eps)
    with _graph(n, f, l, w["lam"], w["mu"]) as g:
        psi, info = g.power_nf(eps)
        psi = psi.cpu().numpy()
        other, info2 = g.power_nf(eps, origins_per_pass=300)
    assert info["status"] == "PSI_OK" and info["converged"]
    scale = np.maximum(np.abs(ref), 1.0 / n)
    assert np.max(np.abs(psi - ref) / scale) <= 1e-11
    assert abs(info["spmv_launches"] - ref_mv) <= max(2, ref_mv // 1000)
    np.testing.assert_array_equal(other.cpu().numpy(), psi)
    assert info2["spmv_launches"] == info["spmv_launches"]


# node and edge counts of the paper's Table III graphs (Konect DBLP and HepPh), as Chung-Lu
# stand-ins with gamma = 2.1 and rates U(0, 1)
TABLE3 = {"dblp": (12_591, 49_743), "hepph": (34_546, 421_578)}


def table3_standin(name, seed):
    n, m = TABLE3[name]
    f, l = psigen.chung_lu_graph(n, 2.1, m, seed)
    lam = psigen.uniform_rates(n, 0.0, 1.0, seed, psigen.STREAM_LAMBDA)
    mu = psigen.uniform_rates(n, 0.0, 1.0, seed, psigen.STREAM_MU)
    return n, f, l, lam, mu


@pytest.mark.parametrize("name", ["dblp", "hepph"])
def test_power_nf_at_table3_sizes_sampled(name):
    """All origins on the GPU (several passes at the HepPh size), 48 of them through the
    oracle's Algorithm 1 one by one: the 16 with the most followers and 32 drawn at random;
    every user's psi against Power-psi; a single wide pass gives the same bits."""
    n, f, l, lam, mu = table3_standin(name, 31)
    eps = 1e-12
    with _graph(n, f, l, lam, mu) as g:
        psi, info = g.power_nf(eps, 100000)
        psi = psi.cpu().numpy()
        one, info1 = g.power_nf(eps, 100000, origins_per_pass=n)
        g.solve(0.0, 100000)
        ps = g.scores().cpu().numpy()
    assert info["status"] == "PSI_OK" and info["converged"]
    np.testing.assert_array_equal(one.cpu().numpy(), psi)
    assert info1["spmv_launches"] == info["spmv_launches"]
    followers = np.bincount(l, minlength=n)
    pick = np.unique(np.concatenate([np.argsort(-followers, kind="stable")[:16],
                                     (psigen.uniform(31, 5, 32) * n).astype(np.int64)]))
    with oracle.Model(n, f, l, lam, mu) as m:
        ref, _ = m.power_nf(eps, origins=pick)
    scale = np.maximum(np.abs(ref), 1.0 / n)
    assert np.max(np.abs(psi[pick] - ref) / scale) <= 1e-11
    assert np.max(np.abs(psi - ps) / np.maximum(np.abs(ps), 1.0 / n)) <= 1e-9
