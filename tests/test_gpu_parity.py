"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: relative L1 of psi <= 1e-12 in FP64 mode and <= 1e-6 with FP32 storage; the top-100
ranking (psi descending, ties by id) identical, except where two oracle values differ by
less than the comparison tolerance (reported as a near-tie, not a mismatch); integer
outputs (ranking ids, edge counts) bit-exact.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import psigen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _torch():
    import torch

    return torch


def gpu_solve(n, f, l, lam, mu, eps, precision="fp32_refine", tol_mode="psi", bnorm_mode="none",
              max_iter=20000, on_device=True, init_s=None, k=100, **kw):
    torch = _torch()
    from paper_2206_09960_gb300 import Graph

    f = np.ascontiguousarray(f, np.int32)
    l = np.ascontiguousarray(l, np.int32)
    lam = np.ascontiguousarray(lam, np.float64)
    mu = np.ascontiguousarray(mu, np.float64)
    if on_device:
        args = [torch.from_numpy(x).cuda() for x in (f, l, lam, mu)]
    else:
        args = [f, l, lam, mu]
    with Graph(n, *args, precision=precision, tol_mode=tol_mode, bnorm_mode=bnorm_mode, **kw) as g:
        init = None if init_s is None else torch.from_numpy(np.ascontiguousarray(init_s, np.float64)).cuda()
        info = g.solve(eps, max_iter, init)
        psi = g.scores().cpu().numpy()
        s = g.iterate().cpu().numpy()
        kk = min(k, n)
        ids, vals = g.topk(kk)
        stats = g.stats()
    return dict(info=info, psi=psi, s=s, ids=ids.cpu().numpy(), vals=vals.cpu().numpy(), stats=stats)


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def assert_same_ranking(gpu_ids, psi_ref, tol):
    """GPU top-k ids equal the oracle's ranking, allowing swaps only among near-ties."""
    k = len(gpu_ids)
    ref_ids, ref_vals = oracle.topk(psi_ref, k)
    if np.array_equal(gpu_ids, ref_ids):
        return
    for pos in np.nonzero(gpu_ids != ref_ids)[0]:
        a, b = psi_ref[gpu_ids[pos]], psi_ref[ref_ids[pos]]
        assert abs(a - b) <= tol * max(abs(a), abs(b)), (pos, gpu_ids[pos], ref_ids[pos], a, b)


def _cases():
    with open(GOLDEN) as fh:
        return json.load(fh)["cases"]


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine", "fp32"])
@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_closed_forms(case, precision):
    n = case["n"]
    e = np.array(case["edges"], np.int32).reshape(-1, 2)
    lam = np.array([float(Fraction(x)) for x in case["lambda"]])
    mu = np.array([float(Fraction(x)) for x in case["mu"]])
    want = np.array([float(Fraction(x)) for x in case["psi"]])
    out = gpu_solve(n, e[:, 0], e[:, 1], lam, mu, 1e-15, precision=precision, tol_mode="s_abs", max_iter=500,
                    k=n)
    tol = 1e-14 if precision != "fp32" else 1e-6
    np.testing.assert_allclose(out["psi"], want, rtol=tol, atol=tol)
    assert abs(out["info"]["psi_sum"] - want.sum()) < 1e-6


def test_two_cycle_gap_sequence_and_stop_rule():
    """Gaps 3/8, 3/16, 9/128 (golden); the stop rule of Algorithm 2 picks t exactly."""
    f, l, lam, mu = [0, 1], [1, 0], [1.0, 3.0], [3.0, 1.0]
    for eps, tol_mode, bn, t in [(0.3, "s_abs", "none", 2), (0.3, "s_abs", "inf", 1), (0.2, "psi", "none", 1),
                                 (0.05, "psi", "none", 3)]:
        for prec in ("fp64", "fp32_refine", "fp32"):
            out = gpu_solve(2, f, l, lam, mu, eps, precision=prec, tol_mode=tol_mode, bnorm_mode=bn, k=2)
            # fp32_refine confirms the FP32 series' stop with one FP64 step (gap 9/128-ish here)
            want = t + 1 if prec == "fp32_refine" else t
            assert out["info"]["iters"] == want, (eps, tol_mode, bn, prec, out["info"])
    out = gpu_solve(2, f, l, lam, mu, 1.0, precision="fp64", tol_mode="s_abs", k=2)
    assert out["info"]["iters"] == 0
    np.testing.assert_allclose(out["s"], [0.75, 0.25])
    out = gpu_solve(2, f, l, lam, mu, 1e-30, precision="fp64", tol_mode="s_abs", max_iter=4, k=2)
    assert out["info"]["iters"] == 4 and out["info"]["status"] == "PSI_ERR_NOT_CONVERGED"


def test_poisson1000_fp64_matches_direct_solve_and_oracle():
    from oracle import dense

    w = psigen.workload("poisson1000", seed=0)
    n = w["n"]
    ref = oracle.solve(n, w["follower"], w["leader"], w["lam"], w["mu"], eps=1e-12, tol_mode=oracle.TOL_S_ABS)
    direct = dense.direct_psi(n, w["follower"], w["leader"], w["lam"], w["mu"])
    out = gpu_solve(n, w["follower"], w["leader"], w["lam"], w["mu"], 1e-12, precision="fp64", tol_mode="s_abs")
    assert out["info"]["converged"]
    assert abs(out["info"]["iters"] - ref["iters"]) <= 1
    assert rel_l1(out["psi"], ref["psi"]) <= 1e-12
    assert rel_l1(out["psi"], direct) <= 1e-12
    assert_same_ranking(out["ids"], direct, 1e-12)
    assert out["stats"]["m_unique"] == ref["m_unique"]


@pytest.mark.parametrize("scale", [14, 17])
def test_chunglu_fp32_refine(scale):
    w = psigen.workload("chunglu", seed=1, scale=scale)
    n = w["n"]
    ref = oracle.solve(n, w["follower"], w["leader"], w["lam"], w["mu"], to_floor=True, max_iter=5000)
    out = gpu_solve(n, w["follower"], w["leader"], w["lam"], w["mu"], 1e-8)
    assert out["info"]["converged"], out["info"]
    assert out["info"]["gap_scaled"] <= 1e-8
    assert rel_l1(out["psi"], ref["psi"]) <= 1e-6
    assert_same_ranking(out["ids"], ref["psi"], 1e-6)
    assert out["stats"]["m_unique"] == ref["m_unique"]
    assert abs(out["info"]["psi_sum"] - ref["psi"].sum()) <= 1e-6 * ref["psi"].sum()


def test_chunglu_full_size_fp32_refine():
    """The Chung-Lu workload at its full size (N=2^20, 2e7 draws)."""
    w = psigen.workload("chunglu", seed=0)
    n = w["n"]
    ref = oracle.solve(n, w["follower"], w["leader"], w["lam"], w["mu"], to_floor=True, max_iter=5000)
    out = gpu_solve(n, w["follower"], w["leader"], w["lam"], w["mu"], 1e-8)
    assert out["info"]["converged"]
    assert rel_l1(out["psi"], ref["psi"]) <= 1e-6
    assert_same_ranking(out["ids"], ref["psi"], 1e-6)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_refine", 1e-6)])
def test_rmat_small(precision, tol):
    w = psigen.workload("rmat", seed=2, scale=16)
    n = w["n"]
    ref = oracle.solve(n, w["follower"], w["leader"], w["lam"], w["mu"], to_floor=True, max_iter=5000)
    eps = 1e-15 if precision == "fp64" else 1e-8
    out = gpu_solve(n, w["follower"], w["leader"], w["lam"], w["mu"], eps, precision=precision, max_iter=5000)
    if precision == "fp64":  # may stop at the rounding floor before eps
        assert out["info"]["gap_scaled"] < 1e-13
    else:
        assert out["info"]["converged"]
    assert rel_l1(out["psi"], ref["psi"]) <= tol
    assert_same_ranking(out["ids"], ref["psi"], tol)


def test_fp32_plain_mode_is_close():
    w = psigen.workload("rmat", seed=3, scale=14)
    n = w["n"]
    ref = oracle.solve(n, w["follower"], w["leader"], w["lam"], w["mu"], to_floor=True)
    out = gpu_solve(n, w["follower"], w["leader"], w["lam"], w["mu"], 1e-6, precision="fp32")
    assert rel_l1(out["psi"], ref["psi"]) <= 2e-5


def _run_pair(n, f, l, lam, mu, precision="fp32_refine", **kw):
    ref = oracle.solve(n, f, l, lam, mu, to_floor=True, max_iter=20000)
    out = gpu_solve(n, f, l, lam, mu, 1e-14 if precision == "fp64" else 1e-9, precision=precision,
                    max_iter=20000, k=min(100, n), **kw)
    return ref, out


@pytest.mark.parametrize("lengths", [[1] * 50, [31, 32, 33], [4096, 1, 2048, 2049, 5], [20000], [2047, 2048, 2049],
                                     [511, 512, 513, 1023, 1024, 1025], [255, 256, 257, 1, 1, 767],
                                     [70001, 3, 66049, 1]],
                         ids=["ones", "warpish", "tiles", "one_long_row", "tile_edges", "small_tile_edges",
                              "step_edges", "rows_over_128_tiles"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("spmv_tile", [512, 2048])
def test_row_length_bins(lengths, precision, spmv_tile):
    """Rows (followers per leader) of chosen lengths, including one row spanning many tiles,
    rows ending exactly on tile and step boundaries and ragged tails, for the smallest and
    the largest tile of the product; with 512-nonzero tiles the last case has two rows that
    span more than 128 tiles, which the fix-up sums with a whole warp."""
    rng = np.random.default_rng(sum(lengths))
    n = max(lengths) + len(lengths) + 10
    f, l = [], []
    for i, L in enumerate(lengths):
        fol = rng.choice(np.delete(np.arange(n), i), L, replace=False)
        f += fol.tolist()
        l += [i] * L
    # leaders follow someone too, so the iteration mixes
    for i in range(len(lengths)):
        f.append(i)
        l.append((i + 1) % len(lengths) if len(lengths) > 1 else n - 1)
    lam, mu = rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    ref, out = _run_pair(n, np.array(f), np.array(l), lam, mu, precision, spmv_tile=spmv_tile)
    assert out["stats"]["spmv_tile"] == spmv_tile
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert rel_l1(out["psi"], ref["psi"]) <= tol
    assert_same_ranking(out["ids"], ref["psi"], tol)


def test_single_row_holds_every_edge():
    n = 300_001
    f = np.arange(1, n, dtype=np.int32)
    l = np.zeros(n - 1, np.int32)
    rng = np.random.default_rng(4)
    lam, mu = rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    c, d = mu / (lam + mu), lam / (lam + mu)
    want = d / n
    want[0] = d[0] * (1 + c[1:].sum()) / n  # star closed form
    for prec, tol in (("fp64", 1e-13), ("fp32_refine", 1e-7)):
        out = gpu_solve(n, f, l, lam, mu, 1e-12, precision=prec, tol_mode="s_abs", k=10)
        assert rel_l1(out["psi"], want) <= tol
        assert abs(out["psi"][0] - want[0]) <= tol * want[0]


def test_empty_graph_and_dropped_self_loops():
    n = 50
    rng = np.random.default_rng(5)
    lam, mu = rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    for prec, steps in (("fp64", 1), ("fp32", 1), ("fp32_refine", 2)):  # refine: + one FP64 check step
        out = gpu_solve(n, np.zeros(0, np.int32), np.zeros(0, np.int32), lam, mu, 1e-10, precision=prec, k=10)
        np.testing.assert_allclose(out["psi"], lam / (lam + mu) / n, rtol=1e-15)
        assert out["info"]["iters"] == steps
    loops = np.arange(n, dtype=np.int32)
    out = gpu_solve(n, loops, loops, lam, mu, 1e-10, self_loops="drop", k=10)
    np.testing.assert_allclose(out["psi"], lam / (lam + mu) / n, rtol=1e-15)
    assert out["stats"]["m_unique"] == 0


def test_duplicates_are_merged():
    w = psigen.workload("rmat", seed=6, scale=12)
    n = w["n"]
    f, l = w["follower"], w["leader"]
    # same operator; the internal numbering (by raw degree) and so the summation order may differ
    a = gpu_solve(n, f, l, w["lam"], w["mu"], 1e-14, precision="fp64")
    b = gpu_solve(n, np.concatenate([f, f[::3]]), np.concatenate([l, l[::3]]), w["lam"], w["mu"], 1e-14,
                  precision="fp64")
    assert rel_l1(a["psi"], b["psi"]) <= 1e-13
    np.testing.assert_array_equal(a["ids"], b["ids"])
    assert a["stats"]["m_unique"] == b["stats"]["m_unique"] == oracle.canonical_edges(n, f, l)[0].size


def test_errors_are_statuses():
    from paper_2206_09960_gb300 import PsiError, _binding as B

    n = 10
    lam, mu = np.ones(n), np.ones(n)
    cases = [
        (np.array([0, 11], np.int32), np.array([1, 2], np.int32), lam, mu, {}, B.PSI_ERR_OUT_OF_RANGE_ID),
        (np.array([0, -1], np.int32), np.array([1, 2], np.int32), lam, mu, {}, B.PSI_ERR_OUT_OF_RANGE_ID),
        (np.array([0, 3], np.int32), np.array([1, 3], np.int32), lam, mu, {}, B.PSI_ERR_SELF_LOOP),
        (np.array([0], np.int32), np.array([1], np.int32), np.r_[np.nan, lam[1:]], mu, {}, B.PSI_ERR_BAD_RATE),
        (np.array([0], np.int32), np.array([1], np.int32), np.r_[-1.0, lam[1:]], mu, {}, B.PSI_ERR_BAD_RATE),
        (np.array([0], np.int32), np.array([1], np.int32), np.r_[0.0, lam[1:]], np.r_[0.0, mu[1:]], {},
         B.PSI_ERR_BAD_RATE),
    ]
    for f, l, la, m_, kw, want in cases:
        with pytest.raises(PsiError) as e:
            gpu_solve(n, f, l, la, m_, 1e-8, **kw)
        assert e.value.status == want
    # a solve-less handle reports NOT_SOLVED; bad k is INVALID_ARG
    from paper_2206_09960_gb300 import Graph

    with Graph(n, np.array([0], np.int32), np.array([1], np.int32), lam, mu) as g:
        with pytest.raises(PsiError) as e:
            g.scores()
        assert e.value.status == B.PSI_ERR_NOT_SOLVED
        g.solve(1e-8)
        with pytest.raises(PsiError) as e:
            g.topk(n + 1)
        assert e.value.status == B.PSI_ERR_INVALID_ARG


def test_host_and_device_inputs_agree_and_results_are_deterministic():
    w = psigen.workload("chunglu", seed=7, scale=15)
    args = (w["n"], w["follower"], w["leader"], w["lam"], w["mu"], 1e-8)
    a = gpu_solve(*args, on_device=True)
    b = gpu_solve(*args, on_device=False)
    c = gpu_solve(*args, on_device=True)
    np.testing.assert_array_equal(a["psi"], b["psi"])
    np.testing.assert_array_equal(a["psi"], c["psi"])
    np.testing.assert_array_equal(a["ids"], c["ids"])
    assert a["info"]["iters"] == c["info"]["iters"]


def test_reorder_off_gives_same_scores():
    w = psigen.workload("rmat", seed=8, scale=13)
    args = (w["n"], w["follower"], w["leader"], w["lam"], w["mu"], 1e-12)
    a = gpu_solve(*args, precision="fp64", reorder=True)
    b = gpu_solve(*args, precision="fp64", reorder=False)
    assert rel_l1(a["psi"], b["psi"]) <= 1e-13


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine", "fp32"])
def test_warm_start_resume(precision):
    """Resuming from the converged iterate takes very few steps and lands on the same psi."""
    w = psigen.workload("chunglu", seed=9, scale=14)
    args = (w["n"], w["follower"], w["leader"], w["lam"], w["mu"])
    eps = 1e-10 if precision != "fp32" else 1e-6  # FP32 storage cannot reach 1e-10
    cold = gpu_solve(*args, eps, precision=precision)
    warm = gpu_solve(*args, eps, precision=precision, init_s=cold["s"])
    assert warm["info"]["iters"] <= max(3, cold["info"]["iters"] // 4)
    tol = 1e-9 if precision != "fp32" else 1e-5
    assert rel_l1(warm["psi"], cold["psi"]) <= tol
    # a warm start from an arbitrary vector still converges to the same fixed point
    rnd = np.random.default_rng(1).uniform(0, 3, w["n"])
    other = gpu_solve(*args, eps, precision=precision, init_s=rnd)
    assert rel_l1(other["psi"], cold["psi"]) <= (1e-8 if precision != "fp32" else 1e-5)


def test_homogeneous_activity_topk_ties_bit_exact():
    """lambda=.15, mu=.85 everywhere: psi is PageRank; users without followers tie exactly at
    (1-alpha)/N, so the ranking's tie-break (ascending id) is exercised."""
    w = psigen.workload("rmat", seed=10, scale=12)
    n = w["n"]
    lam, mu = np.full(n, 0.15), np.full(n, 0.85)
    out = gpu_solve(n, w["follower"], w["leader"], lam, mu, 1e-13, precision="fp64", k=n)
    order = sorted(range(n), key=lambda i: (-out["psi"][i], i))
    np.testing.assert_array_equal(out["ids"], np.array(order, np.int32))
    np.testing.assert_array_equal(out["vals"], out["psi"][order])
    pr = oracle.pagerank(n, w["follower"], w["leader"], 0.85)
    assert rel_l1(out["psi"], pr) <= 1e-12


def test_profile_reports_kernel_time():
    w = psigen.workload("rmat", seed=11, scale=15)
    out = gpu_solve(w["n"], w["follower"], w["leader"], w["lam"], w["mu"], 1e-8, profile=True)
    info = out["info"]
    assert info["spmv_timed"] + info["refine_timed"] == info["iters"]
    assert info["refine_timed"] == info["refinements"] >= 1
    assert 0 < info["spmv_ms"] + info["refine_ms"] <= info["ms"]


def test_tight_absolute_tolerance_takes_the_fp64_products():
    """An absolute s-tolerance near the FP64 floor: the default mode must switch its
    confirming and final products from float pairs to FP64 (float-pair rounding alone would
    keep the gap above eps and the solve would stall).  Its FP32 series still needs a few
    refinement rounds for such a target, so it takes more steps than the FP64 mode, but
    boundedly more, and ends at the same psi."""
    w = psigen.workload("rmat", seed=41, scale=14)
    args = (w["n"], w["follower"], w["leader"], w["lam"], w["mu"], 1e-10)
    ref = gpu_solve(*args, precision="fp64", tol_mode="s_abs")
    out = gpu_solve(*args, precision="fp32_refine", tol_mode="s_abs")
    assert ref["info"]["converged"] and out["info"]["converged"]
    assert out["info"]["iters"] <= 2 * ref["info"]["iters"] + 10, (out["info"]["iters"], ref["info"]["iters"])
    assert rel_l1(out["psi"], ref["psi"]) <= 1e-12


def test_tile_sizes_agree_and_the_automatic_choice():
    """The product's tile (nonzeros per warp) changes only the summation order: FP64 results
    of every tile size agree to rounding, a small graph gets the smallest tile, and tile
    sizes outside {0, 512, 1024, 2048} are rejected."""
    from paper_2206_09960_gb300 import PsiError, _binding as B

    w = psigen.workload("rmat", seed=31, scale=14)
    args = (w["n"], w["follower"], w["leader"], w["lam"], w["mu"], 1e-13)
    outs = {t: gpu_solve(*args, precision="fp64", spmv_tile=t) for t in (0, 512, 1024, 2048)}
    assert outs[0]["stats"]["spmv_tile"] == 512  # ~262K edges: far fewer than 4 tiles per warp at 2048
    ref = oracle.solve(w["n"], w["follower"], w["leader"], w["lam"], w["mu"], eps=1e-13)
    for t in (512, 1024, 2048):
        assert outs[t]["stats"]["spmv_tile"] == t
        assert rel_l1(outs[t]["psi"], outs[2048]["psi"]) <= 1e-13
        assert rel_l1(outs[t]["psi"], ref["psi"]) <= 1e-12
    for bad in (256, 1000, 4096, -1):
        with pytest.raises(PsiError) as e:
            gpu_solve(*args, spmv_tile=bad)
        assert e.value.status == B.PSI_ERR_INVALID_ARG


@pytest.mark.parametrize("scale", [20, 22])
def test_rmat_benchmark_recipe_at_scale(scale):
    """The benchmark's own recipe (R-MAT, edge factor 16, LogNormal(0, 1.5) rates) at scales
    the oracle solves in seconds.  At scale 22 the product uses the benchmark's tile (2048
    nonzeros) and the edge sort's key is over 40 bits wide, so its six-pass path runs, as
    at scale 25."""
    w = psigen.workload("rmat", seed=0, scale=scale)
    n = w["n"]
    ref = oracle.solve(n, w["follower"], w["leader"], w["lam"], w["mu"], to_floor=True, max_iter=5000)
    out = gpu_solve(n, w["follower"], w["leader"], w["lam"], w["mu"], 1e-8)
    st = out["stats"]
    assert out["info"]["converged"], out["info"]
    assert out["info"]["gap_scaled"] <= 1e-8
    assert st["m_unique"] == ref["m_unique"]
    assert rel_l1(out["psi"], ref["psi"]) <= 1e-6
    assert_same_ranking(out["ids"], ref["psi"], 1e-6)
    np.testing.assert_array_equal(out["vals"], out["psi"][out["ids"]])
    assert abs(out["info"]["psi_sum"] - ref["psi"].sum()) <= 1e-6 * ref["psi"].sum()
    # width of the edge sort's key: the leader row field and the follower's gathered index
    key_bits = (st["n_rows"] - 1).bit_length() + st["n_gathered"].bit_length()
    if scale >= 22:
        assert key_bits > 40, key_bits
        # the benchmark's product configurations, each forced: the 8-warp kernel on the
        # fixed rule's tile, and the 32-warp kernel with a shared-memory copy of the most
        # gathered entries on every tile
        for kw in (dict(autotune=False, spmv_hot=0), dict(spmv_tile=2048, spmv_hot=32768),
                   dict(spmv_tile=1024, spmv_hot=28672), dict(spmv_tile=512, spmv_hot=24576)):
            o = gpu_solve(n, w["follower"], w["leader"], w["lam"], w["mu"], 1e-8, **kw)
            assert o["info"]["converged"], kw
            assert o["stats"]["spmv_hot"] == kw["spmv_hot"], (kw, o["stats"])
            assert rel_l1(o["psi"], ref["psi"]) <= 1e-6, kw
            assert rel_l1(o["psi"], out["psi"]) <= 1e-7, kw
            assert_same_ranking(o["ids"], ref["psi"], 1e-6)


def test_autotuner_choice_changes_results_only_by_rounding():
    """The first solve of a large graph times the series product's configurations and keeps
    the fastest; another graph of the same sizes reuses the choice without timing.  Every
    configuration computes the same Algorithm 2: psi agrees with the fixed rule's to rounding
    and with the oracle within the FP32 bar."""
    w = psigen.workload("rmat", seed=11, scale=19)
    n = w["n"]
    ref = oracle.solve(n, w["follower"], w["leader"], w["lam"], w["mu"], to_floor=True, max_iter=5000)
    runs = {}
    for name, kw in (("fixed", dict(autotune=False)), ("tuned", dict(autotune=True)),
                     ("again", dict(autotune=True)), ("hot", dict(autotune=False, spmv_hot=24576))):
        out = gpu_solve(n, w["follower"], w["leader"], w["lam"], w["mu"], 1e-8, **kw)
        assert out["info"]["converged"], name
        assert rel_l1(out["psi"], ref["psi"]) <= 1e-6, name
        assert_same_ranking(out["ids"], ref["psi"], 1e-6)
        runs[name] = out
    assert runs["fixed"]["stats"]["spmv_hot"] == 0 and runs["fixed"]["stats"]["tune_ms"] == 0
    tuned, again = runs["tuned"]["stats"], runs["again"]["stats"]
    assert tuned["m_unique"] >= 1 << 22 and tuned["tune_ms"] > 0
    assert tuned["spmv_tile"] in (512, 1024, 2048) and tuned["spmv_hot"] in (0, 24576, 28672, 32768)
    assert again["tune_ms"] == 0 and (again["spmv_tile"], again["spmv_hot"]) == (tuned["spmv_tile"], tuned["spmv_hot"])
    assert runs["hot"]["stats"]["spmv_hot"] == 24576
    for name in ("tuned", "again", "hot"):
        assert rel_l1(runs[name]["psi"], runs["fixed"]["psi"]) <= 1e-7, name
    np.testing.assert_array_equal(runs["again"]["psi"], runs["tuned"]["psi"])  # same choice: same bits


def test_start_vector_is_c_to_an_ulp_for_any_rates():
    """With no step taken (max_iter = 0), s_0 = c: c_j = mu_j / (lambda_j + mu_j) from the
    device's reciprocals, within 3 ulp of the FP64 quotient, for rates across the whole FP64
    range (the FP32-seeded reciprocal and its FP64 fallback)."""
    rng = np.random.default_rng(21)
    n = 4000
    lam = 10.0 ** rng.uniform(-300, 300, n)
    mu = 10.0 ** rng.uniform(-300, 300, n)
    lam[:1000] = rng.uniform(1e-3, 1e3, 1000)
    mu[:1000] = rng.uniform(1e-3, 1e3, 1000)
    lam[1000:1010] = 0.0  # lambda = 0 alone is allowed: c = 1
    f = rng.integers(0, n, 20000).astype(np.int32)
    l = rng.integers(0, n, 20000).astype(np.int32)
    keep = f != l
    out = gpu_solve(n, f[keep], l[keep], lam, mu, 1e-8, max_iter=0, precision="fp64")
    want = mu / (lam + mu)
    np.testing.assert_allclose(out["s"], want, rtol=6.7e-16, atol=0)


def test_graphs_on_two_streams_from_two_threads():
    """Two host threads, each with its own stream, build and solve graphs at once through the
    C ABI (host and device inputs; the bench's end-to-end mode): every result is bit-identical
    to the same graph solved alone."""
    import threading

    torch = _torch()
    from paper_2206_09960_gb300 import Graph

    ws = [psigen.workload("rmat", seed=31 + i, scale=15) for i in range(2)]
    alone = [gpu_solve(w["n"], w["follower"], w["leader"], w["lam"], w["mu"], 1e-8, on_device=(i == 0))
             for i, w in enumerate(ws)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    got = [[], []]
    errors = []

    def lane(i):
        try:
            w = ws[i]
            args = [np.ascontiguousarray(w[k]) for k in ("follower", "leader", "lam", "mu")]
            with torch.cuda.stream(streams[i]):
                if i == 0:
                    args = [torch.from_numpy(a).cuda() for a in args]
                for _ in range(3):
                    with Graph(w["n"], *args, stream=streams[i]) as g:
                        g.solve(1e-8, 20000)
                        got[i].append(g.scores().cpu().numpy())
            streams[i].synchronize()
        except Exception as exc:
            errors.append(exc)

    threads = [threading.Thread(target=lane, args=(i,)) for i in (0, 1)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i in (0, 1):
        assert len(got[i]) == 3
        for psi in got[i]:
            np.testing.assert_array_equal(psi, alone[i]["psi"])


@pytest.mark.parametrize("tuned", [True, False])
def test_claimed_tiles_are_bit_reproducible(tuned):
    """At R-MAT scale 20 the FP32 series product has far more tiles than two per warp, so most
    tiles are claimed at run time and land on different warps from run to run; each tile's gap
    is summed on its own and the tiles' gaps in fixed slices, so repeated solves (and a
    permuted edge order) give the same bits, step counts and gaps.  Both launch shapes: the
    32-warp blocks with the shared-memory copy and the 8-warp blocks, tiles of 512."""
    torch = _torch()
    w = psigen.workload("rmat", seed=33, scale=20)
    n, f, l = w["n"], w["follower"], w["leader"]
    kw = {"spmv_tile": 512, "spmv_hot": 28672} if tuned else {"spmv_tile": 512, "autotune": 0, "spmv_hot": 0}
    runs = [gpu_solve(n, f, l, w["lam"], w["mu"], 1e-8, **kw) for _ in range(3)]
    order = psigen.permutation(f.size, 33, 4)
    runs.append(gpu_solve(n, f[order], l[order], w["lam"], w["mu"], 1e-8, **kw))
    st = runs[0]["stats"]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    warps = sms * (32 if st["spmv_hot"] > 0 else 5 * 8)
    assert st["m_unique"] / st["spmv_tile"] > 4 * warps  # most tiles are claimed
    assert tuned == (st["spmv_hot"] > 0)
    for r in runs[1:]:
        np.testing.assert_array_equal(r["psi"], runs[0]["psi"])
        np.testing.assert_array_equal(r["ids"], runs[0]["ids"])
        assert r["info"]["iters"] == runs[0]["info"]["iters"]
        assert r["info"]["gap_s_l1"] == runs[0]["info"]["gap_s_l1"]
