"""Learned warm start: the network's GPU forward and backward kernels against the FP64 CPU
reference (oracle/mlp.py), the features against their definition, and what training buys:
fewer Power-psi steps to the same fixed point on a held-out graph."""
import numpy as np
import pytest

import oracle
import psigen
from oracle import mlp as ref

pytestmark = pytest.mark.gpu


def _model(seed=0):
    from paper_2206_09960_gb300.warmstart import WarmStartModel

    return WarmStartModel(seed)


@pytest.mark.parametrize("rows", [300, 100003])
def test_forward_and_gradient_match_cpu_reference(rows):
    """300 rows: a partial tile in one block; 100003 rows: blocks that take several 128-row
    iterations and keep their gradient tiles across them, and a ragged last tile."""
    import torch

    rng = np.random.default_rng(0)
    params = (rng.standard_normal(ref.N_PARAMS) * 0.2).astype(np.float32)
    norm = np.concatenate([rng.normal(0, 1, 8), rng.uniform(0.5, 2, 8), [1.5], [2.0]]).astype(np.float32)
    x = rng.normal(0, 1.5, (rows, 8)).astype(np.float32)
    t = rng.normal(1.0, 2.0, rows).astype(np.float32)
    m = _model()
    m.set_params(params, norm)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    # Both sides round every product operand (weights, inputs, hidden activations, dz2, dz1)
    # to BF16, but from sums taken in different precisions (FP32 on the GPU, FP64 here): a
    # value within ~1e-7 of a BF16 rounding midpoint can round to the neighbouring BF16 on
    # one side, a one-ulp (2^-8 relative) difference in one activation.  Such flips hit a
    # few of the 300 x 128 activations at most; rows without one agree to FP32 rounding.
    y = m.forward(xd).cpu().numpy()
    y_ref = ref.forward(params, norm.astype(np.float64), x)
    err = np.abs(y - y_ref)
    assert np.mean(err > 1e-5 + 1e-5 * np.abs(y_ref)) <= 0.02, np.sort(err)[-8:]
    assert np.max(err / (1.0 + np.abs(y_ref))) <= 2e-2
    loss, g = m.grad(xd, td, want_grad=True)
    loss_ref, g_ref = ref.loss_and_grad(params, norm.astype(np.float64), x, t)
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref
    assert np.linalg.norm(g - g_ref) <= 1e-3 * np.linalg.norm(g_ref)
    # each block of parameters separately (a transposed or dropped block would show here)
    o = 0
    for name, shape in ref.SIZES:
        k = int(np.prod(shape))
        assert np.linalg.norm(g[o:o + k] - g_ref[o:o + k]) <= 2e-3 * max(np.linalg.norm(g_ref[o:o + k]), 1e-12), name
        o += k
    # against the unrounded network the same gradient is off by the BF16 rounding itself
    _, g_exact = ref.loss_and_grad(params, norm.astype(np.float64), x, t, bf16_round=False)
    assert np.linalg.norm(g - g_exact) > np.linalg.norm(g - g_ref)
    m.close()


def test_features_follow_their_definition():
    from paper_2206_09960_gb300 import Graph
    from paper_2206_09960_gb300.warmstart import graph_features

    w = psigen.workload("rmat", seed=3, scale=11)
    n = w["n"]
    with Graph(n, w["follower"], w["leader"], w["lam"], w["mu"]) as g:
        x = graph_features(g).cpu().numpy()
    f, l = oracle.canonical_edges(n, w["follower"], w["leader"])
    followers = np.bincount(l, minlength=n)
    leaders = np.bincount(f, minlength=n)
    base = np.stack([np.log1p(followers), np.log1p(leaders), np.log(w["lam"]), np.log(w["mu"])], 1)
    sums = np.zeros((n, 4))
    np.add.at(sums, l, base[f])
    means = np.where(followers[:, None] > 0, sums / np.maximum(followers, 1)[:, None], 0.0)
    np.testing.assert_allclose(x, np.concatenate([base, means], 1), rtol=1e-5, atol=1e-5)


def test_training_cuts_steps_to_the_same_fixed_point():
    import torch

    from paper_2206_09960_gb300 import Graph
    from paper_2206_09960_gb300.warmstart import train, training_rows

    train_w = [psigen.workload("rmat", seed=100 + k, scale=12 + k % 3) for k in range(8)]
    x, t = training_rows(train_w, rows_per_graph=1 << 13)
    model, losses = train(x, t, steps=300, batch=1 << 14, lr=3e-3)
    assert np.mean(losses[-20:]) < 0.3 * np.mean(losses[:5])
    test_w = psigen.workload("rmat", seed=999, scale=15)
    args = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
            for a in (test_w["follower"], test_w["leader"], test_w["lam"], test_w["mu"])]
    with Graph(test_w["n"], *args) as g:
        cold = g.solve(1e-8, 10000)
        psi_cold = g.scores().cpu().numpy()
        warm = model.solve(g, 1e-8, 10000)
        psi_warm = g.scores().cpu().numpy()
    assert cold["converged"] and warm["converged"]
    assert warm["iters"] < cold["iters"], (warm["iters"], cold["iters"])
    ref_psi = oracle.solve(test_w["n"], test_w["follower"], test_w["leader"], test_w["lam"], test_w["mu"],
                           to_floor=True)["psi"]
    for p in (psi_cold, psi_warm):
        assert np.abs(p - ref_psi).sum() / ref_psi.sum() <= 1e-6
    model.close()
