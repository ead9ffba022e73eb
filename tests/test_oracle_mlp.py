"""Pins of the warm-start network's CPU reference (oracle/mlp.py), on CPU.

The network only proposes Algorithm 2's start vector, so the paper fixes none of its
values; what fixes them is mathematics:
  * GELU(z) = z * Phi(z), with Phi the standard normal distribution function, checked at
    points where Phi is tabulated (values to ten decimals from standard tables);
  * the derivative of GELU against central differences of GELU;
  * a network whose output is worked out by hand from those tabulated values (this also
    fixes the parameter layout: W[i][j] feeds unit i of a layer into unit j of the next);
  * the gradient of the loss against central differences of the loss, parameter by
    parameter, with the BF16 rounding switched off so the loss is smooth.
Each planted mistake at the end (a dropped term of GELU's derivative, a transposed W2
gradient) must make one of these checks fail."""
import numpy as np
import pytest

from oracle import mlp

# Phi(z) of the standard normal distribution, from printed tables
PHI = {0.5: 0.6914624613, 1.0: 0.8413447461, 1.5: 0.9331927987, 2.0: 0.9772498681, 3.0: 0.9986501020}


def test_gelu_at_tabulated_points():
    for z, phi in PHI.items():
        assert abs(mlp.gelu(np.float64(z)) - z * phi) <= 2e-10
        assert abs(mlp.gelu(np.float64(-z)) - (-z) * (1.0 - phi)) <= 2e-10
    assert mlp.gelu(np.float64(0.0)) == 0.0


def _central(f, z, h):
    return (f(z + h) - f(z - h)) / (2 * h)


def _check_gelu_grad(gelu_grad):
    z = np.linspace(-6, 6, 241)
    fd = _central(mlp.gelu, z, 1e-5)
    return float(np.max(np.abs(gelu_grad(z) - fd)))


def test_gelu_grad_against_central_differences():
    assert _check_gelu_grad(mlp.gelu_grad) <= 1e-8
    # at 0 the derivative is exactly 1/2
    assert mlp.gelu_grad(np.float64(0.0)) == 0.5


def _hand_network():
    """x = e_0 (normalisation mean 0, std 1); z1_0 = 1, z1_1 = -1 (bias); z2_0 = a*GELU(1) +
    b*GELU(-1) = 2; output (GELU(2) + b3) * t_std + t_mean.  W2[0][1] = 7 sits at the
    transposed position of W2[1][0]: it feeds z2_1, which the output ignores (W3[1] = 0)."""
    p = mlp.unpack(np.zeros(mlp.N_PARAMS))
    g1, gm1 = PHI[1.0], -(1.0 - PHI[1.0])
    b = 1.0
    a = (2.0 - b * gm1) / g1
    p["W1"][0, 0] = 1.0
    p["b1"][1] = -1.0
    p["W2"][0, 0] = a
    p["W2"][1, 0] = b
    p["W2"][0, 1] = 7.0
    p["W3"][0] = 1.0
    p["b3"][0] = 0.25
    params = np.concatenate([p[name].ravel() for name, _ in mlp.SIZES])
    norm = np.concatenate([np.zeros(8), np.ones(8), [0.5], [2.0]])
    x = np.zeros((1, 8))
    x[0, 0] = 1.0
    want = (2.0 * PHI[2.0] + 0.25) * 2.0 + 0.5
    return params, norm, x, want


def test_forward_of_a_hand_computed_network():
    params, norm, x, want = _hand_network()
    got = mlp.forward(params, norm, x, bf16_round=False)
    assert abs(got[0] - want) <= 1e-8, (got, want)


def test_forward_rounds_like_bf16_when_asked():
    # 1 + 2^-9 is not a BF16 value (7 fraction bits): it rounds to 1
    params, norm, x, want = _hand_network()
    x2 = x.copy()
    x2[0, 0] = 1.0 + 2.0 ** -9
    assert mlp.forward(params, norm, x2, bf16_round=True)[0] == pytest.approx(
        mlp.forward(params, norm, x, bf16_round=True)[0], abs=0)
    assert mlp.forward(params, norm, x2, bf16_round=False)[0] != mlp.forward(params, norm, x, bf16_round=False)[0]


def _problem(seed=0, rows=7):
    rng = np.random.default_rng(seed)
    params = rng.standard_normal(mlp.N_PARAMS) * 0.3
    norm = np.concatenate([rng.normal(0, 1, 8), rng.uniform(0.5, 2, 8), [1.5], [2.0]])
    x = rng.normal(0, 1.5, (rows, 8))
    t = rng.normal(1.0, 2.0, rows)
    return params, norm, x, t


def _fd_gradient(params, norm, x, t, h=1e-6):
    g = np.empty_like(params)
    for i in range(params.size):
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        g[i] = (mlp.loss_and_grad(pp, norm, x, t, bf16_round=False)[0]
                - mlp.loss_and_grad(pm, norm, x, t, bf16_round=False)[0]) / (2 * h)
    return g


def _gradient_error(grad_fn, problem):
    params, norm, x, t = problem
    _, g = grad_fn(params, norm, x, t, bf16_round=False)
    fd = _fd_gradient(params, norm, x, t)
    errs = {}
    o = 0
    for name, shape in mlp.SIZES:
        k = int(np.prod(shape))
        errs[name] = float(np.max(np.abs(g[o:o + k] - fd[o:o + k])) / max(np.max(np.abs(fd[o:o + k])), 1e-12))
        o += k
    return errs


@pytest.fixture(scope="module")
def problem():
    return _problem()


def test_loss_is_the_mean_squared_normalised_error(problem):
    params, norm, x, t = problem
    loss, _ = mlp.loss_and_grad(params, norm, x, t, bf16_round=False)
    y = mlp.forward(params, norm, x, bf16_round=False)
    tn = (t - norm[16]) / norm[17]
    yn = (y - norm[16]) / norm[17]
    assert loss == pytest.approx(float(np.mean((yn - tn) ** 2)), rel=1e-12)


def test_gradient_against_central_differences(problem):
    errs = _gradient_error(mlp.loss_and_grad, problem)
    assert max(errs.values()) <= 1e-6, errs


def test_planted_mistakes_are_caught(problem, monkeypatch):
    # 1. GELU's derivative without its second term
    def grad_dropped(z):
        return 0.5 * (1.0 + mlp.erf(z / np.sqrt(2.0)))

    assert _check_gelu_grad(grad_dropped) > 1e-2
    with monkeypatch.context() as m:
        m.setattr(mlp, "gelu_grad", grad_dropped)
        assert max(_gradient_error(mlp.loss_and_grad, problem).values()) > 1e-2

    # 2. the W2 block of the gradient transposed
    o = sum(int(np.prod(s)) for name, s in mlp.SIZES[:2])

    def transposed(params, norm, x, t, bf16_round=True):
        loss, g = mlp.loss_and_grad(params, norm, x, t, bf16_round=bf16_round)
        g = g.copy()
        g[o:o + 64 * 64] = g[o:o + 64 * 64].reshape(64, 64).T.ravel()
        return loss, g

    errs = _gradient_error(transposed, problem)
    assert errs["W2"] > 1e-2 and errs["W1"] <= 1e-6
