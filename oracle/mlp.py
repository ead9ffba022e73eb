"""FP64 CPU reference of the warm-start network (TEST INFRASTRUCTURE ONLY).

The network is not part of the paper's method: it only proposes the start vector s_0 of
Algorithm 2 (whose fixed point does not depend on s_0). This module is the plain reference
its GPU forward and backward kernels are checked against: 8 -> 64 -> 64 -> 1 with exact
GELU, x -> (x - mean) / std rounded to BF16, weights rounded to BF16, every sum in FP64.
Loss: mean over rows of (yhat - (t - t_mean) / t_std)^2.

Both routines take ``bf16_round``: True (default) rounds every operand of every matrix
product to BF16, as the GPU's BF16-in/FP32-accumulate kernels do -- the weights, the
normalised inputs, the hidden activations h1 and h2, and in the backward pass the
pre-activation gradients dz2 and dz1 where they enter a product -- while element-wise work
and the bias sums stay unrounded; False keeps everything in FP64, which makes the loss a
smooth function of the parameters so the gradient can be checked against finite
differences.

Parity pins (``tests/test_oracle_mlp.py``, CPU): ``gelu`` against tabulated values of the
standard normal distribution function; ``gelu_grad`` against central differences of
``gelu``; ``forward`` against a network whose output is worked out by hand from those
tabulated values; ``loss_and_grad`` against central differences of the loss, parameter by
parameter, with the rounding off.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

K_IN, K_H = 8, 64
SIZES = [("W1", (K_IN, K_H)), ("b1", (K_H,)), ("W2", (K_H, K_H)), ("b2", (K_H,)), ("W3", (K_H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)  # 4801


def bf16(x):
    """Round float32 values to the nearest BF16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params):
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(params[o:o + k], np.float64).reshape(shape)
        o += k
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def _r(a, bf16_round):
    """A product operand: BF16-rounded when the kernels' rounding is modelled."""
    return bf16(a) if bf16_round else a


def _inputs(params, norm, x, bf16_round):
    if bf16_round:
        p = {k: bf16(v) for k, v in unpack(params).items()}
        xn = bf16((np.asarray(x, np.float32) - np.float32(norm[:K_IN])) / np.float32(norm[K_IN:2 * K_IN]))
    else:
        p = unpack(params)
        xn = (np.asarray(x, np.float64) - np.asarray(norm[:K_IN], np.float64)) / np.asarray(norm[K_IN:2 * K_IN],
                                                                                             np.float64)
    return p, xn


def forward(params, norm, x, bf16_round=True):
    """Predicted log s (de-normalised)."""
    p, xn = _inputs(params, norm, x, bf16_round)
    h1 = _r(gelu(xn @ p["W1"] + p["b1"]), bf16_round)
    h2 = _r(gelu(h1 @ p["W2"] + p["b2"]), bf16_round)
    y = h2 @ p["W3"] + p["b3"][0]
    return y * norm[2 * K_IN + 1] + norm[2 * K_IN]


def loss_and_grad(params, norm, x, t, bf16_round=True):
    """(loss, gradient[4801]) with respect to the (BF16-rounded, unless bf16_round is False)
    parameters."""
    p, xn = _inputs(params, norm, x, bf16_round)
    tn = (np.asarray(t, np.float64) - norm[2 * K_IN]) / norm[2 * K_IN + 1]
    z1 = xn @ p["W1"] + p["b1"]
    h1 = _r(gelu(z1), bf16_round)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = _r(gelu(z2), bf16_round)
    y = h2 @ p["W3"] + p["b3"][0]
    e = y - tn
    B = x.shape[0]
    loss = float(np.mean(e * e))
    dy = 2.0 * e / B
    dz2 = np.outer(dy, p["W3"]) * gelu_grad(z2)
    dz2r = _r(dz2, bf16_round)
    dz1 = (dz2r @ p["W2"].T) * gelu_grad(z1)
    g = {"W3": h2.T @ dy, "b3": np.array([dy.sum()]), "W2": h1.T @ dz2r, "b2": dz2.sum(0),
         "W1": xn.T @ _r(dz1, bf16_round), "b1": dz1.sum(0)}
    return loss, np.concatenate([g[name].ravel() for name, _ in SIZES])
