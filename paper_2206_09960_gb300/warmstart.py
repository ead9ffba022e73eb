"""Learned warm start for Power-psi: data from solves, GPU training, use.

The network (include/psi.h, ``psi_mlp_*``) predicts log s_i of the converged iterate from
per-user features (``psi_features``); ``psi_solve_warm`` starts Algorithm 2 from
s_0 = exp(prediction).  Everything numeric runs in the CUDA library; this module only
arranges calls (which graphs to solve, which rows to sample, the Adam loop).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _binding as B
from . import Graph, _ptr

N_PARAMS = 4801


class WarmStartModel:
    def __init__(self, seed=0, stream=None):
        import torch

        B.load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = B.psi_mlp_create(seed, ctypes.c_void_p(self.stream.cuda_stream))

    def close(self):
        if getattr(self, "_h", None):
            B.psi_mlp_destroy(self._h)
            self._h = None

    __del__ = close

    def set_params(self, params=None, norm=None):
        p = None if params is None else np.ascontiguousarray(params, np.float32)
        nm = None if norm is None else np.ascontiguousarray(norm, np.float32)
        B.psi_mlp_set_params(self._h, _ptr(p), _ptr(nm))

    def get_params(self):
        p = np.empty(N_PARAMS, np.float32)
        nm = np.empty(18, np.float32)
        B.psi_mlp_get_params(self._h, _ptr(p), _ptr(nm))
        return p, nm

    def forward(self, x):
        import torch

        y = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
        B.psi_mlp_forward(self._h, x.shape[0], _ptr(x), _ptr(y))
        return y

    def grad(self, x, t, want_grad=False):
        g = np.empty(N_PARAMS, np.float32) if want_grad else None
        loss = B.psi_mlp_grad(self._h, x.shape[0], _ptr(x), _ptr(t), _ptr(g))
        return (loss, g) if want_grad else loss

    def step(self, lr):
        B.psi_mlp_adam_step(self._h, lr)

    def solve(self, graph: Graph, eps, max_iter=100000):
        st, info = B.psi_solve_warm(graph._h, self._h, eps, max_iter)
        out = info.as_dict()
        out["status"] = B.status_name(st)
        return out


def graph_features(g: Graph):
    import torch

    x = torch.empty((g.n, 8), dtype=torch.float32, device="cuda")
    B.psi_features(g._h, _ptr(x))
    return x


def training_rows(workloads, eps=1e-10, rows_per_graph=1 << 15, seed=0):
    """(x, t): features and log s of the converged iterate for users with followers, sampled
    from each workload (dicts with n, follower, leader, lam, mu)."""
    import torch

    xs, ts = [], []
    gen = torch.Generator(device="cpu").manual_seed(seed)
    for w in workloads:
        args = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (w["follower"], w["leader"], w["lam"], w["mu"])]
        with Graph(w["n"], *args) as g:
            g.solve(eps, 100000)
            s = g.iterate()
            x = graph_features(g)
        rows = torch.nonzero(x[:, 0] > 0).squeeze(1)  # users without followers have s = c exactly
        if rows.numel() > rows_per_graph:
            pick = torch.randperm(rows.numel(), generator=gen)[:rows_per_graph].to(rows.device)
            rows = rows[pick]
        xs.append(x[rows])
        ts.append(torch.log(s[rows]).float())
    return torch.cat(xs).contiguous(), torch.cat(ts).contiguous()


def train(x, t, steps=400, batch=1 << 16, lr=3e-3, seed=0, log_every=0):
    """Adam on mean squared error of normalised log s; returns (model, losses)."""
    import torch

    model = WarmStartModel(seed)
    mean = x.mean(0)
    std = x.std(0).clamp_min(1e-3)
    norm = torch.cat([mean, std, t.mean().reshape(1), t.std().clamp_min(1e-3).reshape(1)]).cpu().numpy()
    model.set_params(norm=norm)
    gen = torch.Generator(device=x.device).manual_seed(seed + 1)  # minibatch rows drawn on the device
    losses = []
    n = x.shape[0]
    for k in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=gen, device=x.device)
        xb, tb = x[idx].contiguous(), t[idx].contiguous()
        loss = model.grad(xb, tb)
        model.step(lr * (0.5 * (1 + np.cos(np.pi * k / steps))) + 1e-5)
        losses.append(loss)
        if log_every and k % log_every == 0:
            print(f"step {k} loss {loss:.4f}", flush=True)
    return model, losses
