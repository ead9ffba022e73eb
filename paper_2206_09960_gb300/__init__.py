"""GB300 Power-psi: psi-score ranking of every user of a follower graph.

The computation (graph build, Power-psi iteration, psi, ranking) runs in the CUDA library
``libpsi_gb300.so`` behind the C ABI of ``include/psi.h``.  This package marshals
arguments: numpy arrays or torch tensors (host or device) go in as pointers, device
memory comes from torch's caching allocator through the library's allocator hook, and
work is queued on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _binding as B
from ._binding import (PsiError, psi_get_iterate, psi_graph_create, psi_graph_destroy,  # noqa: F401
                       psi_graph_get_stats, psi_kernel_launches, psi_options_default, psi_scores, psi_solve,
                       psi_topk, psi_version)

__all__ = ["Graph", "Batch", "Multi", "PsiError", "psi_graph_create", "psi_solve", "psi_scores", "psi_topk",
           "psi_get_iterate", "psi_graph_get_stats", "psi_graph_destroy", "psi_options_default",
           "psi_kernel_launches", "psi_version", "load"]

load = B.load


def _ptr(x):
    """Pointer of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return ctypes.c_void_p(x.ctypes.data)
    assert x.is_contiguous()
    return ctypes.c_void_p(x.data_ptr())


class _TorchAllocator:
    """psi_allocator backed by torch.cuda.caching_allocator_alloc/delete."""

    def __init__(self, device):
        import torch

        self._torch = torch
        self._device = device

        def _alloc(nbytes, stream, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self._device, int(stream or 0)))
            except Exception:
                return None

        def _free(ptr, nbytes, stream, ctx):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self._a = B.ALLOC_FN(_alloc)
        self._f = B.FREE_FN(_free)
        self.struct = B.psi_allocator(self._a, self._f, None)


class Graph:
    """One follower graph on the GPU.

    ``follower[k]`` follows ``leader[k]`` (int32, host or device); ``lam``/``mu`` are FP64
    per-user rates.  Options mirror ``psi_options`` (precision ``fp32 | fp32_refine | fp64``,
    tol_mode ``psi | s_abs``, bnorm_mode ``none | inf``, self_loops ``reject | drop``,
    spmv_tile ``0`` (chosen from the edge count) ``| 512 | 1024 | 2048`` nonzeros per tile of
    the sparse product, autotune: time the series product's configurations on the first
    solve of a large graph and keep the fastest, spmv_hot ``-1`` (the autotuner's choice)
    ``| 0 | 24576 | 28672 | 32768`` most-gathered entries read from shared memory).
    ``allocator``: "torch" (the caching allocator), None (the library's stream-ordered
    cudaMallocAsync) or an object whose ``struct`` is a ``psi_allocator``.
    """

    def __init__(self, n, follower, leader, lam, mu, precision="fp32_refine", tol_mode="psi",
                 bnorm_mode="none", self_loops="reject", reorder=True, profile=False, stream=None,
                 allocator="torch", spmv_tile=0, autotune=True, spmv_hot=-1):
        import torch

        B.load()
        self.n = int(n)
        self._keep = [follower, leader, lam, mu]
        opt = psi_options_default()
        opt.precision = B.PRECISION[precision]
        opt.tol_mode = B.TOL_MODE[tol_mode]
        opt.bnorm_mode = B.BNORM_MODE[bnorm_mode]
        opt.self_loops = B.SELF_LOOPS[self_loops]
        opt.reorder = 1 if reorder else 0
        opt.profile = 1 if profile else 0
        opt.spmv_tile = int(spmv_tile)
        opt.autotune = 1 if autotune else 0
        opt.spmv_hot = int(spmv_hot)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        opt.stream = ctypes.c_void_p(stream.cuda_stream)
        self._alloc = None
        if allocator == "torch":
            self._alloc = _TorchAllocator(torch.cuda.current_device())
            opt.allocator = ctypes.pointer(self._alloc.struct)
        elif allocator is not None:  # any object holding a psi_allocator in .struct
            self._alloc = allocator
            opt.allocator = ctypes.pointer(allocator.struct)
        self._opt = opt
        m = int(follower.shape[0]) if follower is not None else 0
        self._h = psi_graph_create(self.n, m, _ptr(follower), _ptr(leader), _ptr(lam), _ptr(mu), opt)
        self._keep = None

    def close(self):
        if getattr(self, "_h", None):
            psi_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, eps, max_iter=10000, init_s=None) -> dict:
        st, info = psi_solve(self._h, eps, max_iter, _ptr(init_s))
        out = info.as_dict()
        out["status"] = B.status_name(st)
        return out

    def pagerank(self, alpha=0.85, eps=1e-9, max_iter=10000, out=None):
        """PageRank power method (Eq. 22) on this graph's follower structure: returns
        (pi in input order, info dict).  The graph's psi scores are left as they were."""
        import torch

        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        st, info = B.psi_pagerank(self._h, alpha, eps, max_iter, _ptr(out))
        d = info.as_dict()
        d["status"] = B.status_name(st)
        return out, d

    def power_nf(self, eps, max_iter=10000, out=None, origins_per_pass=0):
        """Power-NF (Algorithm 1) for every origin of this graph (at most 2^20 users with
        leaders), ``origins_per_pass`` origins at a time (0: as many as a quarter of the free
        device memory holds, 6 to 32 GiB): returns (psi in input order, info dict; iters =
        the most steps of an origin, spmv_launches = the matrix-vector products summed over
        origins).  The graph's psi scores are left as they were."""
        import torch

        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        st, d = B.psi_power_nf(self._h, eps, max_iter, origins_per_pass, _ptr(out))
        d["status"] = B.status_name(st)
        return out, d

    def scores(self, out=None):
        """psi of every user (FP64) into ``out`` (tensor/array, host or device) or a new CUDA tensor."""
        import torch

        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        psi_scores(self._h, _ptr(out))
        return out

    def iterate(self, out=None):
        import torch

        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        psi_get_iterate(self._h, _ptr(out))
        return out

    def topk(self, k, ids=None, vals=None):
        import torch

        if ids is None:
            ids = torch.empty(k, dtype=torch.int32, device="cuda")
        if vals is None:
            vals = torch.empty(k, dtype=torch.float64, device="cuda")
        psi_topk(self._h, k, _ptr(ids), _ptr(vals))
        return ids, vals

    def stats(self) -> dict:
        return psi_graph_get_stats(self._h).as_dict()


class Batch:
    """S activity scenarios on one follower graph, solved together.

    ``lam``/``mu`` are [S, n] FP64 (scenario-major), host or device; 1 <= S <= 64."""

    def __init__(self, n, follower, leader, lam, mu, tol_mode="psi", bnorm_mode="none", self_loops="reject",
                 reorder=True, stream=None, allocator="torch", spmv_tile=0, profile=False):
        import torch

        B.load()
        self.n = int(n)
        self.S = int(lam.shape[0])
        opt = psi_options_default()
        opt.precision = B.PSI_FP32_REFINE
        opt.tol_mode = B.TOL_MODE[tol_mode]
        opt.bnorm_mode = B.BNORM_MODE[bnorm_mode]
        opt.self_loops = B.SELF_LOOPS[self_loops]
        opt.reorder = 1 if reorder else 0
        opt.profile = 1 if profile else 0
        opt.spmv_tile = int(spmv_tile)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        opt.stream = ctypes.c_void_p(stream.cuda_stream)
        self._alloc = None
        if allocator == "torch":
            self._alloc = _TorchAllocator(torch.cuda.current_device())
            opt.allocator = ctypes.pointer(self._alloc.struct)
        self._opt = opt
        m = int(follower.shape[0]) if follower is not None else 0
        self._h = B.psi_batch_create(self.n, m, _ptr(follower), _ptr(leader), self.S, _ptr(lam), _ptr(mu), opt)

    def close(self):
        if getattr(self, "_h", None):
            B.psi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, eps, max_iter=10000):
        st, infos = B.psi_batch_solve(self._h, eps, max_iter, self.S)
        return B.status_name(st), [i.as_dict() for i in infos]

    def scores(self, out=None):
        import torch

        if out is None:
            out = torch.empty((self.S, self.n), dtype=torch.float64, device="cuda")
        B.psi_batch_scores(self._h, _ptr(out))
        return out

    def topk(self, k):
        import torch

        ids = torch.empty((self.S, k), dtype=torch.int32, device="cuda")
        vals = torch.empty((self.S, k), dtype=torch.float64, device="cuda")
        B.psi_batch_topk(self._h, k, _ptr(ids), _ptr(vals))
        return ids, vals

    def stats(self) -> dict:
        return B.psi_batch_get_stats(self._h).as_dict()


class Multi:
    """G independent follower graphs solved together (one block-diagonal build, per-graph
    N_g, stop tests and step counts, steps replayed from a CUDA graph).

    ``n_g``, ``m_g``: per-graph user and edge counts; ``follower``/``leader``: the graphs'
    edge lists one after another, ids local to each graph; ``lam``/``mu``: the graphs' rates
    one after another (sum of n_g values).  Host (numpy) or device (torch) arrays."""

    def __init__(self, n_g, m_g, follower, leader, lam, mu, tol_mode="psi", bnorm_mode="none",
                 self_loops="reject", reorder=True, stream=None, allocator="torch", spmv_tile=0):
        import torch

        B.load()
        self.n_g = np.ascontiguousarray(n_g, dtype=np.int64)
        self.m_g = np.ascontiguousarray(m_g, dtype=np.int64)
        self.G = int(self.n_g.shape[0])
        self.n = int(self.n_g.sum())
        opt = psi_options_default()
        opt.precision = B.PSI_FP32_REFINE
        opt.tol_mode = B.TOL_MODE[tol_mode]
        opt.bnorm_mode = B.BNORM_MODE[bnorm_mode]
        opt.self_loops = B.SELF_LOOPS[self_loops]
        opt.reorder = 1 if reorder else 0
        opt.spmv_tile = int(spmv_tile)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        opt.stream = ctypes.c_void_p(stream.cuda_stream)
        self._alloc = None
        if allocator == "torch":
            self._alloc = _TorchAllocator(torch.cuda.current_device())
            opt.allocator = ctypes.pointer(self._alloc.struct)
        self._opt = opt
        self._h = B.psi_multi_create(self.G, _ptr(self.n_g), _ptr(self.m_g), _ptr(follower), _ptr(leader),
                                     _ptr(lam), _ptr(mu), opt)

    def close(self):
        if getattr(self, "_h", None):
            B.psi_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, eps, max_iter=10000):
        st, infos = B.psi_multi_solve(self._h, eps, max_iter, self.G)
        return B.status_name(st), [i.as_dict() for i in infos]

    def scores(self, out=None):
        import torch

        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        B.psi_multi_scores(self._h, _ptr(out))
        return out

    def topk(self, k):
        import torch

        ids = torch.empty((self.G, k), dtype=torch.int32, device="cuda")
        vals = torch.empty((self.G, k), dtype=torch.float64, device="cuda")
        B.psi_multi_topk(self._h, k, _ptr(ids), _ptr(vals))
        return ids, vals

    def stats(self) -> dict:
        return B.psi_multi_get_stats(self._h).as_dict()
