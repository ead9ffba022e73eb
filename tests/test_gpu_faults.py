"""Failure handling on the GPU path without a GPU fault: allocation failures injected through
the allocator hook (psi_options.allocator) at many points of graph creation and solve must
come back as PSI_ERR_OOM, leave nothing allocated once the handle is gone, and leave the
library usable."""
import ctypes

import numpy as np
import pytest

import psigen

pytestmark = pytest.mark.gpu


class _CountingAllocator:
    """Torch caching allocator behind a psi_allocator that counts calls and live bytes and
    can refuse the k-th allocation (returns NULL)."""

    def __init__(self, fail_at=None):
        import torch

        from paper_2206_09960_gb300 import _binding as B

        self.calls = 0
        self.live = 0
        self.fail_at = fail_at
        dev = torch.cuda.current_device()

        def _alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.fail_at is not None and self.calls == self.fail_at:
                return None
            p = int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0)))
            self.live += int(nbytes)
            return p

        def _free(ptr, nbytes, stream, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))
            self.live -= int(nbytes)

        self._a = B.ALLOC_FN(_alloc)
        self._f = B.FREE_FN(_free)
        self.struct = B.psi_allocator(self._a, self._f, None)


def _run(w, alloc):
    from paper_2206_09960_gb300 import Graph

    with Graph(w["n"], w["follower"], w["leader"], w["lam"], w["mu"], allocator=alloc) as g:
        info = g.solve(1e-8, 1000)
        g.topk(10)
    return info


def test_allocation_failures_become_statuses_and_leak_nothing():
    from paper_2206_09960_gb300 import PsiError, _binding as B

    w = psigen.workload("rmat", seed=31, scale=11)
    ok = _CountingAllocator()
    ref = _run(w, ok)
    total = ok.calls
    assert total > 10 and ok.live == 0
    points = sorted({1, 2, 3, total // 4, total // 2, (3 * total) // 4, total - 1, total})
    for k in points:
        a = _CountingAllocator(fail_at=k)
        with pytest.raises(PsiError) as e:
            _run(w, a)
        assert e.value.status == B.PSI_ERR_OOM, (k, e.value.status)
        assert a.live == 0, (k, a.live)
    # the library still works, with the same result
    again = _run(w, _CountingAllocator())
    assert again["iters"] == ref["iters"] and again["psi_sum"] == ref["psi_sum"]


def test_library_pool_and_trim():
    """Without a caller allocator the library uses its own pool; results match the torch
    allocator's bit for bit, and psi_trim_memory returns the cached memory."""
    from paper_2206_09960_gb300 import Graph, _binding as B

    w = psigen.workload("rmat", seed=32, scale=11)
    outs = []
    for alloc in (None, "torch"):
        with Graph(w["n"], w["follower"], w["leader"], w["lam"], w["mu"], allocator=alloc) as g:
            g.solve(1e-8, 1000)
            outs.append(g.scores().cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    assert B.load().psi_trim_memory() == B.PSI_OK
