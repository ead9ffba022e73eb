"""psi_topk_noalloc: the ranking entry point for callers that cannot let the library
allocate device memory (a process whose device memory is all reserved up front in its own
arena, or owned by a host framework's allocator).  It must return exactly what psi_topk
returns for the same psi, call after call, while using only its fixed internal working
area.  This file runs last so that a failure here never hides another test's result."""
import ctypes

import numpy as np
import pytest

import psigen

pytestmark = pytest.mark.gpu


def _graph_and_psi(seed, scale, homogeneous=False):
    import torch
    from paper_2206_09960_gb300 import Graph

    w = psigen.workload("rmat", seed=seed, scale=scale)
    n = w["n"]
    lam, mu = (np.full(n, 0.15), np.full(n, 0.85)) if homogeneous else (w["lam"], w["mu"])
    args = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (w["follower"], w["leader"], lam, mu)]
    g = Graph(n, *args)
    g.solve(1e-8, 10000)
    return g, g.scores(), n


def _noalloc(psi, n, k):
    import torch
    from paper_2206_09960_gb300 import _binding as B

    ids = torch.full((k,), -7, dtype=torch.int32, device="cuda")
    vals = torch.full((k,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    B.psi_topk_noalloc(ctypes.c_void_p(psi.data_ptr()), n, k, ctypes.c_void_p(ids.data_ptr()),
                       ctypes.c_void_p(vals.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return ids.cpu().numpy(), vals.cpu().numpy()


@pytest.mark.parametrize("scale,k,homogeneous", [(14, 100, False), (13, 4096, False), (12, 1, False),
                                                 (12, 300, True)])
def test_noalloc_topk_matches_psi_topk(scale, k, homogeneous):
    g, psi, n = _graph_and_psi(3, scale, homogeneous)
    with g:
        ids_ref, vals_ref = g.topk(k)
        ids_ref, vals_ref = ids_ref.cpu().numpy(), vals_ref.cpu().numpy()
        for _ in range(2):  # two calls in a row share (and must reset) the working area
            ids, vals = _noalloc(psi, n, k)
            np.testing.assert_array_equal(ids, ids_ref)
            np.testing.assert_array_equal(vals, vals_ref)


def test_noalloc_rejects_sizes_beyond_the_limit():
    import torch
    from paper_2206_09960_gb300 import PsiError, _binding as B

    n = 5000
    psi = torch.rand(n, dtype=torch.float64, device="cuda")
    ids = torch.empty(4097, dtype=torch.int32, device="cuda")
    with pytest.raises(PsiError) as e:
        B.psi_topk_noalloc(ctypes.c_void_p(psi.data_ptr()), n, 4097, ctypes.c_void_p(ids.data_ptr()), None, None)
    assert e.value.status == B.PSI_ERR_INVALID_ARG
    host_ids = np.empty(10, np.int32)
    with pytest.raises(PsiError) as e:
        B.psi_topk_noalloc(ctypes.c_void_p(psi.data_ptr()), n, 10, ctypes.c_void_p(host_ids.ctypes.data), None, None)
    assert e.value.status == B.PSI_ERR_INVALID_ARG
    # a valid call still works after the rejected ones
    got, _ = _noalloc(psi, n, 10)
    want = np.argsort(-psi.cpu().numpy(), kind="stable")[:10]
    np.testing.assert_array_equal(got, want)
