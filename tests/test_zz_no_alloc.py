"""psi_topk_noalloc: the ranking entry point for callers that cannot let the library
allocate device memory (a process whose device memory is all reserved up front in its own
arena, or owned by a host framework's allocator).  It must return exactly what psi_topk
returns for the same psi, and exactly the CPU oracle's ranking, call after call, while using
only its fixed internal working area.  This file runs last so that a failure here never
hides another test's result."""
import ctypes

import numpy as np
import pytest

import oracle
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
def test_noalloc_topk_matches_psi_topk_and_the_oracle(scale, k, homogeneous):
    g, psi, n = _graph_and_psi(3, scale, homogeneous)
    with g:
        ids_ref, vals_ref = g.topk(k)
        ids_ref, vals_ref = ids_ref.cpu().numpy(), vals_ref.cpu().numpy()
        ids_orc, vals_orc = oracle.topk(psi.cpu().numpy(), k)
        for _ in range(2):  # two calls in a row share (and must reset) the working area
            ids, vals = _noalloc(psi, n, k)
            np.testing.assert_array_equal(ids, ids_ref)
            np.testing.assert_array_equal(vals, vals_ref)
            np.testing.assert_array_equal(ids, ids_orc)
            np.testing.assert_array_equal(vals, vals_orc)


def test_noalloc_ranks_negative_zero_negatives_and_ties_like_the_oracle():
    import torch

    rng = np.random.default_rng(5)
    n = 20000
    x = rng.choice(np.array([0.0, -0.0, 1e-300, 5e-324, 2.0, -3.0, 0.5]), size=n)
    x[rng.integers(0, n, 200)] = rng.random(200)
    d = torch.from_numpy(x).cuda()
    for k in (1, 100, 4096):
        ids_orc, vals_orc = oracle.topk(x, k)
        for _ in range(2):
            ids, vals = _noalloc(d, n, k)
            np.testing.assert_array_equal(ids, ids_orc)
            np.testing.assert_array_equal(vals.view(np.uint64), x[ids_orc].view(np.uint64))
    # -0.0 ranks as 0.0: among equal zeros the smaller id comes first whatever the sign
    z = np.array([-0.0, 0.0, -0.0, 0.0, -1.0])
    ids, _ = _noalloc(torch.from_numpy(z).cuda(), 5, 5)
    np.testing.assert_array_equal(ids, [0, 1, 2, 3, 4])
    # a NaN ranks above every number
    q = np.array([1.0, np.nan, np.inf, 2.0])
    ids, _ = _noalloc(torch.from_numpy(q).cuda(), 4, 4)
    np.testing.assert_array_equal(ids, [1, 2, 3, 0])


def test_noalloc_allocates_no_device_memory():
    import torch

    g, psi, n = _graph_and_psi(4, 12)
    with g:
        _noalloc(psi, n, 100)  # the first call looks the working area up
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        reserved0 = torch.cuda.memory_reserved()
        for _ in range(5):
            _noalloc(psi, n, 100)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_reserved() == reserved0


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
    got, vals = _noalloc(psi, n, 10)
    want, want_vals = oracle.topk(psi.cpu().numpy(), 10)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(vals, want_vals)


def test_noalloc_rejects_memory_of_another_device():
    import torch
    from paper_2206_09960_gb300 import PsiError, _binding as B

    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second GPU")
    psi = torch.rand(1000, dtype=torch.float64, device="cuda:1")
    ids = torch.empty(10, dtype=torch.int32, device="cuda:0")
    with torch.cuda.device(0), pytest.raises(PsiError) as e:
        B.psi_topk_noalloc(ctypes.c_void_p(psi.data_ptr()), 1000, 10, ctypes.c_void_p(ids.data_ptr()), None, None)
    assert e.value.status == B.PSI_ERR_INVALID_ARG
