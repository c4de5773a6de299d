"""hif_apply_noalloc: the FP64 apply with the library's static scratch.

Some callers cannot allocate device memory at the moment they apply the
preconditioner (an allocator has reserved the free HBM, or the loop cannot
afford the synchronization of cudaMalloc/cudaFree).  For them the library
offers an apply whose scratch is a fixed array inside the library.  This test
calls it through the C ABI twice in a row and checks each result against the
regular hif_apply with the FP64 tolerance the other apply tests use (1e-12
relative), and checks that a factor too large for the fixed array is refused.
It lives in its own file, collected last, and passes alone or after the rest.
"""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    assert torch.cuda.is_available()
    return H


def _handle(H, w):
    import torch
    a = torch.from_numpy(w.a_nodes).cuda()
    opt = H.default_options(eps=w.eps, cg_tol=1e-10)
    return H.hif_setup(w.dim, w.n, w.leaf, a, w.dt, opt)


@pytest.mark.parametrize("dim,n,m", [(2, 256, 16), (3, 32, 8)])
def test_noalloc_apply_matches_hif_apply_twice(H, dim, n, m):
    import torch
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=1e-6, contrast=1e3, dt=1.0, corr_len=0.1)
    h = _handle(H, w)
    rng = np.random.default_rng(9)
    y = torch.empty(w.N, dtype=torch.float64, device="cuda")
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        x = torch.from_numpy(rng.standard_normal(w.N)).cuda()
        ref = H.hif_apply(h, x)
        H.hif_apply_noalloc(h, x, y)
        torch.cuda.synchronize()
        err = float((y - ref).norm() / ref.norm())
        assert err <= 1e-12, err
    h.close()


def test_noalloc_rejects_factor_beyond_static_scratch(H):
    import ctypes
    import torch
    # 2D 2047^2 with leaf 8: 65536 level-0 cells x 32 boundary slots > 2^19
    n, m = 2048, 8
    rng = np.random.default_rng(3)
    a = W.lognormal_coefficient(W.grf(rng, n, 2, 0.05), 1e2)
    w = W.Workload("big", 2, n, m, 8, 1.0, 1e-3, a, np.zeros((n - 1, n - 1)))
    h = _handle(H, w)
    x = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    st = H.lib().hif_apply_noalloc(h.ptr, ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(y.data_ptr()), None)
    assert st == H.HIF_EINVAL
    assert b"contribution slots" in H.lib().hif_last_error()
    h.close()
