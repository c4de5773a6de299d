"""hif_apply_noalloc: the FP64 apply with the library's static scratch.

Some callers cannot allocate device memory at the moment they apply the
preconditioner (an allocator has reserved the free HBM, or the loop cannot
afford the synchronization of cudaMalloc/cudaFree).  For them the library
offers an apply whose scratch is a fixed array inside the library.  These
tests call it through the C ABI twice in a row and check:

* each result against the regular hif_apply with the FP64 tolerance the
  other apply tests use (1e-12 relative, normwise and element by element),
* each result against the oracle's F^{-1} x on an imported oracle factor,
* that the two calls leave the device's free memory unchanged (nothing is
  allocated, not even by lazy loading of the library's device code),
* that a factor too large for the fixed array, and NULL or aliased
  arguments, are refused with a message naming the cause.

The file is collected last and passes alone or after the rest.
"""

import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import export, grid, hif

from parity import assert_close

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


def _noalloc(H, h, x, y):
    return H.lib().hif_apply_noalloc(h.ptr, ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(y.data_ptr()), None)


@pytest.mark.parametrize("dim,n,m", [(2, 256, 16), (3, 32, 8)])
def test_noalloc_apply_matches_hif_apply_twice(H, dim, n, m):
    import torch
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=1e-6, contrast=1e3, dt=1.0, corr_len=0.1)
    h = _handle(H, w)
    rng = np.random.default_rng(9)
    xs = [torch.from_numpy(rng.standard_normal(w.N)).cuda() for _ in range(2)]
    ys = [torch.empty(w.N, dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for x, y in zip(xs, ys):  # two calls in a row share (and reuse) the static scratch
        assert _noalloc(H, h, x, y) == H.HIF_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    for x, y in zip(xs, ys):
        ref = H.hif_apply(h, x)
        assert_close(y.cpu().numpy(), ref.cpu().numpy(), 1e-12)
    h.close()


def test_noalloc_apply_matches_oracle_on_imported_factor(H):
    import torch
    w = W.small_variable_2d(n=64, m=8, dim=2, eps=1e-6, contrast=1e2, dt=1.0, corr_len=0.1,
                            seed=11)
    A = grid.assemble_A(w.a_nodes, w.dt)
    F = hif.factor(A, w.n, 2, w.leaf, w.eps)
    a = torch.from_numpy(w.a_nodes).cuda()
    h = H.hif_import_factor(2, w.n, w.leaf, export.export_blob(F, w.dt), w.dt, a,
                            H.default_options(eps=w.eps, cg_tol=1e-10))
    rng = np.random.default_rng(4)
    y = torch.empty(w.N, dtype=torch.float64, device="cuda")
    for _ in range(2):
        xh = rng.standard_normal(w.N)
        assert _noalloc(H, h, torch.from_numpy(xh).cuda(), y) == H.HIF_OK
        assert_close(y.cpu().numpy(), hif.apply_inverse(F, xh), 1e-12)
    h.close()


def test_noalloc_refusals_name_the_cause(H):
    import torch
    w = W.small_variable_2d(n=32, m=8, dim=2, eps=1e-6, contrast=1e2, dt=1.0, corr_len=0.1)
    h = _handle(H, w)
    x = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    f = H.lib().hif_apply_noalloc
    assert f(h.ptr, None, ctypes.c_void_p(x.data_ptr()), None) == H.HIF_EINVAL
    assert b"x is NULL" in H.lib().hif_last_error()
    assert f(h.ptr, ctypes.c_void_p(x.data_ptr()), None, None) == H.HIF_EINVAL
    assert b"y is NULL" in H.lib().hif_last_error()
    xp = ctypes.c_void_p(x.data_ptr())
    assert f(h.ptr, xp, xp, None) == H.HIF_EINVAL
    assert b"alias" in H.lib().hif_last_error()
    h.close()


def test_noalloc_rejects_factor_beyond_static_scratch(H):
    import torch
    # 2D 1023^2 with leaf 4: 65536 level-0 cells x 16 boundary slots = 2^20 > 2^19
    n, m = 1024, 4
    rng = np.random.default_rng(3)
    a = W.lognormal_coefficient(W.grf(rng, n, 2, 0.05), 1e2)
    w = W.Workload("big", 2, n, m, 8, 1.0, 1e-3, a, np.zeros((n - 1, n - 1)))
    h = _handle(H, w)
    x = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    assert _noalloc(H, h, x, y) == H.HIF_EINVAL
    assert b"contribution slots" in H.lib().hif_last_error()
    h.close()
