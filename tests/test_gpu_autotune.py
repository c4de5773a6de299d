"""hif_autotune: the per-level CTA cut of the apply and the leaf kernels' CTAs per
SM chosen by timing.  The tuned apply must solve the same systems: CN steps
after tuning match the steps before it to 1e-9 (both at CG tolerance 1e-10;
only the rounding order of the cell kernels may change), in FP64 and FP32,
2D and 3D; the tuned apply is not slower than the default one beyond timing
noise (the default cut is one of the candidates)."""

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


def _apply_ms(H, h, prec, reps=20):
    import torch
    x = torch.ones(h.N, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        H.hif_apply(h, x, y, precision=prec)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        H.hif_apply(h, x, y, precision=prec)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


CASES = [(2, 256, 16, 1e-6, 1.0), (3, 32, 4, 1e-4, 0.1)]


@pytest.mark.parametrize("dim,n,m,eps,dt", CASES, ids=["2d_n256_m16", "3d_n32_m4"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_autotune_keeps_the_solution(H, dim, n, m, eps, dt, precision):
    import torch
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=eps, contrast=1e3, dt=dt, corr_len=0.1, seed=31)
    h = H.hif_setup(dim, n, m, torch.from_numpy(w.a_nodes).cuda(), w.dt,
                    H.default_options(eps=eps, precision=precision, cg_tol=1e-10))
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    u0 = torch.from_numpy(w.u0.ravel().copy()).cuda()

    def steps():
        u = u0.clone()
        for _ in range(2):
            u, _ = H.cn_step(h, u)
        return u

    before = steps()
    t0 = _apply_ms(H, h, precision)
    H.hif_autotune(h)
    after = steps()
    t1 = _apply_ms(H, h, precision)
    assert float(torch.linalg.norm(after - before) / torch.linalg.norm(before)) <= 1e-9
    assert t1 <= 1.25 * t0 + 0.01, (t0, t1)
