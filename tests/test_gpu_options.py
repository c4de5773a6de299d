"""GPU parity of the time-stepping weight, warm start and direct solve options.

* theta = 1 (backward Euler): A = I - dt M and g = u + dt r; the GPU steps
  match the oracle's theta = 1 loop to 1e-9 at CG tolerance 1e-10, and for
  a = 1 the exact per-mode evolution 1 / (1 - dt lambda) of the DST-I basis.
* warm start (x0 = u_k): the solution matches the oracle's cold-start steps
  to 1e-9 and never takes more iterations than the GPU's own cold start; a
  start that is already the solution takes 0 iterations; b = 0 gives x = 0.
* direct (x = F^{-1} g): on a factor imported from the oracle the GPU step
  equals the oracle's direct step to 1e-12 (FP64) and 1e-5 (FP32).
* cn_step_batched over handles with different options equals the steps taken
  one handle at a time, bit for bit.
"""

import math

import numpy as np
import pytest

import workloads as W
from parity import rel_err
from oracle import export, grid, hif, pcg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    assert torch.cuda.is_available()
    return H


# normwise and element-by-element relative error (the larger of the two)
_rel = rel_err


def _work(n=64, m=8, dim=2, eps=1e-6, dt=0.5, seed=21):
    return W.small_variable_2d(n=n, m=m, dim=dim, eps=eps, contrast=1e3, dt=dt, corr_len=0.1,
                               seed=seed)


def _setup(H, w, **kw):
    import torch
    a = torch.from_numpy(w.a_nodes).cuda()
    opt = H.default_options(eps=w.eps, cg_tol=1e-10, **kw)
    return H.hif_setup(w.dim, w.n, w.leaf, a, w.dt, opt)


def _steps(H, h, u0, k, r_on=True):
    import torch
    if r_on:
        H.hif_set_reaction(h, 1, 1.0, 1.0)
    u = torch.from_numpy(u0.ravel().copy()).cuda()
    its = []
    for _ in range(k):
        u, it = H.cn_step(h, u)
        its.append(it)
    return u.cpu().numpy(), its


@pytest.mark.parametrize("dim,n,m", [(2, 64, 8), (2, 128, 16), (3, 16, 4)])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_backward_euler_matches_oracle(H, dim, n, m, precision):
    w = _work(n=n, m=m, dim=dim, eps=1e-6 if dim == 2 else 1e-4, dt=0.5 if dim == 2 else 0.1)
    ref, _, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 3, w.leaf, w.eps, (1, 1.0, 1.0), tol=1e-10,
                             theta=1.0)
    h = _setup(H, w, precision=precision, theta=1.0)
    u, its = _steps(H, h, w.u0, 3)
    assert _rel(u, ref.ravel()) <= 1e-9
    assert all(1 <= i <= 10 for i in its)


def test_backward_euler_matches_dst_closed_form(H):
    import scipy.fft
    n, m, dt, steps = 64, 8, 1e-2, 3
    u0 = W.sine_modes_u0(n, 2, [(1, 1), (3, 2), (7, 5)], rng=np.random.default_rng(4), noise=0.05)
    import torch
    opt = H.default_options(eps=1e-6, cg_tol=1e-12, theta=1.0)
    h = H.hif_setup(2, n, m, torch.ones((n + 1) ** 2, dtype=torch.float64).cuda(), dt, opt)
    u = torch.from_numpy(u0.ravel().copy()).cuda()
    for _ in range(steps):
        u, _ = H.cn_step(h, u)
    hh = 1.0 / n
    ks = np.arange(1, n)
    lam1 = -(4.0 / hh ** 2) * np.sin(ks * math.pi * hh / 2) ** 2
    lam = lam1[:, None] + lam1[None, :]
    exact = scipy.fft.idstn(scipy.fft.dstn(u0, type=1) * (1.0 / (1.0 - dt * lam)) ** steps, type=1)
    assert _rel(u.cpu().numpy(), exact.ravel()) <= 1e-9


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_warm_start_matches_cold_and_saves_iterations(H, precision):
    w = _work(n=128, m=16, dt=1.0)
    ref, _, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 4, w.leaf, w.eps, (1, 1.0, 1.0), tol=1e-10)
    cold = _setup(H, w, precision=precision)
    warm = _setup(H, w, precision=precision, x0_mode=1)
    uc, itc = _steps(H, cold, w.u0, 4)
    uw, itw = _steps(H, warm, w.u0, 4)
    assert _rel(uw, ref.ravel()) <= 1e-9
    assert _rel(uc, ref.ravel()) <= 1e-9
    assert sum(itw) <= sum(itc), (itw, itc)


def test_warm_start_pcg_solve_edge_cases(H):
    import torch
    w = _work(n=64, m=8)
    h = _setup(H, w, x0_mode=1)
    b = torch.from_numpy(np.random.default_rng(3).standard_normal(w.N)).cuda()
    # cold reference solve, then restart from its answer: already converged
    hc = _setup(H, w)
    x, it, rr = H.pcg_solve(hc, b)
    assert it >= 1 and rr <= 1e-10 * 1.01
    x2, it2, rr2 = H.pcg_solve(h, b, x=x.clone())
    assert it2 == 0 and rr2 <= 1e-10 * 1.01
    assert torch.equal(x2, x)
    # a start away from the solution converges to it
    x3, it3, rr3 = H.pcg_solve(h, b, x=x + 1e-3 * torch.ones_like(x))
    assert it3 >= 1 and rr3 <= 1e-10 * 1.01
    assert _rel(x3.cpu().numpy(), x.cpu().numpy()) <= 1e-9
    # b = 0: x = 0 whatever the start
    z = torch.zeros_like(b)
    x4, it4, rr4 = H.pcg_solve(h, z, x=torch.ones_like(b))
    assert it4 == 0 and rr4 == 0.0 and float(x4.abs().max()) == 0.0


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)], ids=["fp64", "fp32"])
def test_direct_step_matches_oracle_on_imported_factor(H, precision, tol):
    import torch
    w = _work(n=64, m=8, eps=1e-6, dt=1.0)
    A = grid.assemble_A(w.a_nodes, w.dt)
    F = hif.factor(A, w.n, w.dim, w.leaf, w.eps)
    blob = export.export_blob(F, w.dt)
    ref, it_ref, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 2, w.leaf, w.eps, (1, 1.0, 1.0), factor=F,
                                  direct=True)
    a = torch.from_numpy(w.a_nodes).cuda()
    opt = H.default_options(eps=w.eps, precision=precision, solver=1)
    h = H.hif_import_factor(w.dim, w.n, w.leaf, blob, w.dt, a, opt)
    u, its = _steps(H, h, w.u0, 2)
    assert its == [0, 0] and it_ref == [0, 0]
    assert _rel(u, ref.ravel()) <= tol
    # pcg_solve with the direct solver returns F^{-1} b and its true residual
    b = np.random.default_rng(5).standard_normal(w.N)
    x, it, rr = H.pcg_solve(h, torch.from_numpy(b).cuda())
    y = hif.apply_inverse(F, b)
    xh = x.cpu().numpy()
    assert it == 0 and _rel(xh, y) <= tol
    # relres is the true residual of the returned x
    assert abs(rr - np.linalg.norm(b - A @ xh) / np.linalg.norm(b)) <= 1e-6 * rr + 1e-15


def test_batched_mixed_options_equals_individual(H):
    import torch
    cfg = [dict(), dict(x0_mode=1), dict(solver=1), dict(theta=1.0), dict(theta=1.0, x0_mode=1,
                                                                        precision=1)]
    hs, us = [], []
    for i, kw in enumerate(cfg):
        w = _work(n=64, m=8, seed=40 + i)
        h = _setup(H, w, **kw)
        H.hif_set_reaction(h, 1, 1.0, 1.0)
        hs.append(h)
        us.append(torch.from_numpy(w.u0.ravel().copy()).cuda())
    ref = [H.cn_step(h, u) for h, u in zip(hs, us)]
    outs, its = H.cn_step_batched(hs, us)
    torch.cuda.synchronize()
    for (o_ref, it_ref), o, it, kw in zip(ref, outs, its, cfg):
        if kw.get("precision", 0) == 0:  # per-handle streams: the single-step kernels
            assert torch.equal(o, o_ref)
            assert it == it_ref
        else:  # merged FP32 steps: equal to the CG tolerance
            assert float(torch.linalg.norm(o - o_ref) / torch.linalg.norm(o_ref)) <= 1e-9
            assert abs(it - it_ref) <= 1
