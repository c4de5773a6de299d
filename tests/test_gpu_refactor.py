"""Coefficients that change in time (Sec. 4): hif_set_coefficient and hif_refactor.

* hif_refactor(h, a2) on a handle built for a1 gives, bit for bit, the steps
  of a fresh hif_setup with a2 (the factorization is deterministic).
* A schedule that replaces a(x) every step and refactors every second step
  matches the oracle's cn_solve_varying on the same schedule to 1e-9, in 2D
  and 3D; for a spatially constant a(t) it matches the exact per-mode products.
* A field that makes A indefinite is refused with HIF_ENOTSPD; the handle then
  refuses to solve until a later refactor succeeds.
"""

import math

import numpy as np
import pytest

import workloads as W
from parity import rel_err
from oracle import pcg

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


def _fields(dim, n, m, seed, k, amp=0.3):
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=1e-6 if dim == 2 else 1e-4, seed=seed,
                            contrast=1e3, dt=0.5 if dim == 2 else 0.1, corr_len=0.1)
    a_seq = [w.a_nodes * (1.0 + amp * math.sin(0.7 * j)) for j in range(k)]
    return w, a_seq


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_refactor_equals_fresh_setup(H, precision):
    import torch
    w1, _ = _fields(2, 128, 16, 3, 1)
    w2, _ = _fields(2, 128, 16, 4, 1)
    opt = H.default_options(eps=1e-6, precision=precision, cg_tol=1e-10)
    a1 = torch.from_numpy(w1.a_nodes).cuda()
    a2 = torch.from_numpy(w2.a_nodes).cuda()
    h = H.hif_setup(2, 128, 16, a1, w1.dt, opt)
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    u = torch.from_numpy(w2.u0.ravel().copy()).cuda()
    H.cn_step(h, u)  # captures the solve graph of the first factor
    H.hif_refactor(h, a2)
    f = H.hif_setup(2, 128, 16, a2, w1.dt, opt)
    H.hif_set_reaction(f, 1, 1.0, 1.0)
    uh, uf = u.clone(), u.clone()
    for _ in range(3):
        uh, ih = H.cn_step(h, uh)
        uf, jf = H.cn_step(f, uf)
        assert ih == jf
    assert torch.equal(uh, uf)
    assert H.hif_query(h)["factor_entries"] == H.hif_query(f)["factor_entries"]


@pytest.mark.parametrize("dim,n,m", [(2, 64, 8), (2, 128, 16), (3, 16, 4)])
def test_varying_schedule_matches_oracle(H, dim, n, m):
    import torch
    k = 5
    w, a_seq = _fields(dim, n, m, 11, k)
    ref, it_ref = pcg.cn_solve_varying(a_seq, w.u0, w.dt, m, w.eps, (1, 1.0, 1.0), tol=1e-10,
                                       refactor_every=2)
    opt = H.default_options(eps=w.eps, cg_tol=1e-10)
    h = H.hif_setup(dim, n, m, torch.from_numpy(a_seq[0]).cuda(), w.dt, opt)
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    its = []
    for j, a in enumerate(a_seq):
        at = torch.from_numpy(a).cuda()
        if j % 2 == 0:
            H.hif_refactor(h, at)
        else:
            H.hif_set_coefficient(h, at)
        u, it = H.cn_step(h, u)
        its.append(it)
    assert _rel(u.cpu().numpy(), ref.ravel()) <= 1e-9
    assert all(abs(a - b) <= 1 for a, b in zip(its, it_ref)), (its, it_ref)


def test_spatially_constant_time_varying_matches_mode_products(H):
    import scipy.fft
    import torch
    n, m, dt = 64, 8, 2e-2
    cs = [1.0, 1.3, 0.8, 1.6, 1.1, 0.9]
    u0 = W.sine_modes_u0(n, 2, [(1, 1), (2, 3), (6, 5)], rng=np.random.default_rng(3), noise=0.05)
    ones = torch.ones((n + 1) ** 2, dtype=torch.float64).cuda()
    h = H.hif_setup(2, n, m, ones, dt, H.default_options(eps=1e-6, cg_tol=1e-12))
    u = torch.from_numpy(u0.ravel().copy()).cuda()
    for j, c in enumerate(cs):
        if j % 3 == 0:
            H.hif_refactor(h, c * ones)
        else:
            H.hif_set_coefficient(h, c * ones)
        u, _ = H.cn_step(h, u)
    hh = 1.0 / n
    ks = np.arange(1, n)
    lam1 = -(4.0 / hh ** 2) * np.sin(ks * math.pi * hh / 2) ** 2
    lam = lam1[:, None] + lam1[None, :]
    coef = scipy.fft.dstn(u0, type=1)
    for c in cs:
        coef = coef * (1 + dt * c * lam / 2) / (1 - dt * c * lam / 2)
    exact = scipy.fft.idstn(coef, type=1)
    assert _rel(u.cpu().numpy(), exact.ravel()) <= 1e-9


def test_refactor_indefinite_field_is_refused(H):
    import torch
    w, _ = _fields(2, 64, 8, 5, 1)
    a = torch.from_numpy(w.a_nodes).cuda()
    h = H.hif_setup(2, 64, 8, a, 1.0, H.default_options(eps=1e-6))
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    u1, _ = H.cn_step(h, u)
    # a < 0 turns -dt/2 M into a negative definite term: A = I - dt/2 M is indefinite
    with pytest.raises(RuntimeError, match="hif_refactor"):
        H.hif_refactor(h, -a)
    with pytest.raises(RuntimeError, match="cn_step"):
        H.cn_step(h, u)
    H.hif_refactor(h, a)
    u2, _ = H.cn_step(h, u)
    assert torch.equal(u1, u2)
