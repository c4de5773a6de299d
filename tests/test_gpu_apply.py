"""GPU parity of the apply / matvec / PCG / CN kernels on oracle factor data.

The oracle factors A on the CPU; its factor is handed to the library through
hif_import_factor (the interchange blob), so both sides apply identical
factor data.  Bars (element-wise, relative to the norm of the reference):
FP64 apply 1e-12, FP32 apply 1e-5, PCG / CN solutions 1e-9 at tolerance
1e-10 with the same iteration count (+-1).
"""

import math

import numpy as np
import pytest

import workloads as W
from parity import rel_err
from oracle import export, grid, hif, pcg

pytestmark = pytest.mark.gpu

CASES = [
    # dim, n, leaf, eps, contrast, dt
    (2, 64, 8, 1e-6, 1e2, 1.0),
    (2, 64, 8, 1e-3, 1e4, 1.0),
    (2, 128, 16, 1e-6, 1e4, 1.0),
    (2, 32, 8, 0.0, 1e2, 0.5),
    (3, 16, 4, 1e-4, 1e3, 0.1),
    (3, 32, 8, 1e-4, 1e3, 0.1),
]
IDS = [f"{d}d_n{n}_m{m}_eps{e:g}" for d, n, m, e, _, _ in CASES]


@pytest.fixture(scope="module")
def H():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    assert torch.cuda.is_available()
    return H


_cache = {}


def _problem(case):
    if case not in _cache:
        dim, n, m, eps, contrast, dt = case
        w = W.small_variable_2d(n=n, m=m, dim=dim, eps=eps, contrast=contrast, dt=dt,
                                corr_len=0.1, seed=11)
        A = grid.assemble_A(w.a_nodes, w.dt)
        F = hif.factor(A, n, dim, m, eps)
        _cache[case] = (w, A, F, export.export_blob(F, w.dt))
    return _cache[case]


def _import(H, case, precision=0):
    import torch
    w, A, F, blob = _problem(case)
    a = torch.from_numpy(w.a_nodes).cuda()
    opt = H.default_options(eps=w.eps, precision=precision, cg_tol=1e-10)
    return H.hif_import_factor(w.dim, w.n, w.leaf, blob, w.dt, a, opt)


# normwise and element-by-element relative error (the larger of the two)
_rel = rel_err


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_matvec_matches_assembly(H, case):
    import torch
    w, A, F, blob = _problem(case)
    h = _import(H, case)
    x = np.random.default_rng(1).standard_normal(F.N)
    y = H.hif_matvec(h, torch.from_numpy(x).cuda()).cpu().numpy()
    assert _rel(y, A @ x) <= 1e-14


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_apply_fp64_matches_oracle(H, case):
    import torch
    w, A, F, blob = _problem(case)
    h = _import(H, case)
    rng = np.random.default_rng(2)
    for _ in range(3):
        x = rng.standard_normal(F.N)
        y = H.hif_apply(h, torch.from_numpy(x).cuda()).cpu().numpy()
        ref = hif.apply_inverse(F, x)
        assert _rel(y, ref) <= 1e-12
    # bitwise reproducible
    xt = torch.from_numpy(x).cuda()
    assert torch.equal(H.hif_apply(h, xt), H.hif_apply(h, xt))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_apply_fp32_matches_oracle(H, case):
    import torch
    w, A, F, blob = _problem(case)
    h = _import(H, case, precision=H.HIF_FP32)
    x = np.random.default_rng(3).standard_normal(F.N)
    y = H.hif_apply(h, torch.from_numpy(x).cuda(), precision=H.HIF_FP32).cpu().numpy()
    assert _rel(y, hif.apply_inverse(F, x)) <= 1e-5


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_apply_fused_upper_sweep_matches_oracle(H, case, precision, tol, monkeypatch):
    """HIFCN_FUSED=1: the top levels and the root in one thread-block-cluster
    kernel (opt-in; one launch per step is the default)."""
    import torch
    monkeypatch.setenv("HIFCN_FUSED", "1")
    w, A, F, blob = _problem(case)
    h = _import(H, case, precision=precision)
    x = np.random.default_rng(3).standard_normal(F.N)
    y = H.hif_apply(h, torch.from_numpy(x).cuda(), precision=precision).cpu().numpy()
    assert _rel(y, hif.apply_inverse(F, x)) <= tol


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_pcg_matches_oracle(H, case):
    import torch
    w, A, F, blob = _problem(case)
    h = _import(H, case)
    b = np.random.default_rng(4).standard_normal(F.N)
    x, it, relres = H.pcg_solve(h, torch.from_numpy(b).cuda())
    xr, itr, rr, conv = pcg.pcg(A, b, lambda v: hif.apply_inverse(F, v), tol=1e-10)
    assert abs(it - itr) <= 1
    assert relres <= 1e-10 * 1.01
    assert _rel(x.cpu().numpy(), xr) <= 1e-9


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_cn_steps_match_oracle(H, case, precision):
    import torch
    w, A, F, blob = _problem(case)
    h = _import(H, case, precision=precision)
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    ref, iters, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 3, w.leaf, w.eps, (1, 1.0, 1.0),
                                 tol=1e-10, factor=F)
    its = []
    for _ in range(3):
        u, it = H.cn_step(h, u)
        its.append(it)
    assert _rel(u.cpu().numpy(), ref.ravel()) <= 1e-9
    if precision == 0:
        assert all(abs(a - b) <= 1 for a, b in zip(its, iters)), (its, iters)


@pytest.mark.parametrize("case", CASES[:3], ids=IDS[:3])
def test_export_roundtrip_is_bitwise(H, case):
    w, A, F, blob = _problem(case)
    h = _import(H, case)
    assert H.hif_export_factor(h) == blob


def test_caller_supplied_reaction_and_aliasing(H):
    """cn_step with an explicit r_k equals the built-in reaction; u_k1 may alias u_k."""
    import torch
    case = CASES[0]
    w, A, F, blob = _problem(case)
    h = _import(H, case)
    u0 = torch.from_numpy(w.u0.ravel().copy()).cuda()
    r = (u0 * (1.0 - u0)).contiguous()
    a, _ = H.cn_step(h, u0, r=r)
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    b, _ = H.cn_step(h, u0)
    assert torch.equal(a, b)
    c = u0.clone()
    H.cn_step(h, c, out=c)
    assert torch.equal(c, b)


def test_zero_rhs_and_bad_arguments(H):
    import torch
    case = CASES[0]
    w, A, F, blob = _problem(case)
    h = _import(H, case)
    x, it, rr = H.pcg_solve(h, torch.zeros(F.N, dtype=torch.float64, device="cuda"))
    assert it == 0 and float(x.abs().max()) == 0.0
    with pytest.raises(ValueError):
        H.hif_apply(h, torch.zeros(F.N + 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(H.HifError):
        H.hif_import_factor(w.dim, w.n, w.leaf, blob[:-8], w.dt,
                            torch.from_numpy(w.a_nodes).cuda())



@pytest.mark.parametrize("period", [0, 2, 3, 7])
def test_true_residual_period_keeps_the_count(H, period):
    """The recurrence residual replaced by b - A x every `period` iterations:
    a loose factor (eps = 0.2, about 10 PCG iterations) takes the oracle's
    iteration count within one whatever the period, and each iteration is
    counted once (the recomputation finishes the iteration it belongs to)."""
    import torch
    case = (2, 64, 8, 0.2, 1e4, 1.0)
    w, A, F, blob = _problem(case)
    a = torch.from_numpy(w.a_nodes).cuda()
    opt = H.default_options(eps=w.eps, precision=0, cg_tol=1e-10, true_res_period=period)
    h = H.hif_import_factor(w.dim, w.n, w.leaf, blob, w.dt, a, opt)
    b = np.random.default_rng(9).standard_normal(F.N)
    x, it, relres = H.pcg_solve(h, torch.from_numpy(b).cuda())
    xr, itr, rr, conv = pcg.pcg(A, b, lambda v: hif.apply_inverse(F, v), tol=1e-10)
    assert itr >= 6, itr
    assert abs(it - itr) <= 1, (period, it, itr)
    assert relres <= 1e-10 * 1.01
    assert _rel(x.cpu().numpy(), xr) <= 1e-9
    h.close()
