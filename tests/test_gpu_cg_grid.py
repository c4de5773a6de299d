"""The PCG vector kernels with many elements per thread, at oracle sizes.

k_cg_wz (w = A z with the dots r.z, w.z, q.z) and k_cg_update (the p, q, x, r
updates with r.r) carry out the pcg call of Algorithm 1.  Each thread walks
the unknowns by the grid stride and loads the operands of its next element
before the arithmetic of the current one.  At the sizes the oracle factors in
seconds, the default grid gives every thread at most one element.
HIFCN_CG_GRID caps the grid of these two kernels, so that the pipelined loop
runs many times per thread: with 1 block of 256 threads a thread takes about
15 elements of the 2D 63^2 grid and 13 of the 3D 15^3 grid; with 3 blocks it
takes about 5 (a ragged last pass).  The stencil neighbours cross grid rows
and planes inside one thread's walk.

Bars, as for the default launch shape: CN steps (Eq. CN2, the captured
solve) and PCG solves at CG tolerance 1e-10 match the oracle to 1e-9
relative (normwise and element by element); the iteration counts of the
FP64 path are within 1 of the oracle's.
"""

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


CASES = [
    # dim, n, leaf, eps, contrast, dt
    (2, 64, 8, 1e-6, 1e2, 1.0),
    (3, 16, 4, 1e-4, 1e3, 0.1),
]
IDS = [f"{d}d_n{n}_m{m}" for d, n, m, _, _, _ in CASES]
CAPS = ["1", "3"]
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


def _import(H, case, precision):
    import torch
    w, A, F, blob = _problem(case)
    dim, n, m, eps, _, _ = case
    opt = H.default_options(eps=eps, precision=precision, cg_tol=1e-10)
    return H.hif_import_factor(dim, n, m, blob, w.dt, torch.from_numpy(w.a_nodes).cuda(), opt)


@pytest.mark.parametrize("cap", CAPS, ids=[f"grid_{c}" for c in CAPS])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_cn_steps_with_capped_cg_grid_match_oracle(H, case, precision, cap, monkeypatch):
    import torch
    monkeypatch.setenv("HIFCN_CG_GRID", cap)  # read when the handle is created
    w, A, F, blob = _problem(case)
    ref, it_ref, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 3, w.leaf, w.eps, (1, 1.0, 1.0), tol=1e-10,
                                  factor=F)
    h = _import(H, case, precision)
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    its = []
    for _ in range(3):
        u, it = H.cn_step(h, u)
        its.append(it)
    assert rel_err(u.cpu().numpy(), ref.ravel()) <= 1e-9
    if precision == 0:
        assert all(abs(a - b) <= 1 for a, b in zip(its, it_ref)), (its, it_ref)
    h.close()


@pytest.mark.parametrize("cap", CAPS, ids=[f"grid_{c}" for c in CAPS])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_pcg_with_capped_cg_grid_matches_oracle(H, case, cap, monkeypatch):
    import torch
    monkeypatch.setenv("HIFCN_CG_GRID", cap)
    w, A, F, blob = _problem(case)
    h = _import(H, case, 0)
    b = np.random.default_rng(4).standard_normal(F.N)
    x, it, relres = H.pcg_solve(h, torch.from_numpy(b).cuda())
    xr, itr, rr, conv = pcg.pcg(A, b, lambda v: hif.apply_inverse(F, v), tol=1e-10)
    assert abs(it - itr) <= 1
    assert relres <= 1e-10 * 1.01
    assert rel_err(x.cpu().numpy(), xr) <= 1e-9
    h.close()
