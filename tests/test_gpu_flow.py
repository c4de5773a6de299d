"""Parity of the dependency-driven upper sweep (HIFCN_FLOW=1) with the oracle.

With HIFCN_FLOW=1 the cell and entity steps of the upper levels and the root
(Eq. Ainv, levels above those applied by the bulk-copy kernels) run as one
persistent kernel whose work units wait only for the units they depend on.
It computes the same operator as the level-by-level launches, so the bars are
theirs: FP64 apply within 1e-12 of the oracle, FP32 within 1e-5, CN steps to
1e-9 at CG tolerance 1e-10, and repeated applies bitwise equal (the units'
arithmetic does not depend on which CTA runs them or when).
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


# normwise and element-by-element relative error (the larger of the two)
_rel = rel_err


CASES = [
    # dim, n, leaf, eps, contrast, dt
    (2, 64, 8, 1e-6, 1e2, 1.0),
    (2, 128, 16, 1e-6, 1e4, 1.0),
    (3, 16, 4, 1e-4, 1e3, 0.1),
    (3, 32, 8, 1e-4, 1e3, 0.1),
]
IDS = [f"{d}d_n{n}_m{m}_eps{e:g}" for d, n, m, e, _, _ in CASES]
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


def _flow_ran(H, h, x, precision):
    H.hif_stats_enable(h, 1)
    H.hif_apply(h, x, precision=precision)
    names = [r["name"] for r in H.hif_stats_read(h)]
    H.hif_stats_enable(h, 0)
    return any(n.startswith("upper_flow") for n in names)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_flow_apply_matches_oracle(H, case, precision, tol, monkeypatch):
    import torch
    monkeypatch.setenv("HIFCN_FLOW", "1")
    w, A, F, blob = _problem(case)
    h = _import(H, case, precision)
    rng = np.random.default_rng(5)
    xt = torch.from_numpy(rng.standard_normal(F.N)).cuda()
    assert _flow_ran(H, h, xt, precision)
    for _ in range(3):
        x = rng.standard_normal(F.N)
        y = H.hif_apply(h, torch.from_numpy(x).cuda(), precision=precision).cpu().numpy()
        assert _rel(y, hif.apply_inverse(F, x)) <= tol
    assert torch.equal(H.hif_apply(h, xt, precision=precision), H.hif_apply(h, xt, precision=precision))
    h.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_flow_cn_steps_match_oracle(H, precision, monkeypatch):
    import torch
    monkeypatch.setenv("HIFCN_FLOW", "1")
    case = CASES[1]
    w, A, F, blob = _problem(case)
    ref, it_ref, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 3, w.leaf, w.eps, (1, 1.0, 1.0), tol=1e-10,
                                  factor=F)
    h = _import(H, case, precision)
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    its = []
    for _ in range(3):  # graph-captured solves: the sweep replays inside the CG loop
        u, it = H.cn_step(h, u)
        its.append(it)
    assert _rel(u.cpu().numpy(), ref.ravel()) <= 1e-9
    assert all(abs(a - b) <= 1 for a, b in zip(its, it_ref)), (its, it_ref)
    h.close()
