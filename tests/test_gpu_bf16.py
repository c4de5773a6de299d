"""HIF_FP32_BF16TOP: the top levels' factor blocks (and the root) stored in BF16.

Bars, from the arithmetic: a BF16 value carries 8 significant bits, so each
stored entry is rounded with relative error at most u = 2^-9; the apply of
F^{-1} passes through at most 4 BF16 stages per fused level (cells and
entities, forward and backward) plus 2 for the root, each adding at most a
few u of relative error for these well-scaled transforms.  On identical
factor data (imported from the oracle) the apply must stay within 3e-2 of the
FP64 oracle (and its error must exceed the FP32 apply's, showing the BF16
levels are in use); CN steps must still match the oracle to 1e-9, since CG in
FP64 corrects the preconditioner error (the extra iterations are reported,
not bounded by the paper).  Batched steps with mixed precisions equal single
steps to the CG tolerance and do not depend on the rest of the batch.
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


CASES = [(2, 64, 8, 1e-6, 1.0), (2, 128, 8, 1e-6, 1.0), (3, 16, 4, 1e-4, 0.1)]


@pytest.mark.parametrize("dim,n,m,eps,dt", CASES, ids=[f"{c[0]}d_n{c[1]}_m{c[2]}" for c in CASES])
def test_bf16_apply_on_imported_factor(H, dim, n, m, eps, dt):
    import torch
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=eps, contrast=1e3, dt=dt, corr_len=0.1, seed=13)
    A = grid.assemble_A(w.a_nodes, w.dt)
    F = hif.factor(A, n, dim, m, eps)
    blob = export.export_blob(F, w.dt)
    a = torch.from_numpy(w.a_nodes).cuda()
    L = len(F.level_factors)
    top = max(1, L - 1)
    hb = H.hif_import_factor(dim, n, m, blob, w.dt, a,
                             H.default_options(eps=eps, precision=H.HIF_FP32_BF16TOP, bf16_top_levels=top))
    hf = H.hif_import_factor(dim, n, m, blob, w.dt, a, H.default_options(eps=eps, precision=H.HIF_FP32))
    rng = np.random.default_rng(4)
    for _ in range(3):
        b = rng.standard_normal(w.N)
        ref = hif.apply_inverse(F, b)
        bt = torch.from_numpy(b).cuda()
        yb = H.hif_apply(hb, bt, precision=H.HIF_FP32_BF16TOP).cpu().numpy()
        yf = H.hif_apply(hf, bt, precision=H.HIF_FP32).cpu().numpy()
        eb, ef = _rel(yb, ref), _rel(yf, ref)
        print(f"apply error: bf16 top {eb:.2e}, fp32 {ef:.2e}")
        assert eb <= 3e-2
        assert ef <= 1e-5
        assert eb > ef  # the BF16 levels are in use
    assert H.hif_query(hb)["apply_bytes"] < H.hif_query(hf)["apply_bytes"]


@pytest.mark.parametrize("dim,n,m,eps,dt", CASES, ids=[f"{c[0]}d_n{c[1]}_m{c[2]}" for c in CASES])
def test_bf16_cn_steps_match_oracle(H, dim, n, m, eps, dt):
    import torch
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=eps, contrast=1e3, dt=dt, corr_len=0.1, seed=17)
    ref, it_ref, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 3, w.leaf, w.eps, (1, 1.0, 1.0), tol=1e-10)
    a = torch.from_numpy(w.a_nodes).cuda()
    h = H.hif_setup(dim, n, m, a, w.dt, H.default_options(eps=eps, precision=H.HIF_FP32_BF16TOP,
                                                          cg_tol=1e-10))
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    its = []
    for _ in range(3):
        u, it = H.cn_step(h, u)
        its.append(it)
    print(f"iterations: bf16 top {its}, oracle FP64 {it_ref}")
    assert _rel(u.cpu().numpy(), ref.ravel()) <= 1e-9
    assert all(i <= 50 for i in its)


def test_bf16_batched_equals_individual(H):
    import torch
    hs, us = [], []
    for i, prec in enumerate([H.HIF_FP32_BF16TOP, H.HIF_FP32, H.HIF_FP32_BF16TOP, H.HIF_FP64]):
        w = W.small_variable_2d(n=128, m=16, eps=1e-6, contrast=1e3, dt=0.5, corr_len=0.1, seed=60 + i)
        h = H.hif_setup(2, 128, 16, torch.from_numpy(w.a_nodes).cuda(), w.dt,
                        H.default_options(eps=1e-6, precision=prec))
        H.hif_set_reaction(h, 1, 1.0, 1.0)
        hs.append(h)
        us.append(torch.from_numpy(w.u0.ravel().copy()).cuda())
    ref = [H.cn_step(h, u) for h, u in zip(hs, us)]
    outs, its = H.cn_step_batched(hs, us)
    torch.cuda.synchronize()
    for (o_ref, i_ref), o, i, h, u in zip(ref, outs, its, hs, us):
        assert float(torch.linalg.norm(o - o_ref) / torch.linalg.norm(o_ref)) <= 1e-9
        alone, _ = H.cn_step_batched([h], [u])
        assert torch.equal(alone[0], o)
