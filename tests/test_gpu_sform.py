"""Parity of the S-form cell kernels (bulk-copy staged, FP32) with the oracle.

The S-form cell steps (forward c_B = V x_I; backward x_I <- S x_I - V^T x_B
with S = A_II^{-1}, Sec. 3 cell elimination) run only where a level's cells
are single work items, which by default takes at least 4 x SMs cells, and
outside the fused upper-level sweep (levels of at most 1 MB).
HIFCN_ITEM_TARGET=1 keeps every cell whole and HIFCN_NO_FUSED=1 launches every
level on its own, so these tests reach the S-form kernels at sizes the oracle
factors in seconds; HIFCN_TMA_GRID caps their
persistent grid so that one CTA takes many cells in turn (both stage and
gather buffers, pairs of rows carried across chunks and cells).

Bars: the FP32 apply within 1e-5 of the oracle's FP64 apply (the bar of the
FP32 apply everywhere); CN steps at CG tolerance 1e-10 match the oracle to
1e-9 with the iteration counts of the FP64 apply (within 1); at the full
benchmark size (1023^2, 4096 leaf cells, default launch shape) the FP32 apply
stays within 1e-5 of the FP64 apply, whose parity with the oracle is pinned
at the small sizes, and the CN steps keep the FP64 iteration counts.
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
    (2, 64, 8, 1e-6, 1e2, 1.0),     # 49 interior DOFs per leaf cell (ragged last quad)
    (2, 128, 16, 1e-6, 1e4, 1.0),   # 225: rows past 32 quads, odd chunk ends
    (2, 128, 16, 1e-3, 1e4, 1.0),   # lower ranks: smaller upper-level cells
    (3, 16, 4, 1e-4, 1e3, 0.1),
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


@pytest.mark.parametrize("cap", ["0", "1", "5"], ids=["grid_full", "grid_1", "grid_5"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_sform_apply_matches_oracle(H, case, cap, monkeypatch):
    import torch
    monkeypatch.setenv("HIFCN_ITEM_TARGET", "1")
    monkeypatch.setenv("HIFCN_NO_FUSED", "1")
    monkeypatch.setenv("HIFCN_TMA_GRID", cap)
    w, A, F, blob = _problem(case)
    h = _import(H, case, H.HIF_FP32)
    assert H.hif_query(h)["sform_levels"] & 1, "the leaf level must run the S-form kernels"
    rng = np.random.default_rng(3)
    for _ in range(2):
        x = rng.standard_normal(F.N)
        y = H.hif_apply(h, torch.from_numpy(x).cuda(), precision=H.HIF_FP32).cpu().numpy()
        assert _rel(y, hif.apply_inverse(F, x)) <= 1e-5
    # the same launch shape gives the same bits
    xt = torch.from_numpy(rng.standard_normal(F.N)).cuda()
    assert torch.equal(H.hif_apply(h, xt, precision=H.HIF_FP32), H.hif_apply(h, xt, precision=H.HIF_FP32))
    h.close()


@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
def test_sform_cn_steps_match_oracle(H, case, monkeypatch):
    import torch
    monkeypatch.setenv("HIFCN_ITEM_TARGET", "1")
    monkeypatch.setenv("HIFCN_NO_FUSED", "1")
    monkeypatch.setenv("HIFCN_TMA_GRID", "7")
    w, A, F, blob = _problem(case)
    ref, it_ref, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 3, w.leaf, w.eps, (1, 1.0, 1.0), tol=1e-10,
                                  factor=F)
    h = _import(H, case, H.HIF_FP32)
    assert H.hif_query(h)["sform_levels"] & 1
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    its = []
    for _ in range(3):
        u, it = H.cn_step(h, u)
        its.append(it)
    assert _rel(u.cpu().numpy(), ref.ravel()) <= 1e-9
    assert all(abs(a - b) <= 1 for a, b in zip(its, it_ref)), (its, it_ref)
    h.close()


def test_sform_zero_input_gives_zero(H, monkeypatch):
    import torch
    monkeypatch.setenv("HIFCN_ITEM_TARGET", "1")
    monkeypatch.setenv("HIFCN_NO_FUSED", "1")
    w, A, F, blob = _problem(CASES[1])
    h = _import(H, CASES[1], H.HIF_FP32)
    z = torch.zeros(F.N, dtype=torch.float64).cuda()
    assert float(H.hif_apply(h, z, precision=H.HIF_FP32).abs().max()) == 0.0
    h.close()


@pytest.mark.slow
def test_sform_full_size_fisher_1023(H):
    """Default launch shape at the benchmark size: 4096 leaf cells on a
    persistent grid, several cells per CTA."""
    import torch
    w = W.config_fisher2d_1023(eps=1e-6)
    a = torch.from_numpy(w.a_nodes).cuda()
    h = H.hif_setup(w.dim, w.n, w.leaf, a, w.dt, H.default_options(eps=w.eps, precision=H.HIF_FP32,
                                                                  cg_tol=1e-10))
    assert H.hif_query(h)["sform_levels"] & 1
    rng = np.random.default_rng(8)
    for _ in range(2):
        x = torch.from_numpy(rng.standard_normal(w.N)).cuda()
        y64 = H.hif_apply(h, x, precision=H.HIF_FP64)
        y32 = H.hif_apply(h, x, precision=H.HIF_FP32)
        assert float(torch.linalg.norm(y32 - y64) / torch.linalg.norm(y64)) <= 1e-5
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    h64 = H.hif_setup(w.dim, w.n, w.leaf, a, w.dt, H.default_options(eps=w.eps, precision=H.HIF_FP64,
                                                                    cg_tol=1e-10))
    H.hif_set_reaction(h64, 1, 1.0, 1.0)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    u64 = u.clone()
    for _ in range(2):
        u, it = H.cn_step(h, u)
        u64, it64 = H.cn_step(h64, u64)
        assert abs(it - it64) <= 1, (it, it64)
    assert float(torch.linalg.norm(u - u64) / torch.linalg.norm(u64)) <= 1e-9
    h.close()
    h64.close()
