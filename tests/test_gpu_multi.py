"""hif_apply_multi: k right-hand sides at once, top levels on the tensor cores.

The levels stored in BF16 (HIF_FP32_BF16TOP) and the root are applied to all
k columns by tcgen05 matrix products (BF16 factor blocks; each FP32 column
split into a high and a low BF16 part, about 16 bits; FP32 accumulation).

Bars, from the arithmetic:
* against the FP64 oracle on identical (imported) factor data, every column
  within 3e-2, the bar of the single-column BF16 apply (each stored entry
  carries 8 significant bits, a few BF16 stages per level);
* against the library's single-column BF16 apply of the same handle, every
  column within 1e-3: the two differ only in the rounding of the vectors
  entering the top levels (2^-16 against FP32's 2^-24) and in the summation
  order, a few times 2^-16 after the handful of top-level stages;
* column independence: a column's result does not depend on the others
  (the same column alone and inside a batch of k agree to 1e-6).
"""

import numpy as np
import pytest

import workloads as W
from parity import rel_err
from oracle import export, grid, hif

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    assert torch.cuda.is_available()
    return H


CASES = [(2, 64, 8, 1e-6, 1.0), (2, 128, 8, 1e-6, 1.0), (3, 16, 4, 1e-4, 0.1), (3, 32, 8, 1e-4, 0.1)]
_cache = {}


def _problem(case):
    if case not in _cache:
        dim, n, m, eps, dt = case
        w = W.small_variable_2d(n=n, m=m, dim=dim, eps=eps, contrast=1e3, dt=dt, corr_len=0.1, seed=13)
        A = grid.assemble_A(w.a_nodes, w.dt)
        F = hif.factor(A, n, dim, m, eps)
        _cache[case] = (w, F, export.export_blob(F, w.dt))
    return _cache[case]


def _handle(H, case):
    import torch
    dim, n, m, eps, dt = case
    w, F, blob = _problem(case)
    top = max(1, len(F.level_factors) - 1)
    return H.hif_import_factor(dim, n, m, blob, w.dt, torch.from_numpy(w.a_nodes).cuda(),
                               H.default_options(eps=eps, precision=H.HIF_FP32_BF16TOP,
                                                 bf16_top_levels=top))


@pytest.mark.parametrize("k", [1, 5, 16, 33])
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d_n{c[1]}_m{c[2]}" for c in CASES])
def test_multi_apply_matches_oracle_and_single(H, case, k):
    import torch
    w, F, blob = _problem(case)
    h = _handle(H, case)
    rng = np.random.default_rng(100 + k)
    X = rng.standard_normal((k, w.N))
    Y = H.hif_apply_multi(h, torch.from_numpy(X).cuda()).cpu().numpy()
    for c in range(k):
        ref = hif.apply_inverse(F, X[c])
        single = H.hif_apply(h, torch.from_numpy(X[c].copy()).cuda(),
                             precision=H.HIF_FP32_BF16TOP).cpu().numpy()
        assert rel_err(Y[c], ref) <= 3e-2, (c, rel_err(Y[c], ref))
        assert rel_err(Y[c], single) <= 1e-3, (c, rel_err(Y[c], single))
    h.close()


def test_multi_columns_independent(H):
    import torch
    case = CASES[2]
    w, F, blob = _problem(case)
    h = _handle(H, case)
    rng = np.random.default_rng(7)
    X = torch.from_numpy(rng.standard_normal((12, w.N))).cuda()
    Y = H.hif_apply_multi(h, X).cpu().numpy()
    for c in (0, 5, 11):
        y1 = H.hif_apply_multi(h, X[c:c + 1].contiguous()).cpu().numpy()[0]
        assert rel_err(y1, Y[c]) <= 1e-6
    h.close()


def test_multi_apply_refusals(H):
    import torch
    case = CASES[0]
    dim, n, m, eps, dt = case
    w, F, blob = _problem(case)
    h32 = H.hif_import_factor(dim, n, m, blob, w.dt, torch.from_numpy(w.a_nodes).cuda(),
                              H.default_options(eps=eps, precision=H.HIF_FP32))
    X = torch.zeros((2, w.N), dtype=torch.float64, device="cuda")
    with pytest.raises(H.HifError) as e:
        H.hif_apply_multi(h32, X)
    assert e.value.status == H.HIF_EINVAL
    hb = _handle(H, case)
    X = torch.zeros((H.HIF_MULTI_MAX_COLS + 1, w.N), dtype=torch.float64, device="cuda")
    with pytest.raises(H.HifError):
        H.hif_apply_multi(hb, X)
    h32.close()
    hb.close()


@pytest.mark.parametrize("case", [CASES[1], CASES[3]], ids=["2d_n128_m8", "3d_n32_m8"])
def test_cn_step_multi_matches_oracle(H, case):
    """k states of one operator stepped together: each column equals the
    oracle's CN step from that state (1e-9 at CG tolerance 1e-10), and its PCG
    count is within 1 of the single-column step on the same handle."""
    import torch
    from oracle import pcg
    w, F, blob = _problem(case)
    h = _handle(H, case)
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    rng = np.random.default_rng(21)
    k = 6
    U = np.stack([(1.0 + 0.2 * c) * w.u0.ravel() + 0.05 * rng.standard_normal(w.N) for c in range(k)])
    U1, its = H.cn_step_multi(h, torch.from_numpy(U).cuda())
    U1 = U1.cpu().numpy()
    for c in range(k):
        ref, it_ref, _ = pcg.cn_solve(w.a_nodes, U[c].reshape(w.u0.shape), w.dt, 1, w.leaf, w.eps,
                                      (1, 1.0, 1.0), tol=1e-10, factor=F)
        assert rel_err(U1[c], ref.ravel()) <= 1e-9, (c, rel_err(U1[c], ref.ravel()))
        _, it1 = H.cn_step(h, torch.from_numpy(U[c].copy()).cuda())
        assert abs(its[c] - it1) <= 1, (c, its[c], it1)
        assert its[c] >= 1
    # in place (U1 = U) gives the same states
    Ut = torch.from_numpy(U).cuda()
    H.cn_step_multi(h, Ut, out=Ut)
    assert rel_err(Ut.cpu().numpy(), U1) <= 1e-12
    h.close()
