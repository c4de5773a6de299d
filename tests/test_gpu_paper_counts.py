"""The GPU factor against the iteration counts printed in Sec. 3.

The FP64 path (GPU factorization, GPU PCG, tolerance 1e-12) runs the
paper's recipes at 63^2 and 15^3, heat and logistic, at eps = 1e-3 and 1e-6.
The same pin as the oracle's applies: the mean count lies within 1.5 of the
count printed for the smallest problem, and eps = 1e-6 takes fewer iterations.
"""

import numpy as np
import pytest

from test_oracle_paper_counts import STEPS, WINDOW, _printed_smallest, _workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    assert torch.cuda.is_available()
    return H


def _gpu_mean_iters(H, w):
    import torch
    a = torch.from_numpy(w.a_nodes).cuda()
    opt = H.default_options(eps=w.eps, precision=0, cg_tol=w.tol)
    h = H.hif_setup(w.dim, w.n, w.leaf, a, w.dt, opt)
    kind, k1, k2 = w.reaction
    if kind:
        H.hif_set_reaction(h, kind, k1, k2)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    its = []
    for _ in range(STEPS):
        u, it = H.cn_step(h, u)
        its.append(it)
    assert np.isfinite(u.cpu().numpy()).all()
    return float(np.mean(its))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("ex", ["heat", "logistic"])
def test_gpu_counts_match_printed(H, ex, dim):
    got = {}
    for eps in (1e-3, 1e-6):
        w = _workload(ex, dim, eps)
        got[eps] = _gpu_mean_iters(H, w)
        printed = _printed_smallest(ex, dim, eps)
        assert abs(got[eps] - printed) <= WINDOW, (ex, dim, eps, got[eps], printed)
    assert got[1e-6] < got[1e-3]


def _printed_at(ex, dim, eps, side):
    from test_oracle_paper_counts import _load
    rows = [r for r in _load() if r[:4] == (ex, dim, eps, side)]
    assert len(rows) == 1
    return rows[0][4]


TABLE_STEPS = 10


@pytest.mark.slow
@pytest.mark.parametrize("side", [1023, 2047, 4095])
@pytest.mark.parametrize("ex", ["heat", "logistic"])
def test_gpu_counts_at_table_sizes(H, ex, side):
    """The table sizes themselves (2D, leaf 16, FP64 factor and CG, tolerance
    1e-12, the paper's recipes): the mean count over the first 10 steps lies
    within 1.5 of the count printed for that size, eps = 1e-6 below 1e-3."""
    import workloads as W
    n = side + 1
    gen = W.paper_heat2d if ex == "heat" else W.paper_logistic2d
    got = {}
    for eps in (1e-3, 1e-6):
        w = gen(n, 16, eps, seed=0)
        w.steps = TABLE_STEPS
        got[eps] = _gpu_mean_iters_n(H, w, TABLE_STEPS)
        printed = _printed_at(ex, 2, eps, side)
        print(f"{ex} {side}^2 eps {eps:g}: GPU mean {got[eps]:.2f}, printed {printed}")
        assert abs(got[eps] - printed) <= WINDOW, (ex, side, eps, got[eps], printed)
    assert got[1e-6] < got[1e-3]


def _gpu_mean_iters_n(H, w, steps):
    import torch
    a = torch.from_numpy(w.a_nodes).cuda()
    opt = H.default_options(eps=w.eps, precision=0, cg_tol=w.tol)
    h = H.hif_setup(w.dim, w.n, w.leaf, a, w.dt, opt)
    kind, k1, k2 = w.reaction
    if kind:
        H.hif_set_reaction(h, kind, k1, k2)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    its = H.cn_steps(h, u, steps)
    assert np.isfinite(u.cpu().numpy()).all()
    h.close()
    return float(np.mean(its))


@pytest.mark.slow
@pytest.mark.parametrize("ex", ["heat", "logistic"])
def test_gpu_counts_at_table_sizes_3d(H, ex):
    """The 3D tables' middle size, 127^3 (leaf 8, FP64 factor and CG, tolerance
    1e-12, the paper's 3D recipes): the mean count over the first 10 steps lies
    within 1.5 of the count printed for 127^3, eps = 1e-6 below 1e-3."""
    import workloads as W
    got = {}
    for eps in (1e-3, 1e-6):
        w = W.paper_heat3d(128, 8, eps, seed=0, logistic=(ex == "logistic"))
        got[eps] = _gpu_mean_iters_n(H, w, TABLE_STEPS)
        printed = _printed_at(ex, 3, eps, 127)
        print(f"{ex} 127^3 eps {eps:g}: GPU mean {got[eps]:.2f}, printed {printed}")
        assert abs(got[eps] - printed) <= WINDOW, (ex, eps, got[eps], printed)
    assert got[1e-6] < got[1e-3]
