"""cn_steps: K Crank-Nicolson steps queued without host synchronization.

cn_steps runs, step after step on the stream, the same kernels and captured
PCG solve as cn_step, so K steps of cn_steps equal K calls of cn_step bit for
bit, with the same iteration counts (FP64 and FP32 apply, cold and warm
start, theta = 1); against the oracle the K steps match its CN loop (Algorithm
1) to 1e-9.  nsteps = 0 leaves u alone; a step that cannot converge within
cg_maxit is reported as HIF_ENOCONV after u has been advanced, as cn_step
does; statistics mode (host-driven solves) gives the same result.
"""

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


def _handle(H, w, **kw):
    import torch
    opt = H.default_options(eps=w.eps, cg_tol=1e-10, **kw)
    h = H.hif_setup(w.dim, w.n, w.leaf, torch.from_numpy(w.a_nodes).cuda(), w.dt, opt)
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    return h


CFG = [dict(), dict(precision=1), dict(x0_mode=1), dict(precision=1, x0_mode=1), dict(theta=1.0)]


@pytest.mark.parametrize("kw", CFG, ids=["fp64", "fp32", "fp64_warm", "fp32_warm", "theta1"])
def test_steps_equal_single_steps(H, kw):
    import torch
    w = W.small_variable_2d(n=128, m=16, eps=1e-6, contrast=1e3, dt=1.0, corr_len=0.1, seed=31)
    h = _handle(H, w, **kw)
    u0 = torch.from_numpy(w.u0.ravel().copy()).cuda()
    u = u0.clone()
    its_single = []
    for _ in range(4):
        u, it = H.cn_step(h, u)
        its_single.append(it)
    v = u0.clone()
    its = H.cn_steps(h, v, 4)
    torch.cuda.synchronize()
    assert its == its_single
    assert torch.equal(v, u)
    h.close()


def test_steps_match_oracle_and_grow(H):
    import torch
    w = W.small_variable_2d(n=64, m=8, eps=1e-6, contrast=1e3, dt=0.5, corr_len=0.1, seed=32)
    ref, it_ref, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 5, w.leaf, w.eps, (1, 1.0, 1.0), tol=1e-10)
    h = _handle(H, w)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    its = H.cn_steps(h, u, 2) + H.cn_steps(h, u, 3)  # the record buffer grows between calls
    assert _rel(u.cpu().numpy(), ref.ravel()) <= 1e-9
    assert all(abs(a - b) <= 1 for a, b in zip(its, it_ref)), (its, it_ref)
    assert H.cn_steps(h, u, 0) == []
    h.close()


def test_steps_stats_mode_and_nonconvergence(H):
    import torch
    w = W.small_variable_2d(n=64, m=8, eps=1e-3, contrast=1e4, dt=1.0, corr_len=0.1, seed=33)
    h = _handle(H, w)
    u0 = torch.from_numpy(w.u0.ravel().copy()).cuda()
    a = u0.clone()
    its_graph = H.cn_steps(h, a, 3)
    H.hif_stats_enable(h, 1)
    b = u0.clone()
    its_host = H.cn_steps(h, b, 3)
    H.hif_stats_enable(h, 0)
    assert its_host == its_graph
    assert _rel(b.cpu().numpy(), a.cpu().numpy()) <= 1e-12
    h.close()
    # one CG iteration cannot reach 1e-14 with a loose factor: ENOCONV, u advanced
    opt = H.default_options(eps=1e-3, cg_tol=1e-14, cg_maxit=1)
    h = H.hif_setup(2, w.n, w.leaf, torch.from_numpy(w.a_nodes).cuda(), w.dt, opt)
    u = u0.clone()
    with pytest.raises(H.HifError) as e:
        H.cn_steps(h, u, 2)
    assert e.value.status == H.HIF_ENOCONV
    assert not torch.equal(u, u0)
    h.close()
