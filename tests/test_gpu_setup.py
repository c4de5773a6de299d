"""GPU factorization (hif_setup) against the oracle and the mathematics.

* eps = 0: the GPU factor is an exact Cholesky of A, so F^{-1} b equals a
  dense Cholesky solve (library routine) to 1e-12 and PCG needs 1 iteration.
* eps > 0: the GPU and the oracle each factor A; several factors are valid
  (pivot near-ties), so what is compared is what is unique: the CN solution
  (1e-9 at tolerance 1e-10) and the iteration counts (+-1); F^{-1} must be
  symmetric positive definite and ||I - A F^{-1}|| = O(eps) like the oracle's.
* full size (2D 1023^2, the benchmark workload): every CN step satisfies
  A u^{k+1} = (I + dt/2 M) u^k + dt r(u^k) with A and M assembled by the
  oracle on the CPU, to the CG tolerance.
"""

import math

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from parity import rel_err
from oracle import grid, hif, pcg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_05566_gb300.hifcn as H
    assert torch.cuda.is_available()
    return H


def _setup(H, w, precision=0, skel_edges_3d=1):
    import torch
    a = torch.from_numpy(w.a_nodes).cuda()
    opt = H.default_options(eps=w.eps, precision=precision, cg_tol=1e-10,
                            skel_edges_3d=skel_edges_3d)
    return H.hif_setup(w.dim, w.n, w.leaf, a, w.dt, opt)


# normwise and element-by-element relative error (the larger of the two)
_rel = rel_err


EXACT = [(2, 32, 8), (2, 32, 4), (2, 16, 8), (3, 16, 4), (3, 8, 4), (3, 16, 8)]


@pytest.mark.parametrize("dim,n,m", EXACT, ids=[f"{d}d_n{n}_m{m}" for d, n, m in EXACT])
def test_eps0_setup_is_exact(H, dim, n, m):
    import torch
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=0.0, contrast=1e3, dt=0.7, corr_len=0.1)
    A = grid.assemble_A(w.a_nodes, w.dt)
    h = _setup(H, w)
    b = np.random.default_rng(0).standard_normal(w.N)
    y = H.hif_apply(h, torch.from_numpy(b).cuda()).cpu().numpy()
    yd = sla.cho_solve(sla.cho_factor(A.toarray()), b)
    assert _rel(y, yd) <= 1e-12
    x, it, rr = H.pcg_solve(h, torch.from_numpy(b).cuda())
    assert it == 1 and rr <= 1e-12


PARITY = [
    # dim, n, leaf, eps, contrast, dt
    (2, 64, 8, 1e-6, 1e2, 1.0),
    (2, 64, 8, 1e-3, 1e4, 1.0),
    (2, 128, 16, 1e-6, 1e4, 1.0),
    (2, 256, 16, 1e-6, 1e4, 1.0),
    (3, 16, 4, 1e-4, 1e3, 0.1),
    (3, 32, 8, 1e-4, 1e3, 0.1),
]
PIDS = [f"{d}d_n{n}_m{m}_eps{e:g}" for d, n, m, e, _, _ in PARITY]
_cache = {}


def _oracle(case):
    if case not in _cache:
        dim, n, m, eps, contrast, dt = case
        w = W.small_variable_2d(n=n, m=m, dim=dim, eps=eps, contrast=contrast, dt=dt,
                                corr_len=0.1, seed=5)
        A = grid.assemble_A(w.a_nodes, w.dt)
        F = hif.factor(A, n, dim, m, eps)
        _cache[case] = (w, A, F)
    return _cache[case]


@pytest.mark.parametrize("case", PARITY, ids=PIDS)
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_cn_steps_match_oracle(H, case, precision):
    import torch
    w, A, F = _oracle(case)
    h = _setup(H, w, precision)
    H.hif_set_reaction(h, 1, 1.0, 1.0)
    ref, iters, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 3, w.leaf, w.eps, (1, 1.0, 1.0),
                                 tol=1e-10, factor=F)
    u = torch.from_numpy(w.u0.ravel().copy()).cuda()
    its = []
    for _ in range(3):
        u, it = H.cn_step(h, u)
        its.append(it)
    assert _rel(u.cpu().numpy(), ref.ravel()) <= 1e-9
    if precision == 0:
        assert all(abs(a - b) <= 1 for a, b in zip(its, iters)), (its, iters)


@pytest.mark.parametrize("case", PARITY, ids=PIDS)
def test_gpu_factor_symmetric_positive(H, case):
    import torch
    w, A, F = _oracle(case)
    h = _setup(H, w)
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.standard_normal(w.N)).cuda()
    y = torch.from_numpy(rng.standard_normal(w.N)).cuda()
    Fx, Fy = H.hif_apply(h, x), H.hif_apply(h, y)
    lhs, rhs = float(x @ Fy), float(y @ Fx)
    assert abs(lhs - rhs) <= 1e-12 * float(x.norm() * Fy.norm())
    assert float(x @ Fx) > 0.0 and float(y @ Fy) > 0.0


def _gpu_err_norm(H, h, N, iters=30):
    """||I - A F^{-1}||_2 by power iteration on E^T E with E = I - A F^{-1}."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(0)
    v = torch.randn(N, generator=g, dtype=torch.float64).cuda()
    v /= v.norm()
    s = 0.0
    for _ in range(iters):
        Ev = v - H.hif_matvec(h, H.hif_apply(h, v))
        w = Ev - H.hif_apply(h, H.hif_matvec(h, Ev))
        s = math.sqrt(float(w.norm()))
        v = w / w.norm()
    return s


@pytest.mark.parametrize("case", PARITY[:4], ids=PIDS[:4])
def test_gpu_factor_accuracy_order_eps(H, case):
    w, A, F = _oracle(case)
    h = _setup(H, w)
    e = _gpu_err_norm(H, h, w.N)
    assert e < 1e3 * w.eps and e < 0.5


def test_skel_edges_off_3d(H):
    """3D with face-only skeletonization is still a valid preconditioner."""
    import torch
    w, A, F = _oracle(PARITY[4])
    h = _setup(H, w, skel_edges_3d=0)
    b = np.random.default_rng(2).standard_normal(w.N)
    x, it, rr = H.pcg_solve(h, torch.from_numpy(b).cuda())
    assert rr <= 1e-10 * 1.01 and it <= 6


@pytest.mark.slow
def test_full_size_fisher_1023_steps_satisfy_cn(H):
    """Benchmark workload (2D Fisher-KPP 1023^2, leaf 16, eps 1e-6, dt 1):
    each GPU step solves the CN system defined by the oracle's stencil."""
    import torch
    w = W.config_fisher2d_1023(eps=1e-6)
    A = grid.assemble_A(w.a_nodes, w.dt)
    for precision in (0, 1):
        h = _setup(H, w, precision)
        H.hif_set_reaction(h, 1, 1.0, 1.0)
        u = w.u0.copy()
        ut = torch.from_numpy(u.ravel().copy()).cuda()
        for _ in range(2):
            u1, it = H.cn_step(h, ut)
            g = grid.cn_rhs(w.a_nodes, u, w.dt, grid.reaction(u, 1, 1.0, 1.0)).ravel()
            un = u1.cpu().numpy()
            assert np.linalg.norm(A @ un - g) <= 1.05e-10 * np.linalg.norm(g)
            assert 1 <= it <= 10
            u = un.reshape(u.shape)
            ut = u1
        h.close()


_A3D = {}


@pytest.mark.slow
@pytest.mark.parametrize("precision", [1, 2], ids=["fp32", "fp32_bf16top"])
def test_full_size_heat3d_127_steps_satisfy_cn(H, precision):
    """3D heat 127^3 (leaf 8, eps 1e-4, dt 0.1, face + edge skeletonization),
    FP32 apply and FP32 with the top levels in BF16: each GPU step solves the
    CN system assembled by the oracle to the CG tolerance (GPU setup ~30 s)."""
    import torch
    w = W.config_heat3d_127()
    if "A" not in _A3D:
        _A3D["A"] = grid.assemble_A(w.a_nodes, w.dt)
    A = _A3D["A"]
    h = _setup(H, w, precision=precision)
    info = H.hif_query(h)
    assert info["levels"] == 4 and info["root_size"] > 0
    u = w.u0.copy()
    ut = torch.from_numpy(u.ravel().copy()).cuda()
    for _ in range(2):
        u1, it = H.cn_step(h, ut)
        g = grid.cn_rhs(w.a_nodes, u, w.dt, None).ravel()
        un = u1.cpu().numpy()
        assert np.linalg.norm(A @ un - g) <= 1.05e-10 * np.linalg.norm(g)
        assert 1 <= it <= 12
        u = un.reshape(u.shape)
        ut = u1
    h.close()
