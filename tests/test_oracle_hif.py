"""Pins of the oracle's HIF factorization, inverse apply, PCG and CN loop.

* eps = 0: every ID keeps all columns, so the factorization is an exact
  nested-dissection Cholesky; F^{-1} b must equal a dense Cholesky solve
  (library routine) to rounding, and PCG must converge in one iteration.
* eps > 0: F^{-1} is a congruence of A_L^{-1} (Eq. Ainv) hence symmetric and
  positive definite; ||I - A F^{-1}||_2 is O(eps) (the paper reports 7.9e-6
  at eps = 1e-6); a sign or index slip in any step breaks one of these.
* ID: exact on matrices of known low rank, and within eps of the input on
  matrices with decaying spectrum (Eq. 2_5).
* One level step by step at eps = 0: the Schur complement of the cell
  elimination, the identity diagonal blocks after block Jacobi and the root
  against dense linear algebra.
* PCG with the identity preconditioner reproduces scipy's CG iterates.
* CN: for a = 1 the oracle matches the exact DST-I mode evolution to the CG
  tolerance, with and without a linear reaction term.
"""

import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import workloads as W
from oracle import grid, hif, pcg

from test_oracle_stencil import _dst_closed_form


def _setup(dim, n, m, eps, seed=7, contrast=1e2, dt=1.0):
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=eps, seed=seed, contrast=contrast,
                            dt=dt, corr_len=0.2)
    A = grid.assemble_A(w.a_nodes, w.dt)
    F = hif.factor(A, n, dim, m, eps)
    return A, F


@pytest.mark.parametrize("dim,n,m", [(2, 32, 8), (2, 32, 4), (2, 16, 4), (3, 16, 4), (3, 8, 4)])
def test_eps0_is_exact_cholesky(dim, n, m):
    A, F = _setup(dim, n, m, 0.0)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(A.shape[0])
    y = hif.apply_inverse(F, b)
    yd = sla.cho_solve(sla.cho_factor(A.toarray()), b)
    assert np.linalg.norm(y - yd) <= 1e-12 * np.linalg.norm(yd)
    x, it, relres, conv = pcg.pcg(A, b, lambda v: hif.apply_inverse(F, v), tol=1e-10)
    assert conv and it == 1 and relres < 1e-12


@pytest.mark.parametrize("dim,n,m,eps", [(2, 32, 8, 1e-6), (2, 32, 4, 1e-3), (3, 16, 4, 1e-4)])
def test_inverse_symmetric_positive(dim, n, m, eps):
    A, F = _setup(dim, n, m, eps)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(A.shape[0])
    y = rng.standard_normal(A.shape[0])
    Fx = hif.apply_inverse(F, x)
    Fy = hif.apply_inverse(F, y)
    assert abs(x @ Fy - y @ Fx) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(Fy)
    for _ in range(5):
        z = rng.standard_normal(A.shape[0])
        assert z @ hif.apply_inverse(F, z) > 0.0


def _power_norm_I_minus_AFinv(A, F, iters=40, seed=0):
    """||I - A F^{-1}||_2 by power iteration on E^T E, E = I - A F^{-1}
    (randomized power iteration, as used by the paper for the same estimate)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(A.shape[0])
    v /= np.linalg.norm(v)

    def E(u):
        return u - A @ hif.apply_inverse(F, u)

    def Et(u):  # E^T = I - F^{-T} A = I - F^{-1} A (F^{-1} symmetric)
        return u - hif.apply_inverse(F, A @ u)

    s = 0.0
    for _ in range(iters):
        w = Et(E(v))
        s = math.sqrt(np.linalg.norm(w))
        v = w / np.linalg.norm(w)
    return s


def test_factor_accuracy_is_order_eps():
    A, F3 = _setup(2, 64, 8, 1e-3, contrast=1e3)
    F6 = hif.factor(A, 64, 2, 8, 1e-6)
    F9 = hif.factor(A, 64, 2, 8, 1e-9)
    e3 = _power_norm_I_minus_AFinv(A, F3)
    e6 = _power_norm_I_minus_AFinv(A, F6)
    e9 = _power_norm_I_minus_AFinv(A, F9)
    assert e3 < 0.5
    assert e6 < 1e-3
    assert e9 < 1e-6
    assert e9 < e6 < e3


def test_id_exact_on_low_rank_and_bounded_otherwise():
    rng = np.random.default_rng(11)
    # exact rank 5 in a 40 x 12 matrix: ID with tiny eps finds rank 5 and is exact
    X = rng.standard_normal((40, 5)) @ rng.standard_normal((5, 12))
    piv, k, T = hif.interpolative_decomposition(X, 1e-10)
    assert k == 5
    np.testing.assert_allclose(X[:, piv[k:]], X[:, piv[:k]] @ T, atol=1e-10 * np.abs(X).max())
    # decaying spectrum: error bounded by a modest multiple of eps ||X||
    U, _ = np.linalg.qr(rng.standard_normal((60, 20)))
    V, _ = np.linalg.qr(rng.standard_normal((20, 20)))
    Y = U @ np.diag(10.0 ** -np.arange(20, dtype=float) * 0.5) @ V.T
    for eps in (1e-2, 1e-4, 1e-6):
        piv, k, T = hif.interpolative_decomposition(Y, eps)
        err = np.linalg.norm(Y[:, piv[k:]] - Y[:, piv[:k]] @ T, 2)
        assert 0 < k < 20
        assert err <= 20.0 * eps * np.linalg.norm(Y, 2)
    # eps = 0 keeps every nonzero pivot
    piv, k, T = hif.interpolative_decomposition(rng.standard_normal((30, 10)), 0.0)
    assert k == 10


def test_skeleton_schur_block_push_through():
    """X = I - T (I + T^T T)^{-1} T^T equals (I + T T^T)^{-1} and is SPD."""
    A, F = _setup(2, 32, 4, 1e-3)
    seen = 0
    for lf in F.level_factors:
        for step in lf.skel_steps:
            for k in step:
                if k.T.size == 0:
                    continue
                S = k.Ls @ k.Ls.T
                np.testing.assert_allclose(S, np.eye(len(k.rd)) + k.T.T @ k.T, atol=1e-12)
                X = np.eye(len(k.sk)) - k.T @ np.linalg.solve(S, k.T.T)
                np.testing.assert_allclose(X, np.linalg.inv(np.eye(len(k.sk)) + k.T @ k.T.T),
                                           atol=1e-12)
                seen += 1
    assert seen > 0


def test_pcg_identity_matches_scipy_cg():
    A, _ = _setup(2, 16, 4, 0.0)
    b = np.random.default_rng(3).standard_normal(A.shape[0])
    for k in (1, 3, 7):
        x, it, _, _ = pcg.pcg(A, b, lambda v: v.copy(), tol=1e-300, maxit=k)
        xs, _ = spla.cg(A, b, x0=np.zeros_like(b), rtol=1e-300, atol=0.0, maxiter=k)
        assert it == k
        np.testing.assert_allclose(x, xs, rtol=1e-10, atol=1e-12 * np.abs(xs).max())


@pytest.mark.parametrize("c_lin", [0.0, 0.8])
def test_cn_matches_dst_closed_form(c_lin):
    """Config-1 shape (a = 1, sine modes + noise) at a reduced size n = 32."""
    n, m, dt, steps = 32, 8, 1e-2, 4
    w = W.config_heat2d_63()
    u0 = W.sine_modes_u0(n, 2, [(1, 1), (2, 3), (5, 2)], rng=np.random.default_rng(0), noise=0.1)
    ones = np.ones((n + 1, n + 1))
    react = (1, c_lin, math.inf) if c_lin else (0, 0.0, 0.0)
    u, iters, _ = pcg.cn_solve(ones, u0, dt, steps, m, 1e-6, react, tol=1e-12)
    exact = _dst_closed_form(u0, dt, steps, c_lin)
    assert np.linalg.norm(u - exact) <= 1e-9 * np.linalg.norm(exact)
    assert max(iters) <= 3
    del w


@pytest.mark.slow
def test_cn_config1_full_size_matches_closed_form():
    """Config 1 itself: 63^2, leaf 8, eps 1e-6, dt 1e-2, 10 steps, tol 1e-10."""
    w = W.config_heat2d_63()
    u, iters, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, w.steps, w.leaf, w.eps, w.reaction,
                               tol=w.tol)
    exact = _dst_closed_form(w.u0, w.dt, w.steps)
    assert np.linalg.norm(u - exact) <= 1e-9 * np.linalg.norm(exact)
    assert max(iters) <= 3


def _dst_be(u0, dt, steps):
    """Exact backward-Euler evolution for a = 1: each DST-I mode is scaled by
    1 / (1 - dt lam) per step."""
    import scipy.fft
    n = u0.shape[0] + 1
    h = 1.0 / n
    coef = scipy.fft.dstn(u0, type=1)
    ks = np.arange(1, n)
    lam = np.zeros(u0.shape)
    for ax in range(u0.ndim):
        s = [1] * u0.ndim
        s[ax] = n - 1
        lam = lam - (4.0 / h ** 2) * np.sin(ks * math.pi * h / 2).reshape(s) ** 2
    return scipy.fft.idstn(coef * (1.0 / (1.0 - dt * lam)) ** steps, type=1)


def test_backward_euler_matches_dst_closed_form():
    n, m, dt, steps = 32, 8, 1e-2, 3
    u0 = W.sine_modes_u0(n, 2, [(1, 1), (3, 2)], rng=np.random.default_rng(1), noise=0.05)
    ones = np.ones((n + 1, n + 1))
    u, iters, _ = pcg.cn_solve(ones, u0, dt, steps, m, 1e-6, tol=1e-12, theta=1.0)
    exact = _dst_be(u0, dt, steps)
    assert np.linalg.norm(u - exact) <= 1e-9 * np.linalg.norm(exact)


def test_warm_start_and_direct_variants():
    w = W.small_variable_2d(n=64, m=8, eps=1e-6, contrast=1e3, dt=0.5, corr_len=0.1)
    cold, it_c, F = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 3, w.leaf, w.eps, (1, 1.0, 1.0), tol=1e-11)
    warm, it_w, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 3, w.leaf, w.eps, (1, 1.0, 1.0), tol=1e-11,
                                 factor=F, warm_start=True)
    direct, it_d, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, 3, w.leaf, w.eps, (1, 1.0, 1.0),
                                   factor=F, direct=True)
    assert np.linalg.norm(warm - cold) <= 1e-9 * np.linalg.norm(cold)
    assert sum(it_w) <= sum(it_c)
    assert it_d == [0, 0, 0]
    # the direct solve is accurate to the factor's precision (O(eps))
    assert np.linalg.norm(direct - cold) <= 1e-3 * np.linalg.norm(cold)


def test_time_varying_coefficient_matches_mode_products():
    """a(x, t_k) = c_k (constant in space): M_k = c_k M_1, so each DST-I mode is
    multiplied per step by (1 + dt c_k lam / 2) / (1 - dt c_k lam / 2), even
    with the factor of an earlier c (refactored every 2 steps)."""
    import scipy.fft
    n, m, dt = 32, 8, 2e-2
    cs = [1.0, 1.3, 0.8, 1.6, 1.1]
    u0 = W.sine_modes_u0(n, 2, [(1, 1), (2, 3), (4, 1)], rng=np.random.default_rng(2), noise=0.05)
    a_seq = [c * np.ones((n + 1, n + 1)) for c in cs]
    u, iters = pcg.cn_solve_varying(a_seq, u0, dt, m, 1e-6, tol=1e-12, refactor_every=2)
    h = 1.0 / n
    ks = np.arange(1, n)
    lam1 = -(4.0 / h ** 2) * np.sin(ks * math.pi * h / 2) ** 2
    lam = lam1[:, None] + lam1[None, :]
    coef = scipy.fft.dstn(u0, type=1)
    for c in cs:
        coef = coef * (1 + dt * c * lam / 2) / (1 - dt * c * lam / 2)
    exact = scipy.fft.idstn(coef, type=1)
    assert np.linalg.norm(u - exact) <= 1e-9 * np.linalg.norm(exact)
    # a stale factor is a worse preconditioner for the steps that reuse it
    u1, it1 = pcg.cn_solve_varying(a_seq, u0, dt, m, 1e-6, tol=1e-12, refactor_every=1)
    assert np.linalg.norm(u1 - exact) <= 1e-9 * np.linalg.norm(exact)
    assert sum(iters) >= sum(it1)


@pytest.mark.parametrize("dim,n,m", [(2, 16, 8), (3, 8, 4)])
def test_one_level_steps_against_dense_algebra(dim, n, m):
    """One level (L = 1) at eps = 0, step by step against dense linear algebra.

    * Cell elimination (Eq. 2_3, the cells' updates adding up as in Eq. 3_1):
      the matrix left on the separators is the dense Schur complement
      S = A_RR - A_RI A_II^{-1} A_IR over all cell interiors at once.
    * Block Jacobi (Eq. jacobi-precond): with D = blockdiag(L_g^{-1}),
      D S D^T has identity diagonal blocks on every entity.
    * At eps = 0 no DOF is redundant, and the root factor reproduces D S D^T.
    """
    A, F = _setup(dim, n, m, 0.0)
    assert F.levels == 1
    lvl = F.level_factors[0]
    Ad = A.toarray()
    I = np.concatenate([c.I for c in lvl.cells])
    R = np.setdiff1d(np.arange(A.shape[0]), I)
    S = Ad[np.ix_(R, R)] - Ad[np.ix_(R, I)] @ np.linalg.solve(Ad[np.ix_(I, I)], Ad[np.ix_(I, R)])
    pos = {d: k for k, d in enumerate(R)}
    D = np.zeros_like(S)
    for j in lvl.jacobi:
        p = [pos[d] for d in j.I]
        D[np.ix_(p, p)] = np.linalg.inv(j.L)
    covered = sorted(pos[d] for j in lvl.jacobi for d in j.I)
    assert covered == list(range(len(R)))  # every separator DOF in exactly one entity
    Bm = D @ S @ D.T
    for j in lvl.jacobi:
        p = [pos[d] for d in j.I]
        assert np.allclose(Bm[np.ix_(p, p)], np.eye(len(p)), atol=1e-12)
    assert all(len(k.rd) == 0 for step in lvl.skel_steps for k in step)
    r = [pos[d] for d in F.root_idx]
    assert sorted(r) == list(range(len(R)))
    AL = F.root_L @ F.root_L.T
    assert np.allclose(AL, Bm[np.ix_(r, r)], rtol=0, atol=1e-10 * np.abs(Bm).max())
