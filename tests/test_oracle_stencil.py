"""Pins of the oracle's grid, stencil and Crank-Nicolson right-hand side.

Pinned against facts the mathematics fixes, not against the oracle itself:
the discrete sine eigenpairs of the constant-coefficient Laplacian
(textbook), a brute-force node-by-node assembly, symmetry / definiteness of M
(Sec. 2), and the exact CN evolution of each sine mode (Eq. CN2).
"""

import math

import numpy as np
import pytest
import scipy.fft
import scipy.sparse.linalg as spla

import workloads as W
from oracle import grid


def _brute_force_M(a_nodes):
    """Node-by-node assembly written independently of the vectorized oracle."""
    dim = a_nodes.ndim
    n = a_nodes.shape[0] - 1
    h = 1.0 / n
    N = (n - 1) ** dim
    M = np.zeros((N, N))

    def a_at(j):  # j = (j_x, j_y[, j_z]) node coordinate
        return a_nodes[tuple(reversed(j))]

    def idx(j):
        return sum((j[ax] - 1) * (n - 1) ** ax for ax in range(dim))

    import itertools
    for j in itertools.product(range(1, n), repeat=dim):
        row = idx(j)
        for ax in range(dim):
            for s in (-1, 1):
                jn = list(j)
                jn[ax] += s
                w = 0.5 * (a_at(j) + a_at(tuple(jn)))
                M[row, row] -= w / h ** 2
                if 1 <= jn[ax] <= n - 1:
                    M[row, idx(tuple(jn))] += w / h ** 2
    return M


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_assembly_matches_brute_force(dim, n):
    rng = np.random.default_rng(3)
    a = np.exp(rng.standard_normal((n + 1,) * dim))
    M = grid.assemble_M(a).toarray()
    Mb = _brute_force_M(a)
    assert np.max(np.abs(M - Mb)) <= 1e-12 * np.max(np.abs(Mb))
    u = rng.standard_normal((n - 1,) * dim)
    Mu = grid.apply_M(a, u, 1.0 / n).ravel()
    np.testing.assert_allclose(Mu, Mb @ u.ravel(), rtol=1e-12, atol=1e-12 * np.abs(Mb).max())


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 8)])
def test_M_symmetric_negative_definite(dim, n):
    rng = np.random.default_rng(4)
    a = np.exp(2 * rng.standard_normal((n + 1,) * dim))
    M = grid.assemble_M(a)
    assert abs(M - M.T).max() == 0.0
    lam_max = spla.eigsh(M, k=1, which="LA", return_eigenvectors=False)[0]
    assert lam_max < 0.0
    A = grid.assemble_A(a, 0.3)
    lam_min = spla.eigsh(A, k=1, which="SA", return_eigenvectors=False)[0]
    assert lam_min > 1.0  # A = I - dt/2 M with M negative definite


@pytest.mark.parametrize("dim,n,mode", [(2, 16, (1, 1)), (2, 16, (3, 5)), (3, 8, (1, 2, 3))])
def test_sine_modes_are_eigenvectors(dim, n, mode):
    """Constant a = 1: prod sin(k pi x) has eigenvalue -(4/h^2) sum sin^2(k pi h / 2)."""
    h = 1.0 / n
    u = W.sine_modes_u0(n, dim, [mode])
    lam = -(4.0 / h ** 2) * sum(math.sin(k * math.pi * h / 2) ** 2 for k in mode)
    Mu = grid.apply_M(np.ones((n + 1,) * dim), u, h)
    np.testing.assert_allclose(Mu, lam * u, rtol=0, atol=1e-9 * abs(lam))


def _dst_closed_form(u0, dt, steps, c_lin=0.0):
    """Exact k-step CN evolution of u0 for a = 1 (each DST-I mode is scaled by
    (1 + dt lam/2 + dt c) / (1 - dt lam/2) per step; c = linear reaction rate)."""
    dim = u0.ndim
    n = u0.shape[0] + 1
    h = 1.0 / n
    coef = scipy.fft.dstn(u0, type=1)
    ks = np.arange(1, n)
    lam = np.zeros(u0.shape)
    for ax in range(dim):
        s = [1] * dim
        s[ax] = n - 1
        lam = lam - (4.0 / h ** 2) * np.sin(ks * math.pi * h / 2).reshape(s) ** 2
    g = (1.0 + 0.5 * dt * lam + dt * c_lin) / (1.0 - 0.5 * dt * lam)
    return scipy.fft.idstn(coef * g ** steps, type=1)


def test_dst_closed_form_is_a_cn_step():
    """The closed form itself: one step satisfies (I - dt/2 M) u1 = (I + dt/2 M) u0."""
    n, dt = 16, 0.05
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal((n - 1, n - 1))
    u1 = _dst_closed_form(u0, dt, 1)
    ones = np.ones((n + 1, n + 1))
    lhs = u1 - 0.5 * dt * grid.apply_M(ones, u1, 1.0 / n)
    rhs = grid.cn_rhs(ones, u0, dt, None)
    np.testing.assert_allclose(lhs, rhs, atol=1e-11 * np.abs(rhs).max())


def test_rhs_with_linear_reaction():
    """Reaction k1 u (1 - u/k2) with k2 = inf is linear; the RHS adds dt k1 u."""
    n, dt, c = 16, 0.1, 0.7
    u = np.random.default_rng(6).standard_normal((n - 1, n - 1))
    ones = np.ones((n + 1, n + 1))
    r = grid.reaction(u, 1, c, math.inf)
    g = grid.cn_rhs(ones, u, dt, r)
    np.testing.assert_allclose(g - grid.cn_rhs(ones, u, dt, None), dt * c * u, rtol=0,
                               atol=1e-14 * np.abs(g).max())


def test_workload_contrast_and_shapes():
    rng = np.random.default_rng(0)
    g = W.grf(rng, 32, 2, 0.05)
    a = W.lognormal_coefficient(g, 1e4)
    assert a.shape == (33, 33)
    assert abs(a.max() / a.min() - 1e4) < 1e-6 * 1e4
    assert abs(g.mean()) < 1e-12
    n, m, L = W.snap_side(300.0)
    assert n == (1 << L) * m and 8 <= m <= 16 and abs(n - 1 - 300) <= 0.125 * 300


def test_paper_recipes_match_the_printed_parameters():
    """Sec. 3 recipes: coefficient ranges, initial conditions and time steps."""
    import math
    w = W.paper_heat2d(64, 8, 1e-3)
    assert (w.a_nodes.min(), w.a_nodes.max()) == pytest.approx((0.1, 10.0), abs=1e-12)
    assert w.dt == 1.0 / 64 and w.tol == 1e-12 and w.reaction[0] == 0
    # the two Gaussians peak at (0.35, 0.35) and (0.65, 0.65): the maximum sits on the
    # diagonal next to one of them (interior node (i, j) is at y = (i+1)/64, x = (j+1)/64)
    i, j = divmod(int(np.argmax(w.u0)), 63)
    x, y = (j + 1) / 64, (i + 1) / 64
    assert x == y and min(abs(x - 0.35), abs(x - 0.65)) < 1.0 / 64
    w = W.paper_logistic2d(64, 8, 1e-6)
    assert w.reaction == (1, 1.0, 10.0) and w.dt == 1.0 / 64
    assert w.u0.max() <= 2.0 / (3.0 * math.sqrt(2 * math.pi * 0.05)) + 1e-12
    w = W.paper_heat3d(16, 4, 1e-3)
    assert (w.a_nodes.min(), w.a_nodes.max()) == pytest.approx((0.05, 20.0), abs=1e-12)
    assert w.dt == 0.1 / 16 and w.u0.max() <= 1.0
    w = W.paper_heat3d(16, 4, 1e-3, logistic=True)
    assert w.reaction == (1, 1.0, 10.0)
    assert w.u0.max() <= (2 * math.pi * math.sqrt(0.05)) ** -1.5 + 1e-12


def test_batched_recipe():
    ws = W.config_batched(count=12)
    seen = set()
    for w in ws:
        assert w.n == (1 << w.levels) * w.leaf and 8 <= w.leaf <= 16
        assert 63 * 0.85 <= w.n - 1 <= 511 * 1.15
        assert 1e-2 <= w.dt <= 1.0 and w.eps == 1e-6 and w.reaction == (1, 1.0, 1.0)
        assert abs(w.a_nodes.max() / w.a_nodes.min() - 1e3) < 1e-6 * 1e3
        seen.add(w.a_nodes.tobytes()[:4096])
    assert len(seen) == len(ws)  # every problem has its own field
