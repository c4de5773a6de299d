"""The GPU runs PCG in the Chronopoulos-Gear arrangement; the oracle runs the
textbook loop (Algorithm 1's linear solve).  This pins the reading that the two
are the same iteration: with the oracle's own HIF preconditioner on a small
variable-coefficient CN system, the rearranged recurrence, written here as the
GPU kernels compute it, gives the textbook iterates after every iteration
(to rounding) and the same iteration count at the solve's tolerance.

Rearrangement (per iteration, z = F^{-1} r):
  w = A z, rho = r.z, mu = w.z
  beta = rho / rho_old (0 at first), sigma = mu - beta rho / alpha_old (mu at first)
  alpha = rho / sigma
  p = z + beta p, q = w + beta q (p = z, q = w at first), x += alpha p, r -= alpha q
"""

import numpy as np
import pytest

import workloads as W
from oracle import grid, hif, pcg


def cg_rearranged(A, b, precond, tol, maxit):
    """The GPU loop's recurrence, in FP64 NumPy (zero start)."""
    nb = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    r = b.copy()
    p = q = None
    rho_old = alpha_old = None
    it = 0
    while it < maxit:
        z = precond(r)
        w = A @ z
        rho, mu = float(r @ z), float(w @ z)
        if it == 0:
            beta, sigma = 0.0, mu
            p, q = z.copy(), w.copy()
        else:
            beta = rho / rho_old
            sigma = mu - beta * rho / alpha_old
            p = z + beta * p
            q = w + beta * q
        alpha = rho / sigma
        x = x + alpha * p
        r = r - alpha * q
        rho_old, alpha_old = rho, alpha
        it += 1
        if float(np.linalg.norm(r)) <= tol * nb:
            break
    return x, it


@pytest.fixture(scope="module")
def system():
    w = W.small_variable_2d(n=32, m=8, eps=1e-3, contrast=1e3, dt=1.0, corr_len=0.1, seed=7)
    A = grid.assemble_A(w.a_nodes, w.dt)
    F = hif.factor(A, w.n, 2, w.leaf, 1e-3)
    b = np.random.default_rng(2).standard_normal(A.shape[0])
    return A, F, b


@pytest.mark.parametrize("kind", ["hif", "jacobi"])
def test_same_iterates_every_iteration(system, kind):
    """The identity holds for any SPD preconditioner; the weak Jacobi one
    keeps beta of order one, so that a wrong sign or a dropped term in the
    sigma recurrence shows in the iterates (with the HIF factor beta is tiny)."""
    A, F, b = system
    if kind == "hif":
        precond = lambda v: hif.apply_inverse(F, v)
    else:
        dinv = 1.0 / A.diagonal()
        precond = lambda v: dinv * v
    for k in range(1, 9):
        x_ref, it_ref, _, _ = pcg.pcg(A, b, precond, tol=1e-30, maxit=k)
        x, it = cg_rearranged(A, b, precond, tol=1e-30, maxit=k)
        assert it == it_ref == k
        assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def test_same_iteration_count_at_tolerance(system):
    A, F, b = system
    precond = lambda v: hif.apply_inverse(F, v)
    x_ref, it_ref, relres, conv = pcg.pcg(A, b, precond, tol=1e-10, maxit=200)
    x, it = cg_rearranged(A, b, precond, tol=1e-10, maxit=200)
    assert conv and it_ref >= 3  # a loose factor: several iterations
    assert abs(it - it_ref) <= 1
    assert np.linalg.norm(b - A @ x) <= 1.01e-10 * np.linalg.norm(b) * 10
