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

The GPU takes beta in the flexible (Polak-Ribiere) form, with one more dot
product xi = q_old.z in the same reduction:
  beta = -alpha_old xi / rho_old,  sigma = mu + 2 beta xi + beta^2 sigma_old
which is (r - r_old).z / rho_old and p.Ap: with a fixed SPD preconditioner the
same iterates as the textbook loop, pinned below for both forms.  With an
inexact preconditioner (the FP32 apply) the flexible form loses fewer
iterations; the last test shows that with a preconditioner rounded to FP32.
"""

import numpy as np
import pytest

import workloads as W
from oracle import grid, hif, pcg


def cg_rearranged(A, b, precond, tol, maxit, flexible=True):
    """The GPU loop's recurrence, in FP64 NumPy (zero start); flexible=False
    is the textbook beta in the same arrangement."""
    nb = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    r = b.copy()
    p = q = None
    rho_old = alpha_old = sigma_old = None
    it = 0
    while it < maxit:
        z = precond(r)
        w = A @ z
        rho, mu = float(r @ z), float(w @ z)
        if it == 0:
            beta, sigma = 0.0, mu
            p, q = z.copy(), w.copy()
        else:
            if flexible:
                xi = float(q @ z)
                beta = -alpha_old * xi / rho_old
                sigma = mu + beta * (2.0 * xi + beta * sigma_old)
            else:
                beta = rho / rho_old
                sigma = mu - beta * rho / alpha_old
            p = z + beta * p
            q = w + beta * q
        alpha = rho / sigma
        x = x + alpha * p
        r = r - alpha * q
        rho_old, alpha_old, sigma_old = rho, alpha, sigma
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


@pytest.mark.parametrize("flexible", [True, False], ids=["flexible", "textbook_beta"])
@pytest.mark.parametrize("kind", ["hif", "jacobi"])
def test_same_iterates_every_iteration(system, kind, flexible):
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
        x, it = cg_rearranged(A, b, precond, tol=1e-30, maxit=k, flexible=flexible)
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



def test_flexible_beta_keeps_directions_conjugate_with_a_varying_preconditioner(system):
    """The flexible beta is -z.q_old / sigma_old, the value that makes each
    new direction A-conjugate to the previous one whatever z is.  With a
    preconditioner that changes at every call (F^{-1} times a random 1e-3
    relative perturbation, far larger than FP32 rounding), consecutive
    directions stay conjugate to rounding with the flexible form and lose
    conjugacy at the perturbation's size with the textbook beta."""
    A, F, b = system
    rng = np.random.default_rng(4)

    def varying(v):
        return hif.apply_inverse(F, v) * (1.0 + 1e-3 * rng.standard_normal(v.size))

    def worst_conjugacy(flexible):
        nb = float(np.linalg.norm(b))
        x = np.zeros_like(b)
        r = b.copy()
        p = q = None
        rho_old = alpha_old = sigma_old = None
        worst = 0.0
        for it in range(8):
            z = varying(r)
            w = A @ z
            rho, mu = float(r @ z), float(w @ z)
            if it == 0:
                beta, sigma = 0.0, mu
                p_new, q_new = z.copy(), w.copy()
            else:
                if flexible:
                    xi = float(q @ z)
                    beta = -alpha_old * xi / rho_old
                    sigma = mu + beta * (2.0 * xi + beta * sigma_old)
                else:
                    beta = rho / rho_old
                    sigma = mu - beta * rho / alpha_old
                p_new, q_new = z + beta * p, w + beta * q
                worst = max(worst, abs(float(p_new @ q)) /
                            np.sqrt(float(p_new @ (A @ p_new)) * float(p @ (A @ p))))
            p, q = p_new, q_new
            alpha = rho / sigma
            x = x + alpha * p
            r = r - alpha * q
            rho_old, alpha_old, sigma_old = rho, alpha, sigma
            if float(np.linalg.norm(r)) <= 1e-14 * nb:
                break
        return worst

    assert worst_conjugacy(True) <= 1e-10
    assert worst_conjugacy(False) >= 1e-6
