"""Preconditioned conjugate gradient and the Crank-Nicolson loop (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``pcg`` is the textbook Hestenes-Stiefel PCG that Algorithm 1 calls as
  pcg(A, g, F^{-1}): initial guess x0 = 0, stop as soon as the recurrence
  residual satisfies ||r||_2 <= tol ||b||_2 (the paper states a relative
  residual without the norm; the 2-norm relative to b is the reading), the
  iteration count is the number of x updates, the returned relres is the
  true residual ||b - A x|| / ||b|| at exit.
* ``cn_solve`` runs Algorithm 1: factor once, then per step the right-hand
  side (I + dt/2 M) u + dt r(u) (Eq. CN2) and one PCG solve with A = I - dt/2 M.
"""

from __future__ import annotations

import numpy as np

from . import grid
from . import hif


def pcg(A, b: np.ndarray, precond, tol: float = 1e-10, maxit: int = 1000):
    """Solve A x = b by PCG; returns (x, iters, relres_true, converged)."""
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    if nb == 0.0:
        return x, 0, 0.0, True
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    converged = False
    while it < maxit:
        q = A @ p
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        if float(np.linalg.norm(r)) <= tol * nb:
            converged = True
            break
        z = precond(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    relres = float(np.linalg.norm(b - A @ x)) / nb
    return x, it, relres, converged


def cn_solve(a_nodes: np.ndarray, u0: np.ndarray, dt: float, steps: int, leaf: int,
             eps: float, reaction=(0, 0.0, 0.0), tol: float = 1e-10, factor=None,
             skel_edges_3d: bool = True):
    """Algorithm 1: returns (u after ``steps`` CN steps, per-step iteration counts, factor)."""
    dim = u0.ndim
    n = u0.shape[0] + 1
    A = grid.assemble_A(a_nodes, dt)
    F = factor if factor is not None else hif.factor(A, n, dim, leaf, eps, skel_edges_3d)
    u = np.array(u0, dtype=np.float64)
    iters = []
    for _ in range(steps):
        r = grid.reaction(u, *reaction) if reaction[0] else None
        g = grid.cn_rhs(a_nodes, u, dt, r)
        x, it, _, _ = pcg(A, g.ravel(), lambda v: hif.apply_inverse(F, v), tol=tol)
        u = x.reshape(u.shape)
        iters.append(it)
    return u, iters, F
