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
* ``cn_solve_varying`` is the variant of Sec. 4 (Conclusions) for coefficients
  that change in time: step k uses a_k in A and in the right-hand side, and
  the factor is recomputed only every few steps, serving as the
  preconditioner in between.
"""

from __future__ import annotations

import numpy as np

from . import grid
from . import hif


def pcg(A, b: np.ndarray, precond, tol: float = 1e-10, maxit: int = 1000, x0=None):
    """Solve A x = b by PCG; returns (x, iters, relres_true, converged).

    x0 = None is the zero initial guess; a given x0 starts from it (warm start)."""
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = float(np.linalg.norm(b))
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64).ravel().copy()
    if nb == 0.0 and x0 is None:
        return x, 0, 0.0, True
    r = b - A @ x if x0 is not None else b.copy()
    if nb == 0.0 or float(np.linalg.norm(r)) <= tol * nb:
        return x, 0, (float(np.linalg.norm(r)) / nb if nb else 0.0), True
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
             skel_edges_3d: bool = True, theta: float = 0.5, warm_start: bool = False,
             direct: bool = False):
    """Algorithm 1: returns (u after ``steps`` steps, per-step iteration counts, factor).

    theta = 1/2 is Crank-Nicolson, theta = 1 backward Euler; warm_start starts
    PCG from u^k instead of 0; direct replaces PCG by u^{k+1} = F^{-1} g (the
    factor used as a solver, Sec. 3 Example 1), reporting 0 iterations."""
    dim = u0.ndim
    n = u0.shape[0] + 1
    A = grid.assemble_A(a_nodes, dt, theta)
    F = factor if factor is not None else hif.factor(A, n, dim, leaf, eps, skel_edges_3d)
    u = np.array(u0, dtype=np.float64)
    iters = []
    for _ in range(steps):
        r = grid.reaction(u, *reaction) if reaction[0] else None
        g = grid.cn_rhs(a_nodes, u, dt, r, theta)
        if direct:
            x, it = hif.apply_inverse(F, g.ravel()), 0
        else:
            x, it, _, _ = pcg(A, g.ravel(), lambda v: hif.apply_inverse(F, v), tol=tol,
                              x0=u.ravel() if warm_start else None)
        u = x.reshape(u.shape)
        iters.append(it)
    return u, iters, F


def cn_solve_varying(a_seq, u0: np.ndarray, dt: float, leaf: int, eps: float,
                     reaction=(0, 0.0, 0.0), tol: float = 1e-10, refactor_every: int = 1,
                     theta: float = 0.5, skel_edges_3d: bool = True):
    """Sec. 4: one step per coefficient field a_seq[k] (nodal arrays); the
    factor is that of the field at the last multiple of ``refactor_every``.
    Returns (u, per-step iteration counts)."""
    dim = u0.ndim
    n = u0.shape[0] + 1
    u = np.array(u0, dtype=np.float64)
    iters = []
    F = None
    for k, a in enumerate(a_seq):
        A = grid.assemble_A(a, dt, theta)
        if k % refactor_every == 0:
            F = hif.factor(A, n, dim, leaf, eps, skel_edges_3d)
        r = grid.reaction(u, *reaction) if reaction[0] else None
        g = grid.cn_rhs(a, u, dt, r, theta)
        x, it, _, _ = pcg(A, g.ravel(), lambda v: hif.apply_inverse(F, v), tol=tol)
        u = x.reshape(u.shape)
        iters.append(it)
    return u, iters
