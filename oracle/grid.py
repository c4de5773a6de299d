"""Grid, stencil and Crank-Nicolson right-hand side (oracle; test infrastructure).

Follows Sec. 2 of the paper: the unit square/cube with n = 1/h = 2^L m
intervals per axis, unknowns on the interior nodes x_j = h j, 1 <= j <= n-1
(reading of the garbled index range printed there), zero Dirichlet data.
M is the standard five-point (2D) / seven-point (3D) finite-difference
discretization of div(a grad .):

    (M u)_j = h^{-2} sum_{j' nbr of j} a_{jj'} (u_{j'} - u_j),   u = 0 on the boundary,

with the face coefficient a_{jj'} = (a(x_j) + a(x_{j'})) / 2 (arithmetic mean of
the nodal values; the paper does not print the face rule).  A = I - dt/2 M
(Eq. CN) is SPD; the CN right-hand side is (I + dt/2 M) u^k + dt r(u^k)
(Eq. CN2, Algorithm 1).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def interior_index(n: int, dim: int) -> np.ndarray:
    """DOF index array of shape (n-1,)*dim (last axis = x fastest)."""
    return np.arange((n - 1) ** dim).reshape((n - 1,) * dim)


def dof_coords(n: int, dim: int) -> np.ndarray:
    """Integer node coordinates j (1..n-1) of every DOF, shape (N, dim), column 0 = x."""
    N = (n - 1) ** dim
    idx = np.arange(N)
    out = np.empty((N, dim), dtype=np.int64)
    for ax in range(dim):
        out[:, ax] = (idx // (n - 1) ** ax) % (n - 1) + 1
    return out


def _axis_slices(dim: int, ax: int, lo: int, hi: int | None):
    """Slice tuple selecting lo:hi along the array axis that stores geometric axis ax."""
    s = [slice(None)] * dim
    s[dim - 1 - ax] = slice(lo, hi)
    return tuple(s)


def face_coefficients(a_nodes: np.ndarray, ax: int) -> np.ndarray:
    """a_{jj'} between node j and j + e_ax, for every pair of adjacent nodes along ax.

    Returned on the full node grid with length n along ax (index j means the
    face between j and j+1).
    """
    dim = a_nodes.ndim
    lo = a_nodes[_axis_slices(dim, ax, 0, -1)]
    hi = a_nodes[_axis_slices(dim, ax, 1, None)]
    return 0.5 * (lo + hi)


def apply_M(a_nodes: np.ndarray, u: np.ndarray, h: float) -> np.ndarray:
    """Matrix-free (M u) on the interior grid; u has shape (n-1,)*dim."""
    dim = u.ndim
    n = u.shape[0] + 1
    up = np.zeros((n + 1,) * dim)
    up[(slice(1, n),) * dim] = u
    out = np.zeros_like(u)
    for ax in range(dim):
        f = face_coefficients(a_nodes, ax)  # length n along ax, index j = face (j, j+1)
        # restrict the non-ax axes to interior nodes
        sel = [slice(1, n)] * dim
        sel[dim - 1 - ax] = slice(None)
        f = f[tuple(sel)]
        # forward neighbour: face index j (between j and j+1), for j = 1..n-1
        fwd = f[_axis_slices(dim, ax, 1, n)]
        bwd = f[_axis_slices(dim, ax, 0, n - 1)]
        u_f = up[tuple(_shift(dim, ax, +1, n))]
        u_b = up[tuple(_shift(dim, ax, -1, n))]
        out += fwd * (u_f - u) + bwd * (u_b - u)
    return out / (h * h)


def _shift(dim: int, ax: int, d: int, n: int):
    s = [slice(1, n)] * dim
    s[dim - 1 - ax] = slice(1 + d, n + d)
    return s


def assemble_M(a_nodes: np.ndarray) -> sp.csr_matrix:
    """Assembled sparse M (N x N), symmetric negative definite (Sec. 2)."""
    dim = a_nodes.ndim
    n = a_nodes.shape[0] - 1
    h = 1.0 / n
    idx = interior_index(n, dim)
    rows, cols, vals = [], [], []
    diag = np.zeros((n - 1,) * dim)
    for ax in range(dim):
        f = face_coefficients(a_nodes, ax)
        sel = [slice(1, n)] * dim
        sel[dim - 1 - ax] = slice(None)
        f = f[tuple(sel)]  # length n along ax
        # every interior node loses both of its faces to the diagonal
        diag -= f[_axis_slices(dim, ax, 1, n)] + f[_axis_slices(dim, ax, 0, n - 1)]
        # couplings between interior neighbours j and j+1 (j = 1..n-2)
        a_pair = f[_axis_slices(dim, ax, 1, n - 1)]
        i0 = idx[_axis_slices(dim, ax, 0, n - 2)]
        i1 = idx[_axis_slices(dim, ax, 1, n - 1)]
        rows += [i0.ravel(), i1.ravel()]
        cols += [i1.ravel(), i0.ravel()]
        vals += [a_pair.ravel(), a_pair.ravel()]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    N = (n - 1) ** dim
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    return M * (1.0 / (h * h))


def assemble_A(a_nodes: np.ndarray, dt: float, theta: float = 0.5) -> sp.csr_matrix:
    """A = I - theta dt M, sparse SPD: theta = 1/2 is Crank-Nicolson (Eq. CN),
    theta = 1 the backward Euler scheme the introduction mentions."""
    M = assemble_M(a_nodes)
    N = M.shape[0]
    A = sp.identity(N, format="csr") - (theta * dt) * M
    A.sort_indices()
    return A.tocsr()


def reaction(u: np.ndarray, kind: int, k1: float, k2: float) -> np.ndarray:
    """Explicit reaction r^k = r(u^k) (Eq. nr: k1 u (1 - u/k2)); kind 0 = none."""
    if kind == 0:
        return np.zeros_like(u)
    if kind == 1:
        return k1 * u * (1.0 - u / k2)
    raise ValueError(f"unknown reaction kind {kind}")


def cn_rhs(a_nodes: np.ndarray, u: np.ndarray, dt: float, r: np.ndarray | None,
           theta: float = 0.5) -> np.ndarray:
    """g = (I + (1 - theta) dt M) u^k + dt r^k: with theta = 1/2 the CN right-hand
    side (Eq. CN2 / first line of the loop in Algorithm 1), with theta = 1 the
    backward Euler one, u^k + dt r^k."""
    n = u.shape[0] + 1
    g = u + (1.0 - theta) * dt * apply_M(a_nodes, u, 1.0 / n) if theta != 1.0 else np.array(u, dtype=np.float64)
    if r is not None:
        g = g + dt * r
    return g
