"""Recursively preconditioned hierarchical interpolative factorization (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 2.2 of the paper step by step on a global sparse matrix that is
updated level by level:

* quadtree / octree: at level l the cells are (m 2^l)^d boxes of grid
  intervals; a node lies on a level-l separator along an axis when its
  coordinate is a multiple of s_l = m 2^l.  The *entity* of an active DOF at
  level l is its position on the doubled grid, code_axis = 2 (j // s_l) +
  [j mod s_l != 0]: odd on every axis = cell interior, one even axis = edge
  (2D) / face (3D), two even = corner (2D) / edge (3D), three = corner (3D).
* (1) cell elimination (Eqs. matrix-3blocks, 2_3, 3_1) for every cell
  (reading of the printed range "1<i<p_l" as all cells),
* (2) block Jacobi rescaling of every edge and corner - in 3D every face,
  edge and corner - (Eqs. jacobi-precond, 3_2),
* (3) skeletonization by interpolative decomposition of every edge (2D) /
  face (3D, then optionally every edge) (Eqs. 2_4, 2_5, T, 2_9, 3_3).
  All IDs of one sub-step are computed from the matrix as it stood before the
  sub-step (level-simultaneous reading; the paper does not fix an order).
  The ID uses column-pivoted QR (greedy largest remaining column, ties to the
  lowest index, a library routine) and keeps the leading pivots while
  |R_ii| > eps |R_00|,
* root: dense Cholesky of the remaining active block (Eq. 3_4),
* apply: F^{-1} = R_0 ... R_{L-1} A_L^{-1} R_{L-1}^T ... R_0^T with
  R_l = E_l C_l K_l (Eqs. A, Ainv), written with triangular solves exactly
  as the blocks of E, C, Z and the second E are printed.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .grid import dof_coords


# --------------------------------------------------------------------------- data


@dataclass
class CellFactor:
    """E_{I} of one cell (Eq. 2_3): L = chol(A_II), and the coupling A_BI."""

    I: np.ndarray
    B: np.ndarray
    L: np.ndarray
    A_BI: np.ndarray


@dataclass
class JacobiFactor:
    """C_{I} of one edge/face/corner (Eq. jacobi-precond): L = chol(A_II)."""

    I: np.ndarray
    L: np.ndarray


@dataclass
class SkelFactor:
    """Z_I and the elimination of the redundant DOFs (Eqs. T, 2_9).

    ``I`` are all DOFs of the entity (ascending global index); ``sk`` / ``rd``
    the skeleton / redundant DOFs in pivot order; ``T`` is k x (|I|-k) with
    A_{R,rd} ~ A_{R,sk} T; ``Ls`` = chol(I + T^T T) (the printed subscript of
    this factor is read as the redundant set, whose size it has).
    """

    I: np.ndarray
    sk: np.ndarray
    rd: np.ndarray
    T: np.ndarray
    Ls: np.ndarray


@dataclass
class LevelFactor:
    cells: list = field(default_factory=list)
    jacobi: list = field(default_factory=list)
    skel_steps: list = field(default_factory=list)  # list of lists of SkelFactor


@dataclass
class HIFFactor:
    dim: int
    n: int
    leaf: int
    levels: int
    eps: float
    level_factors: list
    root_idx: np.ndarray
    root_L: np.ndarray
    stats: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return (self.n - 1) ** self.dim


# ----------------------------------------------------------------------- geometry


def entity_codes(coords: np.ndarray, s: int) -> np.ndarray:
    """Doubled-grid entity code of each node at separator spacing s (see module doc)."""
    return 2 * (coords // s) + (coords % s != 0)


def group_by_entity(dofs: np.ndarray, codes: np.ndarray) -> list[tuple[tuple, np.ndarray]]:
    """Partition ``dofs`` by entity code; groups ordered by code, DOFs ascending."""
    if len(dofs) == 0:
        return []
    order = np.lexsort(tuple(codes[:, ax] for ax in range(codes.shape[1])) + ())
    # lexsort sorts by the last key first; the keys above make the sort
    # primary on the highest axis.  Within a group keep ascending DOF order.
    codes_s = codes[order]
    dofs_s = dofs[order]
    change = np.any(codes_s[1:] != codes_s[:-1], axis=1)
    starts = np.concatenate([[0], np.nonzero(change)[0] + 1, [len(dofs_s)]])
    out = []
    for a, b in zip(starts[:-1], starts[1:]):
        g = np.sort(dofs_s[a:b])
        out.append((tuple(int(c) for c in codes_s[a]), g))
    return out


def codim_of(code: tuple) -> int:
    return sum(1 for c in code if c % 2 == 0)


# ------------------------------------------------------------------------ helpers


def _dense(A: sp.csr_matrix, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    return A[rows][:, cols].toarray()


def _nonzero_cols(A: sp.csr_matrix, rows: np.ndarray) -> np.ndarray:
    sub = A[rows]
    return np.unique(sub.indices)


def _chol(M: np.ndarray) -> np.ndarray:
    return sla.cholesky(M, lower=True)


def _restrict(A: sp.spmatrix, keep: np.ndarray) -> sp.csr_matrix:
    """Zero every row and column of A whose index is not flagged in ``keep``."""
    P = sp.diags(keep.astype(np.float64))
    out = (P @ A @ P).tocsr()
    out.eliminate_zeros()
    return out


def id_rank(diag_abs: np.ndarray, eps: float) -> int:
    """Rank of the ID: leading pivots with |R_ii| > eps |R_00| (reading of Eq. 2_5)."""
    if len(diag_abs) == 0 or diag_abs[0] == 0.0:
        return 0
    thr = eps * diag_abs[0]
    k = 0
    while k < len(diag_abs) and diag_abs[k] > thr:
        k += 1
    return k


def interpolative_decomposition(Arg: np.ndarray, eps: float):
    """ID of the columns of Arg (|R| x |I|): returns (piv, k, T).

    Arg[:, piv[k:]] ~ Arg[:, piv[:k]] @ T with relative precision eps
    (Eq. 2_5), from column-pivoted QR Arg[:, piv] = Q R.
    """
    nI = Arg.shape[1]
    if Arg.shape[0] == 0 or nI == 0:
        return np.arange(nI), 0, np.zeros((0, nI))
    R, piv = sla.qr(Arg, mode="r", pivoting=True)
    ncols = min(R.shape[0], nI)
    d = np.abs(np.diag(R[:ncols, :ncols]))
    k = id_rank(d, eps)
    if k == 0:
        return piv, 0, np.zeros((0, nI))
    T = sla.solve_triangular(R[:k, :k], R[:k, k:], lower=False)
    return piv, k, T


# ------------------------------------------------------------------------- factor


def factor(A: sp.csr_matrix, n: int, dim: int, leaf: int, eps: float,
           skel_edges_3d: bool = True) -> HIFFactor:
    """Build the PHIF of the sparse SPD matrix A on the (n-1)^dim grid (Sec. 2.2)."""
    L = 0
    while leaf * (1 << L) < n:
        L += 1
    if leaf * (1 << L) != n or L < 1:
        raise ValueError("n must be leaf * 2^L with L >= 1")
    N = (n - 1) ** dim
    coords = dof_coords(n, dim)
    A = sp.csr_matrix(A, dtype=np.float64)
    A.sort_indices()
    active = np.ones(N, dtype=bool)
    levels = []
    stats = {"ranks": []}

    for lvl in range(L):
        s = leaf << lvl
        lf = LevelFactor()
        act = np.nonzero(active)[0]
        codes = entity_codes(coords[act], s)
        groups = group_by_entity(act, codes)

        # (1) cell elimination, Eq. 2_3: every cell, interiors are disjoint and
        # mutually uncoupled, their Schur updates add (Eq. 3_1).
        rows_u, cols_u, vals_u = [], [], []
        eliminated = np.zeros(N, dtype=bool)
        for code, I in groups:
            if codim_of(code) != 0:
                continue
            cols = _nonzero_cols(A, I)
            B = np.setdiff1d(cols, I, assume_unique=True)
            A_II = _dense(A, I, I)
            A_BI = _dense(A, B, I)
            Lc = _chol(A_II)
            # X_BB = A_BB - A_BI A_II^{-1} A_BI^T
            W = sla.solve_triangular(Lc, A_BI.T, lower=True)  # L^{-1} A_IB
            U = W.T @ W
            rr, cc = np.meshgrid(B, B, indexing="ij")
            rows_u.append(rr.ravel())
            cols_u.append(cc.ravel())
            vals_u.append(-U.ravel())
            lf.cells.append(CellFactor(I, B, Lc, A_BI))
            eliminated[I] = True
        active &= ~eliminated
        A = _restrict(A, active)
        if rows_u:
            upd = sp.coo_matrix((np.concatenate(vals_u),
                                 (np.concatenate(rows_u), np.concatenate(cols_u))),
                                shape=(N, N)).tocsr()
            A = (A + upd).tocsr()
        A.sort_indices()

        # (2) block Jacobi, Eqs. jacobi-precond / 3_2, on every remaining entity.
        act = np.nonzero(active)[0]
        groups = group_by_entity(act, entity_codes(coords[act], s))
        d_rows, d_cols, d_vals = [], [], []
        for code, I in groups:
            Lg = _chol(_dense(A, I, I))
            lf.jacobi.append(JacobiFactor(I, Lg))
            Linv = sla.solve_triangular(Lg, np.eye(len(I)), lower=True)
            rr, cc = np.meshgrid(I, I, indexing="ij")
            d_rows.append(rr.ravel())
            d_cols.append(cc.ravel())
            d_vals.append(Linv.ravel())
        inactive = np.nonzero(~active)[0]
        Dinv = sp.coo_matrix((np.concatenate(d_vals + [np.ones(len(inactive))]),
                              (np.concatenate(d_rows + [inactive]),
                               np.concatenate(d_cols + [inactive]))), shape=(N, N)).tocsr()
        A = (Dinv @ A @ Dinv.T).tocsr()
        # the diagonal blocks are now the identity (exactly, by definition)
        A = _replace_diag_blocks(A, [I for _, I in groups], [np.eye(len(I)) for _, I in groups], N)

        # (3) skeletonization, Eqs. 2_4 - 3_3: edges (2D) / faces then edges (3D).
        codims = [1] if dim == 2 else ([1, 2] if skel_edges_3d else [1])
        for cd in codims:
            act = np.nonzero(active)[0]
            groups = [(c, I) for c, I in group_by_entity(act, entity_codes(coords[act], s))
                      if codim_of(c) == cd]
            step = []
            rd_all = []
            blocks_idx, blocks_val = [], []
            for code, I in groups:
                cols = _nonzero_cols(A, I)
                R = np.setdiff1d(cols, I, assume_unique=True)
                Arg = _dense(A, R, I)  # A~_{R,I}
                piv, k, T = interpolative_decomposition(Arg, eps)
                sk, rd = I[piv[:k]], I[piv[k:]]
                S = np.eye(len(rd)) + T.T @ T
                Ls = _chol(S)
                X = np.eye(k) - T @ sla.cho_solve((Ls, True), T.T)
                step.append(SkelFactor(I, sk, rd, T, Ls))
                rd_all.append(rd)
                blocks_idx.append(sk)
                blocks_val.append(X)
                stats["ranks"].append((lvl, cd, len(I), k))
            lf.skel_steps.append(step)
            if rd_all:
                rd_all = np.concatenate(rd_all)
                active[rd_all] = False
            A = _restrict(A, active)
            A = _replace_diag_blocks(A, blocks_idx, blocks_val, N)
        levels.append(lf)

    root_idx = np.nonzero(active)[0]
    A_L = _dense(A, root_idx, root_idx)
    root_L = _chol(A_L) if len(root_idx) else np.zeros((0, 0))
    stats["root_size"] = len(root_idx)
    return HIFFactor(dim, n, leaf, L, eps, levels, root_idx, root_L, stats)


def _replace_diag_blocks(A: sp.csr_matrix, idx_list, val_list, N: int) -> sp.csr_matrix:
    """Replace the diagonal blocks A[I, I] by the given dense matrices."""
    if not idx_list:
        return A
    gid = np.full(N, -1, dtype=np.int64)
    for t, I in enumerate(idx_list):
        gid[I] = t
    C = A.tocoo()
    keep = ~((gid[C.row] >= 0) & (gid[C.row] == gid[C.col]))
    rows = [C.row[keep]]
    cols = [C.col[keep]]
    vals = [C.data[keep]]
    for I, V in zip(idx_list, val_list):
        if len(I) == 0:
            continue
        rr, cc = np.meshgrid(I, I, indexing="ij")
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        vals.append(np.asarray(V).ravel())
    out = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                        shape=(N, N)).tocsr()
    out.sort_indices()
    return out


# -------------------------------------------------------------------------- apply


def _lsolve(L, b):
    return sla.solve_triangular(L, b, lower=True)


def _ltsolve(L, b):
    return sla.solve_triangular(L, b, lower=True, trans="T")


def cell_fwd(c: CellFactor, x: np.ndarray) -> None:
    """x <- E_I^T x (Eq. 2_3): t = L^{-1} x_I; x_B -= A_BI L^{-T} t; x_I = t."""
    t = _lsolve(c.L, x[c.I])
    x[c.B] -= c.A_BI @ _ltsolve(c.L, t)
    x[c.I] = t


def cell_bwd(c: CellFactor, x: np.ndarray) -> None:
    """x <- E_I x: x_I = L^{-T} (x_I - L^{-1} A_BI^T x_B)."""
    x[c.I] = _ltsolve(c.L, x[c.I] - _lsolve(c.L, c.A_BI.T @ x[c.B]))


def jacobi_fwd(j: JacobiFactor, x: np.ndarray) -> None:
    """x <- C_I^T x (Eq. jacobi-precond): x_I = L^{-1} x_I."""
    x[j.I] = _lsolve(j.L, x[j.I])


def jacobi_bwd(j: JacobiFactor, x: np.ndarray) -> None:
    """x <- C_I x: x_I = L^{-T} x_I."""
    x[j.I] = _ltsolve(j.L, x[j.I])


def skel_fwd(k: SkelFactor, x: np.ndarray) -> None:
    """x <- K_I^T x = E^T Z^T x (Eqs. T, 2_9).

    Z^T: x_rd -= T^T x_sk.  Then with S = I + T^T T = Ls Ls^T:
    t = Ls^{-1} x_rd; x_sk += T S^{-1} x_rd = T Ls^{-T} t; x_rd = t.
    """
    xr = x[k.rd] - k.T.T @ x[k.sk]
    t = _lsolve(k.Ls, xr)
    x[k.sk] = x[k.sk] + k.T @ _ltsolve(k.Ls, t)
    x[k.rd] = t


def skel_bwd(k: SkelFactor, x: np.ndarray) -> None:
    """x <- K_I x = Z E x: x_rd = Ls^{-T}(x_rd + Ls^{-1} T^T x_sk); x_sk -= T x_rd."""
    xr = _ltsolve(k.Ls, x[k.rd] + _lsolve(k.Ls, k.T.T @ x[k.sk]))
    x[k.rd] = xr
    x[k.sk] = x[k.sk] - k.T @ xr


def apply_inverse(F: HIFFactor, b: np.ndarray) -> np.ndarray:
    """y = F^{-1} b = R_0 ... R_{L-1} A_L^{-1} R_{L-1}^T ... R_0^T b (Eq. Ainv)."""
    x = np.array(b, dtype=np.float64).ravel().copy()
    for lf in F.level_factors:  # R_l^T = K_l^T C_l^T E_l^T
        for c in lf.cells:
            cell_fwd(c, x)
        for j in lf.jacobi:
            jacobi_fwd(j, x)
        for step in lf.skel_steps:
            for k in step:
                skel_fwd(k, x)
    if len(F.root_idx):
        x[F.root_idx] = _ltsolve(F.root_L, _lsolve(F.root_L, x[F.root_idx]))
    for lf in reversed(F.level_factors):  # R_l = E_l C_l K_l
        for step in reversed(lf.skel_steps):
            for k in step:
                skel_bwd(k, x)
        for j in lf.jacobi:
            jacobi_bwd(j, x)
        for c in lf.cells:
            cell_bwd(c, x)
    return x.reshape(np.shape(b))


def factor_bytes(F: HIFFactor, itemsize: int = 8) -> int:
    """Entries of the stored blocks (L's as triangles) times ``itemsize``."""
    tot = 0
    for lf in F.level_factors:
        for c in lf.cells:
            ni = len(c.I)
            tot += ni * (ni + 1) // 2 + c.A_BI.size
        for j in lf.jacobi:
            ni = len(j.I)
            tot += ni * (ni + 1) // 2
        for step in lf.skel_steps:
            for k in step:
                r = len(k.rd)
                tot += k.T.size + r * (r + 1) // 2
    r = len(F.root_idx)
    tot += r * (r + 1) // 2
    return tot * itemsize
