"""Oracle factor -> "HIFF" v1 interchange blob (test infrastructure only).

The blob stores, level by level, the operators of the inverse apply (Eq. Ainv)
in explicit form:

* per cell: G = L^{-1} (L = chol(A_II), Eq. 2_3) packed lower by rows, and
  V = A_BI A_II^{-1}, so that E_I^T acts as  x_B -= V x_I, x_I <- G x_I  and
  E_I acts as  x_I <- G^T x_I - V^T x_B;
* per separator entity: H = (K_I^T C_I^T) restricted to the entity's DOFs
  (Eqs. jacobi-precond, T, 2_9): the block Jacobi rescaling followed, for
  skeletonized entities, by Z^T and the elimination of the redundant DOFs;
* root: G_r = L_r^{-1} with A_L = L_r L_r^T (Eq. 3_4).

H is obtained by running the oracle's own step routines on the columns of
the identity, so the blob is by construction the operator the oracle applies.
"""

from __future__ import annotations

import struct

import numpy as np
import scipy.linalg as sla

from . import hif

MAGIC = b"HIFF"
VERSION = 1


def _packed_lower(M: np.ndarray) -> np.ndarray:
    n = M.shape[0]
    return np.concatenate([M[i, : i + 1] for i in range(n)]) if n else np.zeros(0)


def _group_matrix(I: np.ndarray, jac: hif.JacobiFactor, sk: hif.SkelFactor | None) -> np.ndarray:
    """Matrix of the forward group transform restricted to the DOFs I."""
    pos = {int(d): p for p, d in enumerate(I)}
    ljac = hif.JacobiFactor(np.arange(len(I)), jac.L)
    lsk = None
    if sk is not None:
        lsk = hif.SkelFactor(np.arange(len(I)),
                             np.array([pos[int(d)] for d in sk.sk], dtype=np.int64),
                             np.array([pos[int(d)] for d in sk.rd], dtype=np.int64),
                             sk.T, sk.Ls)
    H = np.zeros((len(I), len(I)))
    for c in range(len(I)):
        x = np.zeros(len(I))
        x[c] = 1.0
        hif.jacobi_fwd(ljac, x)
        if lsk is not None:
            hif.skel_fwd(lsk, x)
        H[:, c] = x
    return H


def export_blob(F: hif.HIFFactor, dt: float) -> bytes:
    out = [MAGIC, struct.pack("<6i", VERSION, F.dim, F.n, F.leaf, F.levels, 0),
           struct.pack("<q", F.N), struct.pack("<2d", F.eps, dt)]
    for lf in F.level_factors:
        skel_of = {}
        for step in lf.skel_steps:
            for k in step:
                skel_of[int(k.I[0])] = k
        out.append(struct.pack("<2i", len(lf.cells), len(lf.jacobi)))
        for c in lf.cells:
            G = sla.solve_triangular(c.L, np.eye(len(c.I)), lower=True)
            V = sla.cho_solve((c.L, True), c.A_BI.T).T if len(c.B) else np.zeros((0, len(c.I)))
            out.append(struct.pack("<2i", len(c.I), len(c.B)))
            out.append(np.asarray(c.I, dtype="<i4").tobytes())
            out.append(np.asarray(c.B, dtype="<i4").tobytes())
            out.append(_packed_lower(G).astype("<f8").tobytes())
            out.append(np.ascontiguousarray(V, dtype="<f8").tobytes())
        for j in lf.jacobi:
            sk = skel_of.get(int(j.I[0]))
            if sk is not None:
                assert np.array_equal(sk.I, j.I)
            H = _group_matrix(j.I, j, sk)
            out.append(struct.pack("<i", len(j.I)))
            out.append(np.asarray(j.I, dtype="<i4").tobytes())
            out.append(np.ascontiguousarray(H, dtype="<f8").tobytes())
    nr = len(F.root_idx)
    Gr = sla.solve_triangular(F.root_L, np.eye(nr), lower=True) if nr else np.zeros((0, 0))
    out.append(struct.pack("<i", nr))
    out.append(np.asarray(F.root_idx, dtype="<i4").tobytes())
    out.append(_packed_lower(Gr).astype("<f8").tobytes())
    return b"".join(out)
