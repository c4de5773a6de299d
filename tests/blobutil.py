"""Reader of the "HIFF" v1 factor blob and a plain NumPy apply of it.

Used by the tests to check that the blob the oracle exports describes the same
operator F^{-1} as the oracle's own step-by-step apply, i.e. that the layout
the CUDA library consumes (G = L^{-1}, V = A_BI A_II^{-1}, H = K^T C^T) is
correct before any kernel reads it.
"""

import struct

import numpy as np


def read_blob(blob: bytes):
    p = 0

    def take(fmt):
        nonlocal p
        sz = struct.calcsize(fmt)
        v = struct.unpack_from(fmt, blob, p)
        p += sz
        return v

    def arr(dtype, n):
        nonlocal p
        a = np.frombuffer(blob, dtype=dtype, count=n, offset=p).copy()
        p += a.nbytes
        return a

    assert blob[:4] == b"HIFF"
    p = 4
    ver, dim, n, leaf, levels, _ = take("<6i")
    (N,) = take("<q")
    eps, dt = take("<2d")
    lv = []
    for _ in range(levels):
        nc, ng = take("<2i")
        cells, groups = [], []
        for _ in range(nc):
            nI, nB = take("<2i")
            I = arr("<i4", nI)
            B = arr("<i4", nB)
            Gp = arr("<f8", nI * (nI + 1) // 2)
            V = arr("<f8", nB * nI).reshape(nB, nI)
            G = np.zeros((nI, nI))
            G[np.tril_indices(nI)] = Gp
            cells.append((I, B, G, V))
        for _ in range(ng):
            (m,) = take("<i")
            idx = arr("<i4", m)
            H = arr("<f8", m * m).reshape(m, m)
            groups.append((idx, H))
        lv.append((cells, groups))
    (nr,) = take("<i")
    ridx = arr("<i4", nr)
    Gp = arr("<f8", nr * (nr + 1) // 2)
    Gr = np.zeros((nr, nr))
    Gr[np.tril_indices(nr)] = Gp
    assert p == len(blob)
    return dict(version=ver, dim=dim, n=n, leaf=leaf, levels=levels, N=N, eps=eps, dt=dt,
                levels_data=lv, root=(ridx, Gr))


def blob_apply(d, b):
    x = np.array(b, dtype=np.float64).copy()
    for cells, groups in d["levels_data"]:
        for I, B, G, V in cells:
            x[B] -= V @ x[I]
            x[I] = G @ x[I]
        for idx, H in groups:
            x[idx] = H @ x[idx]
    ridx, Gr = d["root"]
    x[ridx] = Gr.T @ (Gr @ x[ridx])
    for cells, groups in reversed(d["levels_data"]):
        for idx, H in groups:
            x[idx] = H.T @ x[idx]
        for I, B, G, V in cells:
            x[I] = G.T @ x[I] - V.T @ x[B]
    return x
