"""The exported factor blob applies the same operator as the oracle (CPU)."""

import numpy as np
import pytest

import workloads as W
from oracle import export, grid, hif

from blobutil import blob_apply, read_blob


@pytest.mark.parametrize("dim,n,m,eps", [(2, 32, 8, 1e-6), (2, 32, 4, 1e-3), (3, 16, 4, 1e-4),
                                         (2, 16, 4, 0.0)])
def test_blob_apply_matches_oracle(dim, n, m, eps):
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=eps, corr_len=0.2)
    A = grid.assemble_A(w.a_nodes, w.dt)
    F = hif.factor(A, n, dim, m, eps)
    d = read_blob(export.export_blob(F, w.dt))
    assert (d["dim"], d["n"], d["leaf"], d["levels"], d["N"]) == (dim, n, m, F.levels, F.N)
    rng = np.random.default_rng(0)
    for _ in range(3):
        b = rng.standard_normal(F.N)
        y0 = hif.apply_inverse(F, b)
        y1 = blob_apply(d, b)
        assert np.linalg.norm(y1 - y0) <= 1e-12 * np.linalg.norm(y0)
