"""Structure and size of the oracle's factor against what the geometry and
the paper fix.

* At eps = 0 no interpolative decomposition drops anything. The hierarchy is
  then nested dissection, and the root holds exactly the top-level separator.
  In 2D that is the cross of two grid lines, 2(n-1) - 1 DOFs. In 3D it is the
  three mid-planes, 3(n-1)^2 - 3(n-1) + 1 DOFs.
* At eps > 0 the skeletonization keeps few DOFs per separator. That is what
  makes the factorization linear in time and its apply O(N) (Sec. 2.3, the
  paragraph that opens the CN algorithm). Doubling n must leave the root
  nearly unchanged and the stored values per unknown nearly constant.
  Without compression, the root doubles and the values per unknown grow by
  the nested-dissection log factor.
"""

import pytest

import workloads as W
from oracle import grid, hif


@pytest.mark.parametrize("dim,n,m", [(2, 32, 8), (2, 64, 8), (3, 8, 4), (3, 16, 4), (3, 16, 8)])
def test_exact_root_is_the_top_separator(dim, n, m):
    w = W.small_variable_2d(n=n, m=m, dim=dim, eps=0.0, contrast=1e2, dt=0.1)
    F = hif.factor(grid.assemble_A(w.a_nodes, w.dt), n, dim, m, 0.0)
    k = n - 1
    top = 2 * k - 1 if dim == 2 else 3 * k * k - 3 * k + 1
    assert F.stats["root_size"] == top


def test_compressed_root_and_memory_stay_flat():
    out = {}
    for eps in (0.0, 1e-3):
        for n in (64, 128):
            w = W.paper_heat2d(n, 8, 1e-3, seed=0)
            F = hif.factor(grid.assemble_A(w.a_nodes, w.dt), n, 2, 8, eps)
            out[eps, n] = (F.stats["root_size"], hif.factor_bytes(F) / w.N)
    # exact: the root doubles with n, the bytes per unknown grow (log factor)
    assert out[0.0, 128][0] == 2 * out[0.0, 64][0] + 3
    assert out[0.0, 128][1] / out[0.0, 64][1] > 1.12
    # compressed: the root and the bytes per unknown barely move
    assert out[1e-3, 64][0] < out[0.0, 64][0] / 3
    assert out[1e-3, 128][0] / out[1e-3, 64][0] < 1.3
    assert out[1e-3, 128][1] / out[1e-3, 64][1] < 1.1
