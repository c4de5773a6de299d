"""Pin of the whole oracle chain (stencil, PHIF factor, PCG, CN loop) to the
iteration counts the paper prints, and of the factor to its printed accuracy.

The four result tables of Sec. 3 give n_i, the mean number of PHIF-PCG
iterations per CN step at relative residual 1e-12, for the heat and the logistic
examples in 2D and 3D at eps = 1e-3 and 1e-6 (``golden/paper_iteration_counts.txt``).
The paper reports these counts as essentially independent of N; across a
256-fold range of N its printed means move by at most 1.7 iterations.  The
oracle runs the same recipes (Sec. 3: Gaussian-bump coefficient fields, the
printed initial conditions, dt = h in 2D and 0.1 h in 3D) on small grids, and
its mean count must lie within 1.5 iterations of the count printed for the
smallest problem, with eps = 1e-6 needing fewer iterations than eps = 1e-3.

The window is loose on purpose: the paper's draws, sizes and FLAM-based
factorization differ from these.  It is still narrow against real mistakes.
On the 63^2 heat case, these faults each break the pin:
* dropping the cell Schur updates (61 iterations);
* flipping their sign (85);
* leaving out the skeleton diagonal correction (42-48);
* loosening the ID tolerance 100-fold (11 at eps = 1e-3).
Omitting the block-Jacobi scaling, or the I + T^T T of the redundant block,
makes the factorization fail outright.
"""

import os

import numpy as np
import pytest

import workloads as W
from oracle import pcg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "paper_iteration_counts.txt")
WINDOW = 1.5
STEPS = 3


def _load():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            ex, dim, eps, side, ni = line.split()
            rows.append((ex, int(dim), float(eps), int(side), float(ni)))
    return rows


def _printed_smallest(ex, dim, eps):
    rows = [r for r in _load() if r[:3] == (ex, dim, eps)]
    return min(rows, key=lambda r: r[3])[4]


def _workload(ex, dim, eps):
    if dim == 2:
        gen = W.paper_heat2d if ex == "heat" else W.paper_logistic2d
        return gen(64, 8, eps, seed=0)
    return W.paper_heat3d(16, 4, eps, seed=0, logistic=(ex == "logistic"))


def _mean_iters(w):
    _, iters, _ = pcg.cn_solve(w.a_nodes, w.u0, w.dt, STEPS, w.leaf, w.eps, w.reaction,
                               tol=w.tol)
    return float(np.mean(iters))


def test_golden_table_is_complete():
    rows = _load()
    assert len(rows) == 28
    for ex in ("heat", "logistic"):
        for dim in (2, 3):
            for eps in (1e-3, 1e-6):
                sides = sorted(r[3] for r in rows if r[:3] == (ex, dim, eps))
                assert sides == ([511, 1023, 2047, 4095] if dim == 2 else [63, 127, 255])
    # the paper's own observation that the counts hardly move with N
    for ex in ("heat", "logistic"):
        for dim in (2, 3):
            for eps in (1e-3, 1e-6):
                ni = [r[4] for r in rows if r[:3] == (ex, dim, eps)]
                assert max(ni) - min(ni) <= 1.7


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("ex", ["heat", "logistic"])
def test_oracle_counts_match_printed(ex, dim):
    got = {}
    for eps in (1e-3, 1e-6):
        w = _workload(ex, dim, eps)
        assert w.tol == 1e-12
        got[eps] = _mean_iters(w)
        printed = _printed_smallest(ex, dim, eps)
        assert abs(got[eps] - printed) <= WINDOW, (ex, dim, eps, got[eps], printed)
    assert got[1e-6] < got[1e-3]


@pytest.mark.slow
def test_oracle_counts_do_not_grow_with_N():
    """63^2 against 127^2 on the 2D heat recipe: the same count to within one."""
    a = _mean_iters(W.paper_heat2d(64, 8, 1e-3, seed=0))
    b = _mean_iters(W.paper_heat2d(128, 8, 1e-3, seed=0))
    assert abs(a - b) <= 1.0


def test_factor_error_matches_printed():
    """Sec. 3, Example 1: the paper estimates ||I - A F^{-1}|| = 7.9e-6 at
    eps = 1e-6 (``golden/paper_factor_error.txt``).  On the same recipe at 63^2
    the oracle's estimate (the same power iteration) must lie within a factor
    of 10 of it: the paper's grid is 4000 times larger and the norm grows
    slowly with N (2.6e-6 at 63^2, 5.6e-6 at 127^2).  A 100-fold looser ID gives
    3.4e-4, a 100-fold tighter one 2.2e-8, and a missing skeleton diagonal
    correction gives 3.6."""
    from oracle import grid, hif
    from test_oracle_hif import _power_norm_I_minus_AFinv
    path = os.path.join(os.path.dirname(GOLDEN), "paper_factor_error.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.lstrip().startswith("#")]
    (ex, dim, eps, side, printed), = rows
    assert (ex, dim, float(eps), side) == ("heat", "2", 1e-6, "4095")
    printed = float(printed)
    w = W.paper_heat2d(64, 8, float(eps), seed=0)
    A = grid.assemble_A(w.a_nodes, w.dt)
    F = hif.factor(A, w.n, 2, w.leaf, w.eps)
    e = _power_norm_I_minus_AFinv(A, F, iters=30)
    assert printed / 10 <= e <= printed * 10, (e, printed)


@pytest.mark.slow
@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_oracle_counts_at_the_papers_own_size(eps):
    """511^2, the smallest 2D heat row of the Sec. 3 table, at its own size: the
    oracle's mean over three steps (4.67 at eps = 1e-3, 2.33 at 1e-6) must lie
    within one iteration of the printed mean over 100 steps (4.6 and 2.3)."""
    w = W.paper_heat2d(512, 8, eps, seed=0)
    got = _mean_iters(w)
    printed = [r[4] for r in _load() if r[:4] == ("heat", 2, eps, 511)][0]
    assert abs(got - printed) <= 1.0, (got, printed)
