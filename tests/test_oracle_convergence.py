"""The oracle's CN discretization converges to the PDE at second order.

Sec. 2 builds the scheme from second-order differences in space and the
Crank-Nicolson rule in time, and the paper steps with dt = h.  The error is then
O(h^2), and Sec. 3 (Example 2, the error plot) reports the error of the
logistic problem as close to second order asymptotically.  These tests check
the oracle against the continuous problem, not against its own discrete
closed form:

* a = 1: u = sin(pi x) sin(pi y) exp(-2 pi^2 t) solves the heat equation
  exactly, and halving h (and dt = h) must divide the error by about 4;
* the paper's 2D logistic recipe (variable a, explicit reaction): differences
  of solutions on successively refined grids, compared at the common nodes,
  must shrink by close to 4 per halving.
"""

import math

import numpy as np
import pytest

import workloads as W
from oracle import pcg


def _solve(a_nodes, u0, T, n, reaction=(0, 0.0, 0.0), leaf=8):
    steps = int(round(T * n))  # dt = h = 1/n, as in the paper's examples
    u, _, _ = pcg.cn_solve(a_nodes, u0, T / steps, steps, leaf, 1e-10, reaction, tol=1e-13)
    return u


def test_heat_a1_second_order_against_exact_solution():
    T = 0.25
    errs = []
    for n in (16, 32, 64, 128):
        xs = W.interior_coords(n, 2)
        u0 = np.sin(math.pi * xs[0]) * np.sin(math.pi * xs[1])
        u = _solve(np.ones((n + 1,) * 2), u0, T, n)
        exact = u0 * math.exp(-2.0 * math.pi ** 2 * T)
        errs.append(np.linalg.norm(u - exact) / np.linalg.norm(exact))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(r > 3.5 for r in ratios), ratios
    assert abs(ratios[-1] - 4.0) < 0.2, ratios


@pytest.mark.slow
def test_logistic_recipe_close_to_second_order():
    T = 1.0 / 16
    sols = {}
    for n in (64, 128, 256):
        w = W.paper_logistic2d(n, 8, 1e-10, seed=0)
        sols[n] = _solve(w.a_nodes, w.u0, T, n, w.reaction, w.leaf)
    # node j of the grid with spacing 1/n is node 2j of the grid with 1/(2n)
    d1 = np.linalg.norm(sols[64] - sols[128][1::2, 1::2]) / np.linalg.norm(sols[128])
    d2 = np.linalg.norm(sols[128] - sols[256][1::2, 1::2]) / np.linalg.norm(sols[256])
    assert d2 < d1
    assert d1 / d2 > 3.0, (d1, d2)  # observed order > 1.58, approaching 2
