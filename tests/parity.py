"""Comparison helpers of the GPU parity tests.

``rel_err(a, b)`` is the larger of two relative errors of ``a`` against the
reference ``b``:

* normwise, ||a - b||_2 / ||b||_2;
* element by element, max_i |a_i - b_i| / max_i |b_i|: every entry is held to
  the bar, relative to the largest reference entry, so one bad entry (a wrong
  index, a missed boundary DOF) cannot hide in the norm of a large vector.

A test asserting ``rel_err(a, b) <= tol`` therefore checks both.
"""

import numpy as np


def rel_err(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    assert a.shape == b.shape, (a.shape, b.shape)
    if b.size == 0:
        return 0.0
    d = np.abs(a - b)
    nb = float(np.linalg.norm(b))
    mb = float(np.abs(b).max())
    norm_rel = float(np.linalg.norm(d)) / nb if nb > 0 else float(np.linalg.norm(d))
    elem_rel = float(d.max()) / mb if mb > 0 else float(d.max())
    return max(norm_rel, elem_rel)


def assert_close(a, b, tol: float) -> None:
    """Both relative errors of ``rel_err`` at most ``tol``; the message names the
    worst entry."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    e = rel_err(a, b)
    if e > tol:
        i = int(np.argmax(np.abs(a - b)))
        raise AssertionError(f"relative error {e:.3e} > {tol:g}; worst entry {i}: "
                             f"{a[i]!r} vs {b[i]!r}")
