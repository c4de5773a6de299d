"""Plain, slow FP64 CPU oracle for the HIF-preconditioned Crank-Nicolson step.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` use it.  It shares no code with the
CUDA library (no kernels, headers, helpers or generators); the only common
dependency is the seeded input module ``workloads``.

Modules (each function cites the passage of the paper it follows):

* ``grid``   - grid, variable-coefficient 5/7-point stencil M, A = I - dt/2 M,
               Crank-Nicolson right-hand side and reaction (Sec. 2, Eq. CN2).
* ``hif``    - recursively preconditioned hierarchical interpolative
               factorization: cell elimination, block Jacobi rescaling,
               skeletonization by interpolative decomposition, root Cholesky
               (Sec. 2.2, Eqs. 2_3 - 3_4) and the inverse apply (Eq. Ainv).
* ``pcg``    - preconditioned conjugate gradient and the CN loop (Algorithm 1).
* ``export`` - conversion of an oracle factor to the packed interchange blob
               that the library's ``hif_import_factor`` reads.

Every function is pinned by ``tests/test_oracle_*.py`` (closed forms, exactness
at eps = 0, invariants).  The iteration counts at eps > 0 are pinned loosely,
to within 1.5 iterations, against the counts the paper prints for its Sec. 3
recipes (``tests/golden/paper_iteration_counts.txt``); the paper's draws and
problem sizes differ from the oracle's, so no tighter pin is possible.
"""
