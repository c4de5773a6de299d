"""GB300-native HIF-preconditioned Crank-Nicolson solver (arxiv 2004.05566).

The solver is the CUDA library ``_lib/libhifcn.so`` behind the C ABI of
``include/hifcn.h``; ``hifcn`` is its Python binding (argument marshalling
only).  Build with ``paper_2004_05566_gb300.build.build()``.
"""

__all__ = ["hifcn", "build"]
