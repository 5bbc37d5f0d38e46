"""GB300 (sm_103a) block ILU(k) preconditioned BiCGSTAB.

The C-ABI library ``libbilu.so`` (include/bilu.h) holds the method: host
symbolic phase plus CUDA kernels for the backfill, block factorization,
triangular apply, block SpMV and BiCGSTAB.  ``paper_1703_01325_gb300.bilu``
is the thin torch-facing binding with the same names; ``reservoir`` draws the
seeded synthetic inputs.  Importing this package loads nothing; the binding
loads the library on first use and raises if it is not built.
"""

__all__ = ["bilu", "reservoir", "build"]
