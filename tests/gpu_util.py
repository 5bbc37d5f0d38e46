"""Helpers of the GPU parity tests: run the oracle and the library on the same
seeded inputs and compare."""
from __future__ import annotations

import numpy as np

import oracle

# Tolerances (FP64): factors and applies 1e-10 relative (max-norm over the
# compared section), SpMV 1e-13 relative, solutions 1e-8 relative.
TOL_FACTOR = 1e-10
TOL_APPLY = 1e-10
TOL_SPMV = 1e-13
TOL_X = 1e-8


def rel_maxerr(got: np.ndarray, ref: np.ndarray) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    if ref.size == 0:
        return 0.0
    scale = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (scale if scale > 0 else 1.0))


class OracleRun:
    """The oracle's symbolic + backfill + factor for one system."""

    def __init__(self, n, b, rp, ci, vals, k):
        self.n, self.b = n, b
        self.rp, self.ci, self.vals = rp, ci, vals
        self.prp, self.pci, self.plev = oracle.symbolic(n, rp, ci, k)
        self.A1 = oracle.backfill(n, b, rp, ci, vals, self.prp, self.pci)
        self.F, self.Dinv = oracle.factor(n, b, self.prp, self.pci, self.A1)
        rows = np.repeat(np.arange(n), np.diff(self.prp))
        self.lower = self.pci < rows
        self.upper = self.pci > rows

    def L(self):
        return self.F[self.lower]

    def U(self):
        return self.F[self.upper]

    def apply(self, r):
        return oracle.apply(self.n, self.b, self.prp, self.pci, self.F, self.Dinv, r)

    def spmv(self, x):
        return oracle.spmv(self.n, self.b, self.rp, self.ci, self.vals, x)


def device_system(S, device):
    import torch
    rp = torch.from_numpy(np.ascontiguousarray(S.row_ptr)).to(device)
    ci = torch.from_numpy(np.ascontiguousarray(S.col_idx)).to(device)
    vals = torch.from_numpy(np.ascontiguousarray(S.vals).reshape(-1)).to(device)
    rhs = torch.from_numpy(np.ascontiguousarray(S.rhs)).to(device)
    return rp, ci, vals, rhs
