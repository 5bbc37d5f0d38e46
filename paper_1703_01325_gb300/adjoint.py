"""Differentiable block ILU(k)-preconditioned solve x = A^{-1} b.

``BlockILUSolver.solve(vals, rhs)`` runs the forward solve (block ILU(k)
factorization, Algorithm 4 / Eq. 5, inside right-preconditioned BiCGSTAB) and
returns x as a tensor that autograd can differentiate with respect to A's
block values and to b.  The backward pass is the hand-written adjoint of the
exact solve map:

    A^T lambda = dL/dx,     dL/db = lambda,     dL/dA_IJ = -lambda_I x_J^T

on A's block pattern.  The adjoint system is solved by the same BiCGSTAB with
A^T (its block CSR gathered on the device, bsr_gather_transpose) and the
transposed preconditioner M^{-T} = L^{-T} D^{-T} U'^{-T}, i.e. the apply of
Eq. 6 / Algorithm 7 on the transposed pattern P'^T with transposed blocks
(bilu_factor_transpose).  All arithmetic runs in libbilu's kernels; this
module only orders the calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import bilu as B


class BlockILUSolver:
    """A block pattern with its ILU(k) symbolic phase done once.

    ``solve`` may be called with different values on the same pattern; each
    call factors anew (the decoupling of Section 1: the symbolic phase depends
    on the pattern only).
    """

    def __init__(self, n: int, b: int, row_ptr, col_idx, k: int, tol: float = 1e-10, maxit: int = 5000,
                 device="cuda"):
        self.n, self.b, self.k = n, b, k
        self.tol, self.maxit = tol, maxit
        self.device = torch.device(device)
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        self.nnzb = int(rp[n]) if n else 0
        self.P = B.bilu_symbolic(n, rp, ci, k).upload()
        self.rp = torch.from_numpy(rp).to(self.device)
        self.ci = torch.from_numpy(ci).to(self.device)
        self._host_pattern = (rp, ci)
        self._t = None  # (P'^T, row_ptr_t, col_idx_t, perm) once the adjoint is first needed

    def transposed(self):
        if self._t is None:
            rp, ci = self._host_pattern
            rpt, cit, perm = B.bsr_transpose_pattern(self.n, rp, ci)
            dev = self.device
            self._t = (self.P.transpose(), torch.from_numpy(rpt).to(dev), torch.from_numpy(cit).to(dev),
                       torch.from_numpy(perm).to(dev))
        return self._t

    def _solve(self, P, A, F, rhs):
        x, info = B.bicgstab_solve(P, A, F, rhs, tol=self.tol, maxit=self.maxit)
        if info.status != 0:
            raise B.BiluError(info.status, "BlockILUSolver", f" after {info.iters} iterations, "
                                                               f"relres {info.true_relres:.3e}")
        return x

    def solve(self, vals: torch.Tensor, rhs: torch.Tensor) -> torch.Tensor:
        """x = A^{-1} rhs, differentiable in vals (nnzb*b*b) and rhs (n*b)."""
        return _BlockILUSolve.apply(vals, rhs, self)


class _BlockILUSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, rhs, solver: BlockILUSolver):
        vals = vals.detach().contiguous()
        rhs = rhs.detach().contiguous()
        F, finfo = B.bilu_factor(solver.P, solver.b, vals)
        x = solver._solve(solver.P, (solver.n, solver.b, solver.rp, solver.ci, vals), F, rhs)
        ctx.solver = solver
        ctx.F = F
        ctx.save_for_backward(vals, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        s = ctx.solver
        vals, x = ctx.saved_tensors
        PT, rpt, cit, perm = s.transposed()
        FT = B.bilu_factor_transpose(PT, s.b, ctx.F)
        vals_t = B.bsr_gather_transpose(s.b, perm, vals)
        lam = s._solve(PT, (s.n, s.b, rpt, cit, vals_t), FT, gx.detach().contiguous())
        g_vals = B.bsr_outer_grad(s.n, s.b, s.rp, s.ci, lam, x) if ctx.needs_input_grad[0] else None
        g_rhs = lam if ctx.needs_input_grad[1] else None
        return g_vals, g_rhs, None
