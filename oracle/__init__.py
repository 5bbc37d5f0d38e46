"""CPU oracle for the decoupled block-wise ILU(k) method -- TEST INFRASTRUCTURE.

Plain single-threaded C (``bilu_oracle.c``, fp64, no fused multiply-add) loaded
through ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_1703_01325_gb300`` and is never a fallback for it.

Every function takes and returns numpy arrays in block CSR with column-major
b x b blocks (Section 2.1): element (r, c) of block t is ``vals[t, c*b + r]``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build as _build, library_path

_lib = None

OK, ERR_ARG, ERR_PATTERN, ERR_SINGULAR, ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_OOM = range(7)


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str, row: int = -1):
        super().__init__(f"{what}: oracle status {status}" + (f" (row {row})" if row >= 0 else ""))
        self.status = status
        self.row = row


def lib():
    global _lib
    if _lib is None:
        path = library_path()
        src = os.path.join(os.path.dirname(__file__), "bilu_oracle.c")
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(src):
            _build()
        _lib = C.CDLL(path)
        i32p = C.POINTER(C.c_int32)
        f64p = C.POINTER(C.c_double)
        L = _lib
        L.or_check_pattern.argtypes = [C.c_int32, i32p, i32p]
        L.or_symbolic.argtypes = [C.c_int32, i32p, i32p, C.c_int32,
                                  C.POINTER(i32p), C.POINTER(i32p), C.POINTER(i32p)]
        L.or_levels.argtypes = [C.c_int32, i32p, i32p, i32p, i32p]
        L.or_backfill.argtypes = [C.c_int32, C.c_int32, i32p, i32p, f64p, i32p, i32p, f64p]
        L.or_factor.argtypes = [C.c_int32, C.c_int32, i32p, i32p, f64p, f64p, i32p]
        L.or_apply.argtypes = [C.c_int32, C.c_int32, i32p, i32p, f64p, f64p, f64p, f64p]
        L.or_spmv.argtypes = [C.c_int32, C.c_int32, i32p, i32p, f64p, f64p, f64p]
        L.or_bicgstab.argtypes = [C.c_int32, C.c_int32, i32p, i32p, f64p, i32p, i32p, f64p, f64p,
                                  f64p, f64p, C.c_double, C.c_int32, i32p, f64p]
        L.or_gmres.argtypes = [C.c_int32, C.c_int32, i32p, i32p, f64p, i32p, i32p, f64p, f64p,
                               f64p, f64p, C.c_double, C.c_int32, C.c_int32, i32p, f64p]
        L.or_free.argtypes = [C.c_void_p]
        for f in ("or_check_pattern", "or_symbolic", "or_levels", "or_backfill", "or_factor",
                  "or_apply", "or_spmv", "or_bicgstab", "or_gmres"):
            getattr(L, f).restype = C.c_int
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def check_pattern(n, rp, ci) -> int:
    rp, prp = _i32(rp)
    ci, pci = _i32(ci)
    return lib().or_check_pattern(n, prp, pci)


def symbolic(n, rp, ci, k):
    """Algorithm 3 (Eq. 1-2): returns (prp, pci, plev) of the level-<=k pattern P'."""
    rp, prp = _i32(rp)
    ci, pci = _i32(ci)
    orp, oci, olev = C.POINTER(C.c_int32)(), C.POINTER(C.c_int32)(), C.POINTER(C.c_int32)()
    st = lib().or_symbolic(n, prp, pci, k, C.byref(orp), C.byref(oci), C.byref(olev))
    if st != OK:
        raise OracleError(st, "or_symbolic")
    try:
        P_rp = np.ctypeslib.as_array(orp, shape=(n + 1,)).copy()
        nnz = int(P_rp[n])
        P_ci = np.ctypeslib.as_array(oci, shape=(max(nnz, 1),))[:nnz].copy()
        P_lev = np.ctypeslib.as_array(olev, shape=(max(nnz, 1),))[:nnz].copy()
    finally:
        for p in (orp, oci, olev):
            lib().or_free(C.cast(p, C.c_void_p))
    return P_rp, P_ci, P_lev


def levels(n, prp, pci):
    """Eq. 4 dependency levels (0-based) of the lower and upper parts of P'."""
    prp, pp = _i32(prp)
    pci, pc = _i32(pci)
    lo = np.zeros(max(n, 1), np.int32)
    up = np.zeros(max(n, 1), np.int32)
    st = lib().or_levels(n, pp, pc, lo.ctypes.data_as(C.POINTER(C.c_int32)),
                         up.ctypes.data_as(C.POINTER(C.c_int32)))
    if st != OK:
        raise OracleError(st, "or_levels")
    return lo[:n], up[:n]


def backfill(n, b, rp, ci, vals, prp, pci):
    """Algorithm 5 steps 3-4: A' on pattern P' (fill blocks zero)."""
    rp, a = _i32(rp)
    ci, c = _i32(ci)
    vals, v = _f64(vals)
    prp, pp = _i32(prp)
    pci, pc = _i32(pci)
    out = np.zeros((max(len(pci), 1), b * b), np.float64)
    st = lib().or_backfill(n, b, a, c, v, pp, pc, out.ctypes.data_as(C.POINTER(C.c_double)))
    if st != OK:
        raise OracleError(st, "or_backfill")
    return out[: len(pci)]


def factor(n, b, prp, pci, fvals):
    """Algorithm 4 + Eq. 5 on a copy of A'.  Returns (F, Dinv): F holds L (j<i),
    D (j=i) and U' (j>i) blocks; Dinv holds D_i^{-1}."""
    prp, pp = _i32(prp)
    pci, pc = _i32(pci)
    F = np.array(fvals, dtype=np.float64, copy=True, order="C").reshape(-1, b * b)
    dinv = np.zeros((max(n, 1), b * b), np.float64)
    bad = C.c_int32(-1)
    st = lib().or_factor(n, b, pp, pc, F.ctypes.data_as(C.POINTER(C.c_double)),
                         dinv.ctypes.data_as(C.POINTER(C.c_double)), C.byref(bad))
    if st != OK:
        raise OracleError(st, "or_factor", bad.value)
    return F, dinv[:n]


def apply(n, b, prp, pci, F, dinv, r):
    """Eq. 6 / Algorithm 7: x = U'^{-1} D^{-1} L^{-1} r."""
    prp, pp = _i32(prp)
    pci, pc = _i32(pci)
    F, pf = _f64(F)
    dinv, pd = _f64(dinv)
    r, pr = _f64(r)
    x = np.zeros(max(n * b, 1), np.float64)
    st = lib().or_apply(n, b, pp, pc, pf, pd, pr, x.ctypes.data_as(C.POINTER(C.c_double)))
    if st != OK:
        raise OracleError(st, "or_apply")
    return x[: n * b]


def spmv(n, b, rp, ci, vals, x):
    rp, a = _i32(rp)
    ci, c = _i32(ci)
    vals, v = _f64(vals)
    x, px = _f64(x)
    y = np.zeros(max(n * b, 1), np.float64)
    st = lib().or_spmv(n, b, a, c, v, px, y.ctypes.data_as(C.POINTER(C.c_double)))
    if st != OK:
        raise OracleError(st, "or_spmv")
    return y[: n * b]


def bicgstab(n, b, rp, ci, vals, prp, pci, F, dinv, rhs, x0=None, tol=1e-8, maxit=1000):
    """Right-preconditioned BiCGSTAB.  Returns (x, iters, true_relres, status)."""
    rp, a = _i32(rp)
    ci, c = _i32(ci)
    vals, v = _f64(vals)
    prp, pp = _i32(prp)
    pci, pc = _i32(pci)
    F, pf = _f64(F)
    dinv, pd = _f64(dinv)
    rhs, prh = _f64(rhs)
    x = np.zeros(max(n * b, 1), np.float64)
    if x0 is not None:
        x[: n * b] = x0
    it = C.c_int32(0)
    rr = C.c_double(0.0)
    st = lib().or_bicgstab(n, b, a, c, v, pp, pc, pf, pd, prh,
                           x.ctypes.data_as(C.POINTER(C.c_double)), tol, maxit,
                           C.byref(it), C.byref(rr))
    return x[: n * b], it.value, rr.value, st


def gmres(n, b, rp, ci, vals, prp, pci, F, dinv, rhs, x0=None, tol=1e-8, maxit=1000, restart=20):
    """Restarted GMRES(restart), right-preconditioned.  Returns (x, iters,
    true_relres, status)."""
    rp, a = _i32(rp)
    ci, c = _i32(ci)
    vals, v = _f64(vals)
    prp, pp = _i32(prp)
    pci, pc = _i32(pci)
    F, pf = _f64(F)
    dinv, pd = _f64(dinv)
    rhs, prh = _f64(rhs)
    x = np.zeros(max(n * b, 1), np.float64)
    if x0 is not None:
        x[: n * b] = x0
    it = C.c_int32(0)
    rr = C.c_double(0.0)
    st = lib().or_gmres(n, b, a, c, v, pp, pc, pf, pd, prh,
                        x.ctypes.data_as(C.POINTER(C.c_double)), tol, maxit, restart,
                        C.byref(it), C.byref(rr))
    return x[: n * b], it.value, rr.value, st
