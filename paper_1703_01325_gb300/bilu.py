"""Python face of libbilu: the same names as the C ABI, taking torch tensors.

Argument marshalling only (dtype/device checks, pointer and stream
extraction, buffer allocation through torch).  PyTorch provides device memory
and streams; every step of the method runs in libbilu's CUDA kernels and its
host symbolic phase.  Errors from the library raise ``BiluError``.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


class BiluError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        msg = L.load().bilu_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status}){detail}")
        self.status = status


def _check(status: int, what: str, detail: str = ""):
    if status != L.BILU_OK:
        raise BiluError(status, what, detail)


def _stream_handle(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str) -> C.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _host_i32(a) -> np.ndarray:
    if isinstance(a, torch.Tensor):
        a = a.cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.int32)


class Pattern:
    """Library-owned level-of-fill pattern (handle from bilu_symbolic)."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle
        info = L.PatternInfo()
        _check(L.load().bilu_pattern_query(self._h, C.byref(info)), "bilu_pattern_query")
        self.info = info
        self.uploaded = False

    @property
    def handle(self) -> C.c_void_p:
        if self._h is None:
            raise ValueError("pattern destroyed")
        return self._h

    @property
    def n(self) -> int:
        return self.info.n

    def export(self):
        """P' and the Eq. 4 levels as numpy arrays (bilu_pattern_export)."""
        n, nnz = self.info.n, self.info.nnz_p
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(max(nnz, 1), np.int32)
        lev = np.zeros(max(nnz, 1), np.int32)
        lo = np.zeros(max(n, 1), np.int32)
        up = np.zeros(max(n, 1), np.int32)
        p = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
        _check(L.load().bilu_pattern_export(self.handle, p(rp), p(ci), p(lev), p(lo), p(up)),
               "bilu_pattern_export")
        return dict(row_ptr=rp, col_idx=ci[:nnz], lev=lev[:nnz], lvl_lower=lo[:n], lvl_upper=up[:n])

    def upload(self, stream=None):
        """bilu_pattern_upload: the device copy and the schedules."""
        _check(L.load().bilu_pattern_upload(self.handle, _stream_handle(stream)), "bilu_pattern_upload")
        self.uploaded = True
        return self

    def reschedule(self, stream=None):
        """bilu_pattern_schedule: rebuild the schedules with the current tuning
        settings (chunk targets)."""
        _check(L.load().bilu_pattern_schedule(self.handle, _stream_handle(stream)), "bilu_pattern_schedule")
        return self

    def schedule_info(self) -> dict:
        """bilu_pattern_schedule_info: rows per chunk of the current solve and
        factorization schedules."""
        sr, fr = C.c_int32(), C.c_int32()
        _check(L.load().bilu_pattern_schedule_info(self.handle, C.byref(sr), C.byref(fr)),
               "bilu_pattern_schedule_info")
        return {"solve_rows": sr.value, "factor_rows": fr.value}

    def schedule(self, rows: int) -> dict:
        """The sync-free solve schedule for a target of `rows` rows per chunk
        (bilu_schedule_export): chunk bounds, chunk-local row orders and the
        chunk claim orders of both solves."""
        n = self.info.n
        nch = C.c_int32(0)
        bounds = np.zeros(n + 1, np.int32)
        lo = np.zeros(max(n, 1), np.int32)
        up = np.zeros(max(n, 1), np.int32)
        tl = np.zeros(max(n, 1), np.int32)
        tu = np.zeros(max(n, 1), np.int32)
        p = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
        _check(L.load().bilu_schedule_export(self.handle, rows, C.byref(nch), p(bounds), p(lo), p(up), p(tl),
                                             p(tu)), "bilu_schedule_export")
        m = nch.value
        return {"bounds": bounds[:m + 1], "ord_lower": lo[:n], "ord_upper": up[:n], "tick_lower": tl[:m],
                "tick_upper": tu[:m]}

    def factor_bytes(self, b: int) -> int:
        return int(L.load().bilu_factor_bytes(self.handle, b))

    def factor_workspace_bytes(self, b: int) -> int:
        return int(L.load().bilu_factor_workspace_bytes(self.handle, b))

    def apply_workspace_bytes(self, b: int) -> int:
        return int(L.load().bilu_apply_workspace_bytes(self.handle, b))

    def bicgstab_workspace_bytes(self, b: int) -> int:
        return int(L.load().bicgstab_workspace_bytes(self.handle, b))

    def bicgstab_mixed_workspace_bytes(self, b: int) -> int:
        return int(L.load().bicgstab_mixed_workspace_bytes(self.handle, b))

    def factor_bytes_f32(self, b: int) -> int:
        return int(L.load().bilu_factor_bytes_f32(self.handle, b))

    def transpose(self, upload: bool = True) -> "Pattern":
        """P'^T for the adjoint solve (bilu_pattern_transpose)."""
        h = C.c_void_p()
        _check(L.load().bilu_pattern_transpose(self.handle, C.byref(h)), "bilu_pattern_transpose")
        pt = Pattern(h)
        return pt.upload() if upload else pt

    def close(self):
        if self._h is not None:
            L.load().bilu_destroy_pattern(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bilu_symbolic(n: int, row_ptr, col_idx, k: int) -> Pattern:
    """Level-of-fill pattern P' of ILU(k) (host; Algorithm 3, Eq. 1-2, Eq. 4)."""
    rp = _host_i32(row_ptr)
    ci = _host_i32(col_idx)
    if len(rp) != n + 1:
        raise ValueError("row_ptr must hold n + 1 entries")
    h = C.c_void_p()
    p = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    _check(L.load().bilu_symbolic(n, p(rp), p(ci) if len(ci) else None, k, C.byref(h)), "bilu_symbolic")
    return Pattern(h)


def bilu_symbolic_gpu(n: int, row_ptr, col_idx, k: int, row_capacity: int = 256, stream=None) -> Pattern:
    """The same pattern as bilu_symbolic, with Algorithm 3's row merges run on
    the current CUDA device (bilu_symbolic_gpu)."""
    rp = _host_i32(row_ptr)
    ci = _host_i32(col_idx)
    if len(rp) != n + 1:
        raise ValueError("row_ptr must hold n + 1 entries")
    h = C.c_void_p()
    p = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    _check(L.load().bilu_symbolic_gpu(n, p(rp), p(ci) if len(ci) else None, k, row_capacity,
                                      _stream_handle(stream), C.byref(h)), "bilu_symbolic_gpu")
    return Pattern(h)


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """A device scratch buffer of at least nbytes bytes (torch allocation)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8,
                       device=device if device is not None else "cuda")


def new_factors(pattern: Pattern, b: int, device=None) -> torch.Tensor:
    nb = pattern.factor_bytes(b)
    return torch.empty(max(nb // 8, 1), dtype=torch.float64, device=device if device is not None else "cuda")


def factor_sections(pattern: Pattern, b: int, factors: torch.Tensor):
    """Views (L, Dinv, U') of a factor buffer, each shaped (blocks, b*b)."""
    bb = b * b
    nl, n, nu = pattern.info.nnz_l, pattern.info.n, pattern.info.nnz_u
    f = factors[: (nl + n + nu) * bb].view(-1, bb) if (nl + n + nu) else factors[:0].view(0, bb)
    return f[:nl], f[nl:nl + n], f[nl + n:nl + n + nu]


def bilu_factor(pattern: Pattern, b: int, a_vals: torch.Tensor, factors: torch.Tensor | None = None,
                work: torch.Tensor | None = None, stream=None, check: bool = True):
    """Backfill + Algorithm 4 + Eq. 5 on the device.  Returns (factors, info)."""
    if factors is None:
        factors = new_factors(pattern, b, a_vals.device)
    if work is None:
        work = workspace(pattern.factor_workspace_bytes(b), a_vals.device)
    info = L.FactorInfo()
    st = L.load().bilu_factor(pattern.handle, b, _dev(a_vals, torch.float64, "a_vals"),
                              _dev(factors, torch.float64, "factors"), _dev(work, torch.uint8, "work"),
                              work.numel(), _stream_handle(stream), C.byref(info))
    if check:
        _check(st, "bilu_factor", f" (bad_row {info.bad_row})" if st == L.BILU_ERR_SINGULAR else "")
    return factors, info


def bilu_apply(pattern: Pattern, b: int, factors: torch.Tensor, r: torch.Tensor,
               x: torch.Tensor | None = None, work: torch.Tensor | None = None, stream=None):
    """x = (L D U')^{-1} r on the device (Eq. 6, Algorithm 7).  Asynchronous."""
    if x is None:
        x = torch.empty_like(r)
    if work is None:
        work = workspace(pattern.apply_workspace_bytes(b), r.device)
    _check(L.load().bilu_apply(pattern.handle, b, _dev(factors, torch.float64, "factors"),
                               _dev(r, torch.float64, "r"), _dev(x, torch.float64, "x"),
                               _dev(work, torch.uint8, "work"), work.numel(), _stream_handle(stream)),
           "bilu_apply")
    return x


def bilu_apply_noalloc(pattern: Pattern, b: int, factors: torch.Tensor, r: torch.Tensor,
                       x: torch.Tensor, stream=None) -> int:
    """x = (L D U')^{-1} r using the library's fixed scratch array instead of a
    workspace (for callers that may not allocate device memory).  The caller
    still provides x.  Returns the library status (BILU_ERR_STATE when the
    system is too large for the fixed scratch)."""
    return L.load().bilu_apply_noalloc(pattern.handle, b, _dev(factors, torch.float64, "factors"),
                                       _dev(r, torch.float64, "r"), _dev(x, torch.float64, "x"),
                                       _stream_handle(stream))


def bilu_apply_noalloc_status(stream=None) -> int:
    """Status the last bilu_apply_noalloc on the current device recorded in the
    fixed scratch (synchronises the stream; allocates nothing)."""
    return L.load().bilu_apply_noalloc_status(_stream_handle(stream))


def bilu_workspace_status(work: torch.Tensor, stream=None) -> int:
    return L.load().bilu_workspace_status(_dev(work, torch.uint8, "work"), _stream_handle(stream))


def bsr_spmv(n: int, b: int, row_ptr: torch.Tensor, col_idx: torch.Tensor, vals: torch.Tensor,
             x: torch.Tensor, y: torch.Tensor | None = None, stream=None):
    """y = A x for a block CSR matrix on the device.  Asynchronous."""
    if y is None:
        y = torch.empty_like(x)
    _check(L.load().bsr_spmv(n, b, _dev(row_ptr, torch.int32, "row_ptr"), _dev(col_idx, torch.int32, "col_idx"),
                             _dev(vals, torch.float64, "vals"), _dev(x, torch.float64, "x"),
                             _dev(y, torch.float64, "y"), _stream_handle(stream)), "bsr_spmv")
    return y


def bicgstab_solve(pattern: Pattern, A, factors: torch.Tensor, rhs: torch.Tensor,
                   x: torch.Tensor | None = None, tol: float = 1e-8, maxit: int = 1000,
                   work: torch.Tensor | None = None, stream=None):
    """Right-preconditioned BiCGSTAB on the device.  A = (n, b, row_ptr, col_idx,
    vals) with device tensors.  Returns (x, info); info.status says whether it
    converged (no exception for NOT_CONVERGED / BREAKDOWN / TIMEOUT)."""
    n, b, rp, ci, vals = A
    if x is None:
        x = torch.zeros_like(rhs)
    if work is None:
        work = workspace(pattern.bicgstab_workspace_bytes(b), rhs.device)
    bsr = L.BSR(n, b, _dev(rp, torch.int32, "row_ptr"), _dev(ci, torch.int32, "col_idx"),
                _dev(vals, torch.float64, "vals"))
    info = L.SolveInfo()
    st = L.load().bicgstab_solve(pattern.handle, C.byref(bsr), _dev(factors, torch.float64, "factors"),
                                 _dev(rhs, torch.float64, "rhs"), _dev(x, torch.float64, "x"), tol, maxit,
                                 _dev(work, torch.uint8, "work"), work.numel(), _stream_handle(stream),
                                 C.byref(info))
    if st in (L.BILU_ERR_ARG, L.BILU_ERR_STATE, L.BILU_ERR_CUDA, L.BILU_ERR_OOM):
        _check(st, "bicgstab_solve")
    return x, info


def bicgstab_solve_f32prec(pattern: Pattern, A, factors32: torch.Tensor, rhs: torch.Tensor,
                           x: torch.Tensor | None = None, tol: float = 1e-8, maxit: int = 1000,
                           work: torch.Tensor | None = None, stream=None):
    """FP64 BiCGSTAB with the FP32-stored preconditioner (bicgstab_solve_f32prec)."""
    n, b, rp, ci, vals = A
    if x is None:
        x = torch.zeros_like(rhs)
    if work is None:
        work = workspace(pattern.bicgstab_workspace_bytes(b), rhs.device)
    bsr = L.BSR(n, b, _dev(rp, torch.int32, "row_ptr"), _dev(ci, torch.int32, "col_idx"),
                _dev(vals, torch.float64, "vals"))
    info = L.SolveInfo()
    st = L.load().bicgstab_solve_f32prec(pattern.handle, C.byref(bsr), _dev(factors32, torch.float32, "factors32"),
                                         _dev(rhs, torch.float64, "rhs"), _dev(x, torch.float64, "x"), tol, maxit,
                                         _dev(work, torch.uint8, "work"), work.numel(), _stream_handle(stream),
                                         C.byref(info))
    if st in (L.BILU_ERR_ARG, L.BILU_ERR_STATE, L.BILU_ERR_CUDA, L.BILU_ERR_OOM):
        _check(st, "bicgstab_solve_f32prec")
    return x, info


def gmres_solve(pattern: Pattern, A, factors: torch.Tensor, rhs: torch.Tensor, x: torch.Tensor | None = None,
                tol: float = 1e-8, maxit: int = 1000, restart: int = 20, work: torch.Tensor | None = None,
                stream=None):
    """Restarted GMRES(restart), right-preconditioned, on the device.  Same
    conventions as bicgstab_solve; info.iters counts Arnoldi steps."""
    n, b, rp, ci, vals = A
    if x is None:
        x = torch.zeros_like(rhs)
    if work is None:
        nb = int(L.load().gmres_workspace_bytes(pattern.handle, b, restart))
        if nb == 0:
            _check(L.BILU_ERR_ARG, "gmres_workspace_bytes")
        work = workspace(nb, rhs.device)
    bsr = L.BSR(n, b, _dev(rp, torch.int32, "row_ptr"), _dev(ci, torch.int32, "col_idx"),
                _dev(vals, torch.float64, "vals"))
    info = L.SolveInfo()
    st = L.load().gmres_solve(pattern.handle, C.byref(bsr), _dev(factors, torch.float64, "factors"),
                              _dev(rhs, torch.float64, "rhs"), _dev(x, torch.float64, "x"), tol, maxit, restart,
                              _dev(work, torch.uint8, "work"), work.numel(), _stream_handle(stream), C.byref(info))
    if st in (L.BILU_ERR_ARG, L.BILU_ERR_STATE, L.BILU_ERR_CUDA, L.BILU_ERR_OOM):
        _check(st, "gmres_solve")
    return x, info


# ---- mixed precision ----

def bilu_convert_f32(src: torch.Tensor, dst: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """FP32 copy of an FP64 device array (factors or matrix values)."""
    if dst is None:
        dst = torch.empty(src.numel(), dtype=torch.float32, device=src.device)
    _check(L.load().bilu_convert_f32(_dev(src, torch.float64, "src"), _dev(dst, torch.float32, "dst"),
                                     src.numel(), _stream_handle(stream)), "bilu_convert_f32")
    return dst


def bilu_factor_f32(pattern: Pattern, b: int, a_vals: torch.Tensor, factors32: torch.Tensor | None = None,
                    work: torch.Tensor | None = None, stream=None, check: bool = True):
    """The factorization computed and stored in FP32 (from FP64 A values)."""
    if factors32 is None:
        nb = int(L.load().bilu_factor_bytes_f32(pattern.handle, b))
        factors32 = torch.empty(max(nb // 4, 1), dtype=torch.float32, device=a_vals.device)
    if work is None:
        work = workspace(pattern.factor_workspace_bytes(b), a_vals.device)
    info = L.FactorInfo()
    st = L.load().bilu_factor_f32(pattern.handle, b, _dev(a_vals, torch.float64, "a_vals"),
                                  _dev(factors32, torch.float32, "factors32"), _dev(work, torch.uint8, "work"),
                                  work.numel(), _stream_handle(stream), C.byref(info))
    if check:
        _check(st, "bilu_factor_f32", f" (bad_row {info.bad_row})" if st == L.BILU_ERR_SINGULAR else "")
    return factors32, info


def bilu_apply_f32(pattern: Pattern, b: int, factors32: torch.Tensor, r: torch.Tensor,
                   x: torch.Tensor | None = None, work: torch.Tensor | None = None, stream=None):
    """x = M^{-1} r with FP32-stored factors (FP32 arithmetic, FP64 vectors)."""
    if x is None:
        x = torch.empty_like(r)
    if work is None:
        work = workspace(pattern.apply_workspace_bytes(b), r.device)
    _check(L.load().bilu_apply_f32(pattern.handle, b, _dev(factors32, torch.float32, "factors32"),
                                   _dev(r, torch.float64, "r"), _dev(x, torch.float64, "x"),
                                   _dev(work, torch.uint8, "work"), work.numel(), _stream_handle(stream)),
           "bilu_apply_f32")
    return x


def bsr_spmv_f32(n: int, b: int, row_ptr: torch.Tensor, col_idx: torch.Tensor, vals32: torch.Tensor,
                 x: torch.Tensor, y: torch.Tensor | None = None, stream=None):
    """y = A x with A's values in FP32 (FP32 arithmetic, FP64 vectors)."""
    if y is None:
        y = torch.empty_like(x)
    _check(L.load().bsr_spmv_f32(n, b, _dev(row_ptr, torch.int32, "row_ptr"),
                                 _dev(col_idx, torch.int32, "col_idx"), _dev(vals32, torch.float32, "vals32"),
                                 _dev(x, torch.float64, "x"), _dev(y, torch.float64, "y"),
                                 _stream_handle(stream)), "bsr_spmv_f32")
    return y


def bsr_spmv_f32x(n: int, b: int, row_ptr: torch.Tensor, col_idx: torch.Tensor, vals32: torch.Tensor,
                  x32: torch.Tensor, y: torch.Tensor | None = None, stream=None):
    """y = A x with A's values and x in FP32 (FP32 arithmetic, y in FP64)."""
    if y is None:
        y = torch.empty(x32.shape, dtype=torch.float64, device=x32.device)
    _check(L.load().bsr_spmv_f32x(n, b, _dev(row_ptr, torch.int32, "row_ptr"),
                                  _dev(col_idx, torch.int32, "col_idx"), _dev(vals32, torch.float32, "vals32"),
                                  _dev(x32, torch.float32, "x32"), _dev(y, torch.float64, "y"),
                                  _stream_handle(stream)), "bsr_spmv_f32x")
    return y


def bicgstab_solve_mixed(pattern: Pattern, A, vals32: torch.Tensor, factors32: torch.Tensor,
                         rhs: torch.Tensor, x: torch.Tensor | None = None, tol: float = 1e-8,
                         maxit: int = 1000, inner_tol: float = 1e-4, inner_maxit: int = 200,
                         work: torch.Tensor | None = None, stream=None):
    """FP64 iterative refinement around FP32-preconditioned BiCGSTAB.
    Returns (x, info) like bicgstab_solve."""
    n, b, rp, ci, vals = A
    if x is None:
        x = torch.zeros_like(rhs)
    if work is None:
        work = workspace(int(L.load().bicgstab_mixed_workspace_bytes(pattern.handle, b)), rhs.device)
    bsr = L.BSR(n, b, _dev(rp, torch.int32, "row_ptr"), _dev(ci, torch.int32, "col_idx"),
                _dev(vals, torch.float64, "vals"))
    info = L.SolveInfo()
    st = L.load().bicgstab_solve_mixed(pattern.handle, C.byref(bsr), _dev(vals32, torch.float32, "vals32"),
                                       _dev(factors32, torch.float32, "factors32"), _dev(rhs, torch.float64, "rhs"),
                                       _dev(x, torch.float64, "x"), tol, maxit, inner_tol, inner_maxit,
                                       _dev(work, torch.uint8, "work"), work.numel(), _stream_handle(stream),
                                       C.byref(info))
    if st in (L.BILU_ERR_ARG, L.BILU_ERR_STATE, L.BILU_ERR_CUDA, L.BILU_ERR_OOM):
        _check(st, "bicgstab_solve_mixed")
    return x, info


# ---- tuning / test hooks ----

def bilu_set_trisolve_chunk(rows: int):
    _check(L.load().bilu_set_trisolve_chunk(rows), "bilu_set_trisolve_chunk")


def bilu_set_trisolve_warps(warps: int):
    _check(L.load().bilu_set_trisolve_warps(warps), "bilu_set_trisolve_warps")


def bilu_set_trisolve_ctas_per_sm(ctas: int):
    _check(L.load().bilu_set_trisolve_ctas_per_sm(ctas), "bilu_set_trisolve_ctas_per_sm")


def bilu_get_trisolve_chunk() -> int:
    return int(L.load().bilu_get_trisolve_chunk())


def bilu_auto_trisolve_chunk(P: "Pattern") -> int:
    """The chunk target the solves use for P when none is set."""
    return int(L.load().bilu_auto_trisolve_chunk(P.handle))


def bilu_auto_factor_chunk(P: "Pattern") -> int:
    """The chunk target the factorization uses for P when none is set."""
    return int(L.load().bilu_auto_factor_chunk(P.handle))


def bilu_set_factor_chunk(rows: int):
    _check(L.load().bilu_set_factor_chunk(rows), "bilu_set_factor_chunk")


def bilu_get_factor_chunk() -> int:
    return int(L.load().bilu_get_factor_chunk())


def bilu_set_spin_limit_ns(ns: int):
    _check(L.load().bilu_set_spin_limit_ns(ns), "bilu_set_spin_limit_ns")


def bilu_set_check_every(iters: int):
    _check(L.load().bilu_set_check_every(iters), "bilu_set_check_every")


def bilu_test_withhold_row(row: int):
    _check(L.load().bilu_test_withhold_row(row), "bilu_test_withhold_row")


# ---- adjoint ----

def bilu_factor_transpose(pattern_t: Pattern, b: int, factors: torch.Tensor,
                          factors_t: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Factors of P'^T ([U'^T | D^-T | L^T]) from those of P'."""
    if factors_t is None:
        factors_t = torch.empty_like(factors)
    _check(L.load().bilu_factor_transpose(pattern_t.handle, b, _dev(factors, torch.float64, "factors"),
                                          _dev(factors_t, torch.float64, "factors_t"), _stream_handle(stream)),
           "bilu_factor_transpose")
    return factors_t


def bsr_transpose_pattern(n: int, row_ptr, col_idx):
    """(row_ptr_t, col_idx_t, perm) of A^T on the host (bsr_transpose_pattern)."""
    rp = _host_i32(row_ptr)
    ci = _host_i32(col_idx)
    nnz = int(rp[n]) if n > 0 else 0
    rpt = np.zeros(n + 1, np.int32)
    cit = np.zeros(max(nnz, 1), np.int32)
    perm = np.zeros(max(nnz, 1), np.int32)
    p = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    _check(L.load().bsr_transpose_pattern(n, p(rp), p(ci), p(rpt), p(cit), p(perm)), "bsr_transpose_pattern")
    return rpt, cit[:nnz], perm[:nnz]


def bsr_gather_transpose(b: int, perm: torch.Tensor, src: torch.Tensor, dst: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """dst block t = (src block perm[t])^T on the device."""
    nblocks = perm.numel()
    if dst is None:
        dst = torch.empty(nblocks * b * b, dtype=torch.float64, device=src.device)
    _check(L.load().bsr_gather_transpose(nblocks, b, _dev(perm, torch.int32, "perm"),
                                         _dev(src, torch.float64, "src"), _dev(dst, torch.float64, "dst"),
                                         _stream_handle(stream)), "bsr_gather_transpose")
    return dst


def bsr_outer_grad(n: int, b: int, row_ptr: torch.Tensor, col_idx: torch.Tensor, lam: torch.Tensor,
                   x: torch.Tensor, grad: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """grad block (I, J) = -lambda_I x_J^T on A's block pattern."""
    if grad is None:
        grad = torch.empty(col_idx.numel() * b * b, dtype=torch.float64, device=x.device)
    _check(L.load().bsr_outer_grad(n, b, _dev(row_ptr, torch.int32, "row_ptr"),
                                   _dev(col_idx, torch.int32, "col_idx"), _dev(lam, torch.float64, "lambda"),
                                   _dev(x, torch.float64, "x"), _dev(grad, torch.float64, "grad"),
                                   _stream_handle(stream)), "bsr_outer_grad")
    return grad
