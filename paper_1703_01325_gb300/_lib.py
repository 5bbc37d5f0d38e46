"""ctypes binding of libbilu.so (the C ABI in include/bilu.h and
include/bilu_tuning.h).  Argument marshalling only: every step of the method
runs in the library's CUDA kernels (and its host symbolic phase).  There is no
fallback: a missing library raises at load time.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbilu.so")

BILU_OK = 0
BILU_ERR_ARG = 1
BILU_ERR_PATTERN = 2
BILU_ERR_SINGULAR = 3
BILU_ERR_BREAKDOWN = 4
BILU_ERR_NOT_CONVERGED = 5
BILU_ERR_TIMEOUT = 6
BILU_ERR_CUDA = 7
BILU_ERR_OOM = 8
BILU_ERR_STATE = 9


class PatternInfo(C.Structure):
    _fields_ = [("n", C.c_int32), ("k", C.c_int32), ("nnz_a", C.c_int64), ("nnz_p", C.c_int64),
                ("nnz_l", C.c_int64), ("nnz_u", C.c_int64), ("nlev_l", C.c_int32),
                ("nlev_u", C.c_int32)]


class FactorInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("bad_row", C.c_int32), ("ms", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("true_relres", C.c_double),
                ("ms", C.c_double)]


class BSR(C.Structure):
    _fields_ = [("n", C.c_int32), ("b", C.c_int32), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("vals", C.c_void_p)]


# Every symbol the two public headers declare, with its ctypes signature.
_i32p = C.POINTER(C.c_int32)
_vp = C.c_void_p
SIGNATURES = {
    "bilu_status_string": (C.c_char_p, [C.c_int]),
    "bilu_symbolic": (C.c_int, [C.c_int32, _i32p, _i32p, C.c_int32, C.POINTER(_vp)]),
    "bilu_pattern_query": (C.c_int, [_vp, C.POINTER(PatternInfo)]),
    "bilu_pattern_export": (C.c_int, [_vp, _i32p, _i32p, _i32p, _i32p, _i32p]),
    "bilu_pattern_upload": (C.c_int, [_vp, _vp]),
    "bilu_destroy_pattern": (None, [_vp]),
    "bilu_factor_bytes": (C.c_size_t, [_vp, C.c_int32]),
    "bilu_factor_workspace_bytes": (C.c_size_t, [_vp, C.c_int32]),
    "bilu_factor": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, C.c_size_t, _vp, C.POINTER(FactorInfo)]),
    "bilu_apply_workspace_bytes": (C.c_size_t, [_vp, C.c_int32]),
    "bilu_apply": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "bilu_workspace_status": (C.c_int, [_vp, _vp]),
    "bilu_apply_noalloc": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, _vp]),
    "bilu_apply_noalloc_status": (C.c_int, [_vp]),
    "bilu_pattern_schedule": (C.c_int, [_vp, _vp]),
    "bilu_pattern_schedule_info": (C.c_int, [_vp, _i32p, _i32p]),
    "bsr_spmv": (C.c_int, [C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "bicgstab_workspace_bytes": (C.c_size_t, [_vp, C.c_int32]),
    "bicgstab_solve": (C.c_int, [_vp, C.POINTER(BSR), _vp, _vp, _vp, C.c_double, C.c_int32, _vp,
                                 C.c_size_t, _vp, C.POINTER(SolveInfo)]),
    "bilu_factor_bytes_f32": (C.c_size_t, [_vp, C.c_int32]),
    "bilu_factor_f32": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, C.c_size_t, _vp, C.POINTER(FactorInfo)]),
    "bilu_convert_f32": (C.c_int, [_vp, _vp, C.c_int64, _vp]),
    "bilu_apply_f32": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "bsr_spmv_f32": (C.c_int, [C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "bsr_spmv_f32x": (C.c_int, [C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "bicgstab_mixed_workspace_bytes": (C.c_size_t, [_vp, C.c_int32]),
    "bicgstab_solve_mixed": (C.c_int, [_vp, C.POINTER(BSR), _vp, _vp, _vp, _vp, C.c_double, C.c_int32,
                                       C.c_double, C.c_int32, _vp, C.c_size_t, _vp, C.POINTER(SolveInfo)]),
    "bilu_set_trisolve_chunk": (C.c_int, [C.c_int32]),
    "bilu_get_trisolve_chunk": (C.c_int32, []),
    "bilu_set_trisolve_warps": (C.c_int, [C.c_int32]),
    "bilu_set_trisolve_ctas_per_sm": (C.c_int, [C.c_int32]),
    "bilu_auto_trisolve_chunk": (C.c_int32, [C.c_void_p]),
    "bilu_auto_factor_chunk": (C.c_int32, [C.c_void_p]),
    "bilu_set_factor_chunk": (C.c_int, [C.c_int32]),
    "bilu_get_factor_chunk": (C.c_int32, []),
    "bilu_set_spin_limit_ns": (C.c_int, [C.c_int64]),
    "bilu_set_check_every": (C.c_int, [C.c_int32]),
    "bilu_test_withhold_row": (C.c_int, [C.c_int32]),
    "bilu_profile_enable": (C.c_int, [C.c_int32]),
    "bilu_profile_read": (C.c_int, [C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "bilu_launch_count": (C.c_int64, []),
    "bilu_schedule_export": (C.c_int, [_vp, C.c_int32, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p]),
    "bicgstab_solve_f32prec": (C.c_int, [_vp, C.POINTER(BSR), _vp, _vp, _vp, C.c_double, C.c_int32, _vp,
                                         C.c_size_t, _vp, C.POINTER(SolveInfo)]),
    "gmres_workspace_bytes": (C.c_size_t, [_vp, C.c_int32, C.c_int32]),
    "gmres_solve": (C.c_int, [_vp, C.POINTER(BSR), _vp, _vp, _vp, C.c_double, C.c_int32, C.c_int32, _vp,
                              C.c_size_t, _vp, C.POINTER(SolveInfo)]),
    "bilu_symbolic_gpu": (C.c_int, [C.c_int32, _i32p, _i32p, C.c_int32, C.c_int32, _vp, C.POINTER(_vp)]),
    "bilu_pattern_transpose": (C.c_int, [_vp, C.POINTER(_vp)]),
    "bilu_factor_transpose": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp]),
    "bsr_transpose_pattern": (C.c_int, [C.c_int32, _i32p, _i32p, _i32p, _i32p, _i32p]),
    "bsr_gather_transpose": (C.c_int, [C.c_int64, C.c_int32, _vp, _vp, _vp, _vp]),
    "bsr_outer_grad": (C.c_int, [C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]),
}

PROF_KERNELS = ["spmv", "apply_prep", "lower_solve", "upper_solve", "backfill", "factor",
                "scale_upper", "krylov_vector", "factor_init", "adjoint", "symbolic", "diag_scale"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libbilu.so and attach signatures.  Raises if it is not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libbilu.so is not built ({path}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
