"""The C-ABI library loads and exports every function the public headers
declare (no compute calls: CPU only)."""
from __future__ import annotations

import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in ("bilu.h", "bilu_tuning.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(libbilu):
    from paper_1703_01325_gb300 import _lib
    names = declared_functions()
    assert len(names) >= 20
    for name in sorted(names):
        assert hasattr(libbilu, name), f"libbilu.so does not export {name}"
    assert names == set(_lib.SIGNATURES), names ^ set(_lib.SIGNATURES)


def test_library_is_sm103a_build():
    from paper_1703_01325_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_compute_calls_never_build_a_schedule(libbilu):
    """Schedules come from the set-up calls only (bilu_pattern_upload,
    bilu_pattern_schedule).  On a pattern that was never uploaded, a new chunk
    setting followed by factor, apply and solve calls leaves the pattern
    without schedules and every call returns BILU_ERR_STATE before touching a
    device (no CUDA call is made on this path, so it runs without a GPU)."""
    import ctypes as C

    import paper_1703_01325_gb300.bilu as B
    from paper_1703_01325_gb300 import _lib as L
    from paper_1703_01325_gb300.reservoir import grid_pattern
    rp, ci = grid_pattern(6, 5, 4, 7)
    P = B.bilu_symbolic(120, rp, ci, 1)
    lib = L.load()
    fake = C.c_void_p(0x1000)  # never dereferenced: the state check comes first
    old = B.bilu_get_trisolve_chunk()
    try:
        B.bilu_set_trisolve_chunk(17)
        assert P.schedule_info() == {"solve_rows": 0, "factor_rows": 0}
        assert lib.bilu_apply(P.handle, 3, fake, fake, C.c_void_p(0x2000), fake, 1 << 30, None) == L.BILU_ERR_STATE
        info = L.FactorInfo()
        assert lib.bilu_factor(P.handle, 3, fake, fake, fake, 1 << 30, None, C.byref(info)) == L.BILU_ERR_STATE
        bsr = L.BSR(120, 3, fake, fake, fake)
        si = L.SolveInfo()
        assert lib.bicgstab_solve(P.handle, C.byref(bsr), fake, fake, C.c_void_p(0x2000), 1e-8, 10, fake, 1 << 30,
                                  None, C.byref(si)) == L.BILU_ERR_STATE
        assert lib.bilu_pattern_schedule(P.handle, None) == L.BILU_ERR_STATE
        assert P.schedule_info() == {"solve_rows": 0, "factor_rows": 0}
    finally:
        B.bilu_set_trisolve_chunk(old)


def test_tuning_setters_and_spmv_reject_bad_arguments(libbilu):
    """Argument checks that run before any CUDA call: the solves' knobs take
    only their documented ranges, and the FP32 SpMV calls reject a bad block
    size, missing pointers and x aliasing y."""
    import ctypes as C

    from paper_1703_01325_gb300 import _lib as L
    lib = L.load()
    for bad in (-1, 33):
        assert lib.bilu_set_trisolve_ctas_per_sm(bad) == L.BILU_ERR_ARG
    for good in (0, 1, 32, 0):
        assert lib.bilu_set_trisolve_ctas_per_sm(good) == L.BILU_OK
    for bad in (2, 5, 32):
        assert lib.bilu_set_trisolve_warps(bad) == L.BILU_ERR_ARG
    assert lib.bilu_set_trisolve_warps(4) == L.BILU_OK
    p = C.c_void_p(0x1000)  # never dereferenced: the checks come first
    for fn in (lib.bsr_spmv_f32, lib.bsr_spmv_f32x):
        assert fn(10, 0, p, p, p, p, C.c_void_p(0x2000), None) == L.BILU_ERR_ARG
        assert fn(10, 9, p, p, p, p, C.c_void_p(0x2000), None) == L.BILU_ERR_ARG
        assert fn(-1, 3, p, p, p, p, C.c_void_p(0x2000), None) == L.BILU_ERR_ARG
        assert fn(10, 3, None, p, p, p, C.c_void_p(0x2000), None) == L.BILU_ERR_ARG
        assert fn(10, 3, p, p, p, C.c_void_p(0x3000), C.c_void_p(0x3000), None) == L.BILU_ERR_ARG
        assert fn(0, 3, p, p, p, p, C.c_void_p(0x2000), None) == L.BILU_OK  # nothing to do
