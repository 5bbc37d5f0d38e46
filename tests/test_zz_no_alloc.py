"""bilu_apply_noalloc: the preconditioner apply for callers that may not
allocate device memory (a host program that owns all device memory and gives
plugins none, or code that must avoid the synchronisation an allocation can
cause).  It must give the same x as bilu_apply, call after call, although its
scratch is one fixed array reused by every call.  This file is collected last
so that a run stopping at the first failure has run everything else first."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1703_01325_gb300.reservoir import reservoir_system  # noqa: E402
from tests.gpu_util import TOL_APPLY, device_system, rel_maxerr  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("grid,b,k", [((16, 16, 8), 3, 1), ((40, 30, 20), 4, 2)])
def test_noalloc_matches_workspace_apply(libbilu, grid, b, k):
    import paper_1703_01325_gb300.bilu as B
    torch.cuda.set_device(0)
    S = reservoir_system(*grid, b, sigma=1.0, accum=0.01, seed=7)
    rp, ci, vals, rhs = device_system(S, "cuda:0")
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
    F, info = B.bilu_factor(P, b, vals)
    assert info.status == 0
    x_ref = B.bilu_apply(P, b, F, rhs)
    r2 = torch.flip(rhs, [0]).contiguous()
    x_ref2 = B.bilu_apply(P, b, F, r2)
    torch.cuda.synchronize()
    # two calls in a row through the same fixed scratch, different inputs
    for r, ref in ((rhs, x_ref), (r2, x_ref2)):
        x = torch.full_like(rhs, float("nan"))
        assert B.bilu_apply_noalloc(P, b, F, r, x) == 0
        assert B.bilu_apply_noalloc_status() == 0
        torch.cuda.synchronize()
        assert rel_maxerr(x.cpu().numpy(), ref.cpu().numpy()) <= TOL_APPLY


def test_noalloc_reports_a_timed_out_wait(libbilu):
    """A wait that runs out inside bilu_apply_noalloc is reported by
    bilu_apply_noalloc_status (the test hook withholds one row of the lower
    solve, so its dependents' bounded waits run out); the next call starts
    from a clean error word and succeeds."""
    import paper_1703_01325_gb300.bilu as B
    torch.cuda.set_device(0)
    S = reservoir_system(10, 8, 6, 3, sigma=1.0, accum=0.01, seed=2)
    rp, ci, vals, rhs = device_system(S, "cuda:0")
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, 1).upload()
    F, _ = B.bilu_factor(P, 3, vals)
    x_ref = B.bilu_apply(P, 3, F, rhs)
    x = torch.empty_like(rhs)
    B.bilu_set_spin_limit_ns(20_000_000)
    B.bilu_test_withhold_row(5)
    try:
        assert B.bilu_apply_noalloc(P, 3, F, rhs, x) == 0
        assert B.bilu_apply_noalloc_status() == 6
    finally:
        B.bilu_test_withhold_row(-1)
        B.bilu_set_spin_limit_ns(2_000_000_000)
    assert B.bilu_apply_noalloc(P, 3, F, rhs, x) == 0
    assert B.bilu_apply_noalloc_status() == 0
    torch.cuda.synchronize()
    assert rel_maxerr(x.cpu().numpy(), x_ref.cpu().numpy()) <= TOL_APPLY


def test_noalloc_rejects_systems_beyond_the_fixed_scratch(libbilu):
    import paper_1703_01325_gb300.bilu as B
    from paper_1703_01325_gb300 import _lib as L
    torch.cuda.set_device(0)
    n, b = 600_000, 8          # n*b*8 bytes = 38.4 MB > 32 MiB
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    P = B.bilu_symbolic(n, rp, ci, 0).upload()
    F = torch.zeros(n * b * b, dtype=torch.float64, device="cuda:0")
    r = torch.zeros(n * b, dtype=torch.float64, device="cuda:0")
    x = torch.zeros_like(r)
    assert B.bilu_apply_noalloc(P, b, F, r, x) == L.BILU_ERR_STATE
