"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Sizes span many warps/chunks and ragged tails; the full
128 x 128 x 64 workload is compared as well (the oracle finishes it in
seconds except the solve, which is checked through its true residual)."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1703_01325_gb300.reservoir import (BlockSystem, random_block_values,  # noqa: E402
                                              random_pattern, reservoir_system)
from tests.gpu_util import (TOL_APPLY, TOL_FACTOR, TOL_SPMV, TOL_X, OracleRun,  # noqa: E402
                            device_system, rel_maxerr)

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def B(libbilu):
    import paper_1703_01325_gb300.bilu as B
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return B


def _random_system(n, b, density, seed, symmetric=False):
    rp, ci = random_pattern(n, density=density, seed=seed, symmetric=symmetric)
    vals = random_block_values(int(rp[-1]), b, seed=seed + 1)
    rows = np.repeat(np.arange(n), np.diff(rp))
    for t in np.nonzero(ci == rows)[0]:
        for q in range(b):
            vals[t, q * b + q] += 2.0 * b * (rp[rows[t] + 1] - rp[rows[t]])
    rhs = random_block_values(n, b, seed=seed + 2)[:, :b].reshape(-1).copy()
    return BlockSystem(n=n, b=b, row_ptr=rp, col_idx=ci, vals=vals, rhs=rhs)


def _check_factor_apply(B, S, k, chunks=(32, 1024), factor_chunks=(None,)):
    o = OracleRun(S.n, S.b, S.row_ptr, S.col_idx, S.vals, k)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
    old_f = B.bilu_get_factor_chunk()
    try:
        for fch in factor_chunks:
            if fch is not None:
                B.bilu_set_factor_chunk(fch)
                P.reschedule()  # chunk settings take effect at set-up only
            F, info = B.bilu_factor(P, S.b, vals)
            assert info.status == 0
            Lg, Dg, Ug = (t.cpu().numpy() for t in B.factor_sections(P, S.b, F))
            assert rel_maxerr(Lg, o.L()) <= TOL_FACTOR, fch
            assert rel_maxerr(Dg, o.Dinv) <= TOL_FACTOR, fch
            assert rel_maxerr(Ug, o.U()) <= TOL_FACTOR, fch
    finally:
        B.bilu_set_factor_chunk(old_f)
    xo = o.apply(S.rhs)
    old = B.bilu_get_trisolve_chunk()
    try:
        for ch in chunks:
            B.bilu_set_trisolve_chunk(ch)
            P.reschedule()
            assert P.schedule_info()["solve_rows"] == ch
            work = B.workspace(P.apply_workspace_bytes(S.b))
            x = B.bilu_apply(P, S.b, F, rhs, work=work)
            assert B.bilu_workspace_status(work) == 0
            assert rel_maxerr(x.cpu().numpy(), xo) <= TOL_APPLY, ch
    finally:
        B.bilu_set_trisolve_chunk(old)
    return P, F, o


@pytest.mark.parametrize("b", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("stencil", [7, 27])
def test_spmv(B, b, stencil):
    S = reservoir_system(11, 7, 5, b, stencil=stencil, seed=b)
    rp, ci, vals, _ = device_system(S, DEV)
    x = np.linspace(-1.0, 1.0, S.n * b)
    y = B.bsr_spmv(S.n, b, rp, ci, vals, torch.from_numpy(x).to(DEV))
    yo = oracle.spmv(S.n, b, S.row_ptr, S.col_idx, S.vals, x)
    assert rel_maxerr(y.cpu().numpy(), yo) <= TOL_SPMV


@pytest.mark.parametrize("b", [1, 2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_factor_apply_grid(B, b, k):
    S = reservoir_system(13, 9, 6, b, sigma=1.0, accum=0.01, seed=10 * b + k)
    _check_factor_apply(B, S, k, chunks=(1, 7, 32, 1024) if b in (1, 3, 8) else (32, 1024),
                        factor_chunks=(1, 7, 512, 1024) if b in (1, 3, 8) else (None,))


@pytest.mark.parametrize("k", [0, 1, 3])
def test_factor_apply_27pt(B, k):
    S = reservoir_system(9, 8, 7, 3, stencil=27, sigma=1.5, accum=1e-3, seed=5 + k)
    _check_factor_apply(B, S, k, chunks=(1, 32, 100), factor_chunks=(3, 100, 1024))


@pytest.mark.parametrize("b", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("dims,k,width", [((300, 1, 1), 0, 1), ((17, 13, 1), 0, 2), ((9, 8, 6), 0, 3),
                                          ((9, 8, 6), 1, 6)])
def test_apply_row_widths(B, b, dims, k, width):
    """Rows of at most 1, 2, 3 and 6 blocks in L and in U' (a chain, a 5-point
    plane, a 7-point grid at ILU(0) and ILU(1)).  Each solve spreads a row over
    the fewest block groups that hold it in one pass, so these widths run
    every group count of every b; FP64 and FP32 applies against the oracle."""
    S = reservoir_system(*dims, b, sigma=1.0, accum=0.01, seed=7 * b + width)
    o = OracleRun(S.n, b, S.row_ptr, S.col_idx, S.vals, k)
    rows = np.repeat(np.arange(S.n), np.diff(o.prp))
    assert np.bincount(rows[o.lower], minlength=S.n).max() == width
    assert np.bincount(rows[o.upper], minlength=S.n).max() == width
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
    F, info = B.bilu_factor(P, b, vals)
    assert info.status == 0
    old = B.bilu_get_trisolve_chunk()
    try:
        for ch in (1, 32):
            B.bilu_set_trisolve_chunk(ch)
            P.reschedule()
            x = B.bilu_apply(P, b, F, rhs).cpu().numpy()
            assert rel_maxerr(x, o.apply(S.rhs)) <= TOL_APPLY, ch
            x32 = B.bilu_apply_f32(P, b, B.bilu_convert_f32(F), rhs).cpu().numpy()
            xo32 = oracle.apply(S.n, b, o.prp, o.pci, o.F.astype(np.float32).astype(np.float64),
                                o.Dinv.astype(np.float32).astype(np.float64),
                                S.rhs.astype(np.float32).astype(np.float64))
            assert rel_maxerr(x32, xo32) <= 1e-4, ch  # FP32 arithmetic, as in the mixed-precision tests
    finally:
        B.bilu_set_trisolve_chunk(old)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("b", [2, 3, 7])
def test_factor_apply_random_nonsymmetric(B, seed, b):
    S = _random_system(300 + 37 * seed, b, density=0.01 + 0.004 * seed, seed=50 + seed)
    _check_factor_apply(B, S, seed % 3, chunks=(1, 16, 64), factor_chunks=(1, 64, 512))


def test_long_rows_full_fill(B):
    """Arrow pattern at k = 1 fills completely: rows of 150 blocks exercise
    the multi-pass loops of the solves and of the factor's update batches."""
    n, b = 150, 2
    rows = [list(range(n))] + [[0, i] for i in range(1, n)]
    rp = np.array([0] + list(np.cumsum([len(r) for r in rows])), np.int32)
    ci = np.array([c for r in rows for c in r], np.int32)
    vals = random_block_values(int(rp[-1]), b, seed=9)
    for i in range(n):
        t = rp[i] + (i if i == 0 else 1)
        for q in range(b):
            vals[t, q * b + q] += 4.0 * n
    rhs = random_block_values(n, b, seed=10)[:, :b].reshape(-1).copy()
    S = BlockSystem(n=n, b=b, row_ptr=rp, col_idx=ci, vals=vals, rhs=rhs)
    P, F, o = _check_factor_apply(B, S, 1, chunks=(1, 32))
    assert P.info.nnz_p == n * n


def test_long_chain_b1(B):
    """Scalar tridiagonal system: one dependency chain through all 20000 rows."""
    n = 20000
    rp = [0]
    cols = []
    for i in range(n):
        cols += [j for j in (i - 1, i, i + 1) if 0 <= j < n]
        rp.append(len(cols))
    rp, ci = np.array(rp, np.int32), np.array(cols, np.int32)
    rows = np.repeat(np.arange(n), np.diff(rp))
    vals = np.where(ci == rows, 4.0, -1.0)[:, None] + 0.1 * random_block_values(len(ci), 1, seed=3)
    rhs = random_block_values(n, 1, seed=4)[:, 0].copy()
    S = BlockSystem(n=n, b=1, row_ptr=rp, col_idx=ci, vals=vals, rhs=rhs)
    _check_factor_apply(B, S, 0, chunks=(1, 32, 1000, 1024))


def test_single_row_and_block_diagonal(B):
    for n, b in ((1, 3), (257, 5)):
        rp = np.arange(n + 1, dtype=np.int32)
        ci = np.arange(n, dtype=np.int32)
        vals = random_block_values(n, b, seed=n)
        for q in range(b):
            vals[:, q * b + q] += 3.0
        rhs = random_block_values(n, b, seed=n + 1)[:, :b].reshape(-1).copy()
        S = BlockSystem(n=n, b=b, row_ptr=rp, col_idx=ci, vals=vals, rhs=rhs)
        P, F, o = _check_factor_apply(B, S, 2)
        assert P.info.nnz_l == 0 and P.info.nnz_u == 0


def test_empty_system(B):
    P = B.bilu_symbolic(0, np.zeros(1, np.int32), np.zeros(0, np.int32), 1).upload()
    F, info = B.bilu_factor(P, 3, torch.zeros(1, dtype=torch.float64, device=DEV))
    assert info.status == 0


def test_singular_pivot_reported(B):
    S = reservoir_system(6, 5, 4, 3, seed=1)
    bad = 37
    vals = S.vals.copy()
    t = [u for u in range(S.row_ptr[bad], S.row_ptr[bad + 1]) if S.col_idx[u] == bad][0]
    prp, pci, _ = oracle.symbolic(S.n, S.row_ptr, S.col_idx, 0)
    # make the factored pivot of row `bad` exactly singular: zero the row's
    # lower blocks and its diagonal block
    for u in range(S.row_ptr[bad], S.row_ptr[bad + 1]):
        if S.col_idx[u] <= bad:
            vals[u] = 0.0
    with pytest.raises(oracle.OracleError) as e:
        oracle.factor(S.n, 3, prp, pci, oracle.backfill(S.n, 3, S.row_ptr, S.col_idx, vals, prp, pci))
    assert e.value.row == bad
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, 0).upload()
    dv = torch.from_numpy(vals.reshape(-1)).to(DEV)
    with pytest.raises(B.BiluError) as e2:
        B.bilu_factor(P, 3, dv)
    assert e2.value.status == 3
    _, info = B.bilu_factor(P, 3, dv, check=False)
    assert info.status == 3 and info.bad_row == bad
    assert t >= 0


def test_dependency_wait_times_out_and_recovers(B):
    """A withheld row makes its dependents' bounded waits run out: the apply
    reports BILU_ERR_TIMEOUT and the context stays usable."""
    S = reservoir_system(10, 8, 6, 3, seed=2)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, 1).upload()
    rp, ci, vals, rhs = device_system(S, DEV)
    F, _ = B.bilu_factor(P, 3, vals)
    work = B.workspace(P.apply_workspace_bytes(3))
    old_chunk = B.bilu_get_trisolve_chunk()
    B.bilu_set_trisolve_chunk(16)  # row 5's dependent 5 + 80 lies in another chunk
    P.reschedule()
    B.bilu_set_spin_limit_ns(20_000_000)
    B.bilu_test_withhold_row(5)
    try:
        B.bilu_apply(P, 3, F, rhs, work=work)
        assert B.bilu_workspace_status(work) == 6
    finally:
        B.bilu_test_withhold_row(-1)
        B.bilu_set_spin_limit_ns(2_000_000_000)
        B.bilu_set_trisolve_chunk(old_chunk)
    work2 = B.workspace(P.apply_workspace_bytes(3))
    x = B.bilu_apply(P, 3, F, rhs, work=work2)
    assert B.bilu_workspace_status(work2) == 0
    o = OracleRun(S.n, 3, S.row_ptr, S.col_idx, S.vals, 1)
    assert rel_maxerr(x.cpu().numpy(), o.apply(S.rhs)) <= TOL_APPLY


@pytest.mark.parametrize("k", [0, 1])
def test_bicgstab_small_workload(B, k):
    """16 x 16 x 8 cells, b = 3: both solvers reach 1e-8; with tol 1e-12 the
    solutions agree to 1e-8 relative."""
    S = reservoir_system(16, 16, 8, 3, sigma=1.0, accum=0.01)
    o = OracleRun(S.n, 3, S.row_ptr, S.col_idx, S.vals, k)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
    F, _ = B.bilu_factor(P, 3, vals)
    A = (S.n, 3, rp, ci, vals)
    x, info = B.bicgstab_solve(P, A, F, rhs, tol=1e-8, maxit=1000)
    xo, ito, rro, sto = oracle.bicgstab(S.n, 3, S.row_ptr, S.col_idx, S.vals, o.prp, o.pci, o.F, o.Dinv,
                                        S.rhs, tol=1e-8, maxit=1000)
    assert info.status == 0 and sto == 0
    assert info.true_relres <= 1e-8 and rro <= 1e-8
    # BiCGSTAB's iteration count is not a continuous function of rounding: the
    # oracle's own count moves by several iterations (57..61 at k = 0) when the
    # rhs is perturbed at 1e-15 relative.  The GPU count, whose sums round in a
    # different order, must lie within that spread, widened by 2.
    its = [ito]
    for seed in range(1, 7):
        pert = S.rhs * (1.0 + 1e-15 * np.random.default_rng(seed).standard_normal(S.rhs.shape))
        its.append(oracle.bicgstab(S.n, 3, S.row_ptr, S.col_idx, S.vals, o.prp, o.pci, o.F, o.Dinv,
                                   pert, tol=1e-8, maxit=1000)[1])
    assert min(its) - 2 <= info.iters <= max(its) + 2, (info.iters, its)
    # the reported residual is the true one: recompute it with the oracle's SpMV
    xg = x.cpu().numpy()
    res = np.linalg.norm(S.rhs - oracle.spmv(S.n, 3, S.row_ptr, S.col_idx, S.vals, xg)) / np.linalg.norm(S.rhs)
    assert res == pytest.approx(info.true_relres, rel=1e-6, abs=1e-15)
    x12, info12 = B.bicgstab_solve(P, A, F, rhs, tol=1e-12, maxit=1000)
    xo12, _, _, st12 = oracle.bicgstab(S.n, 3, S.row_ptr, S.col_idx, S.vals, o.prp, o.pci, o.F, o.Dinv,
                                       S.rhs, tol=1e-12, maxit=1000)
    assert info12.status == 0 and st12 == 0
    assert np.linalg.norm(x12.cpu().numpy() - xo12) <= TOL_X * np.linalg.norm(xo12)


def test_bicgstab_edge_cases(B):
    S = reservoir_system(6, 5, 4, 3, sigma=1.0, accum=0.01)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, 0).upload()
    F, _ = B.bilu_factor(P, 3, vals)
    A = (S.n, 3, rp, ci, vals)
    x, info = B.bicgstab_solve(P, A, F, torch.zeros_like(rhs), x=torch.ones_like(rhs), tol=1e-8, maxit=10)
    assert info.status == 0 and info.iters == 0 and not x.any()
    x, info = B.bicgstab_solve(P, A, F, rhs, tol=1e-30, maxit=3)
    assert info.status == 5 and info.iters == 3
    x, info = B.bicgstab_solve(P, A, F, rhs, tol=1e-8, maxit=0)
    assert info.status == 5 and info.iters == 0
    # warm start from the solution: converged at once
    x1, info1 = B.bicgstab_solve(P, A, F, rhs, tol=1e-8, maxit=100)
    x2, info2 = B.bicgstab_solve(P, A, F, rhs, x=x1.clone(), tol=1e-8, maxit=100)
    assert info2.status == 0 and info2.iters == 0


def test_bicgstab_exact_preconditioner(B):
    """Full fill makes M = A: one iteration solves the system, as in the oracle."""
    S = _random_system(40, 2, density=0.1, seed=123)
    o = OracleRun(S.n, 2, S.row_ptr, S.col_idx, S.vals, S.n)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, S.n).upload()
    F, _ = B.bilu_factor(P, 2, vals)
    x, info = B.bicgstab_solve(P, (S.n, 2, rp, ci, vals), F, rhs, tol=1e-12, maxit=10)
    xo, ito, _, _ = oracle.bicgstab(S.n, 2, S.row_ptr, S.col_idx, S.vals, o.prp, o.pci, o.F, o.Dinv,
                                    S.rhs, tol=1e-12, maxit=10)
    assert info.status == 0 and info.iters == ito == 1
    assert rel_maxerr(x.cpu().numpy(), xo) <= 1e-10


@pytest.fixture(scope="module")
def full_size(B):
    """The 128 x 128 x 64, b = 3, ILU(1) workload at full size."""
    S = reservoir_system(128, 128, 64, 3, sigma=2.0, accum=1e-3)
    o = OracleRun(S.n, 3, S.row_ptr, S.col_idx, S.vals, 1)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, 1).upload()
    F, info = B.bilu_factor(P, 3, vals)
    return S, o, P, F, (rp, ci, vals, rhs), info


def test_full_size_factor_apply_spmv(B, full_size):
    S, o, P, F, (rp, ci, vals, rhs), info = full_size
    assert info.status == 0
    Lg, Dg, Ug = (t.cpu().numpy() for t in B.factor_sections(P, 3, F))
    assert rel_maxerr(Lg, o.L()) <= TOL_FACTOR
    assert rel_maxerr(Dg, o.Dinv) <= TOL_FACTOR
    assert rel_maxerr(Ug, o.U()) <= TOL_FACTOR
    x = B.bilu_apply(P, 3, F, rhs)
    assert rel_maxerr(x.cpu().numpy(), o.apply(S.rhs)) <= TOL_APPLY
    y = B.bsr_spmv(S.n, 3, rp, ci, vals, rhs)
    assert rel_maxerr(y.cpu().numpy(), o.spmv(S.rhs)) <= TOL_SPMV


def test_full_size_solve_fixed_iterations(B, full_size):
    """At full size ILU(1)-BiCGSTAB does not reach 1e-8 on this workload
    (sigma = 2, accumulation 1e-3; the oracle stagnates as well), so the solve
    is compared after a fixed number of iterations: the GPU iterate matches the
    oracle's to 1e-8, and the reported true residual is the oracle SpMV's."""
    S, o, P, F, (rp, ci, vals, rhs), info = full_size
    A = (S.n, 3, rp, ci, vals)
    x, sinfo = B.bicgstab_solve(P, A, F, rhs, tol=1e-30, maxit=3)
    assert sinfo.status == 5 and sinfo.iters == 3
    xo, ito, rro, sto = oracle.bicgstab(S.n, 3, S.row_ptr, S.col_idx, S.vals, o.prp, o.pci, o.F, o.Dinv,
                                        S.rhs, tol=1e-30, maxit=3)
    assert sto == oracle.ERR_NOT_CONVERGED and ito == 3
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= TOL_X * np.linalg.norm(xo)
    res = np.linalg.norm(S.rhs - o.spmv(xg)) / np.linalg.norm(S.rhs)
    assert res == pytest.approx(sinfo.true_relres, rel=1e-6)
    assert rro == pytest.approx(sinfo.true_relres, rel=1e-6)
    # a longer run reports its outcome honestly (no convergence claimed)
    x, sinfo = B.bicgstab_solve(P, A, F, rhs, tol=1e-8, maxit=200)
    assert sinfo.status in (4, 5) and sinfo.true_relres > 1e-8
    res = np.linalg.norm(S.rhs - o.spmv(x.cpu().numpy())) / np.linalg.norm(S.rhs)
    assert res == pytest.approx(sinfo.true_relres, rel=1e-6)


def test_full_size_gmres_fixed_steps(B, full_size):
    """GMRES(20) at full size, 12 Arnoldi steps (one cycle, no restart) and
    25 steps (a restart after 20): the GPU iterate matches the oracle's to
    1e-8 and the reported true residual is the oracle SpMV's."""
    S, o, P, F, (rp, ci, vals, rhs), info = full_size
    A = (S.n, 3, rp, ci, vals)
    for steps in (12, 25):
        x, sinfo = B.gmres_solve(P, A, F, rhs, tol=1e-30, maxit=steps, restart=20)
        assert sinfo.status == 5 and sinfo.iters == steps
        xo, ito, rro, sto = oracle.gmres(S.n, 3, S.row_ptr, S.col_idx, S.vals, o.prp, o.pci, o.F, o.Dinv,
                                         S.rhs, tol=1e-30, maxit=steps, restart=20)
        assert sto == oracle.ERR_NOT_CONVERGED and ito == steps
        xg = x.cpu().numpy()
        assert np.linalg.norm(xg - xo) <= TOL_X * np.linalg.norm(xo)
        res = np.linalg.norm(S.rhs - o.spmv(xg)) / np.linalg.norm(S.rhs)
        assert res == pytest.approx(sinfo.true_relres, rel=1e-6)
        assert rro == pytest.approx(sinfo.true_relres, rel=1e-6)


@pytest.mark.parametrize("fp32", [False, True])
def test_apply_input_holding_the_pending_pattern(B, fp32):
    """A right-hand side entry that carries the solves' internal "pending" bit
    pattern (a signalling NaN) must not stall them: every computed value is
    stored as a quiet NaN instead, the apply completes with status 0 and the
    rows it reaches are NaN while the others match the clean apply."""
    S = reservoir_system(9, 7, 5, 3, sigma=1.0, accum=0.01, seed=3)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, 1).upload()
    F, _ = B.bilu_factor(P, 3, vals)
    Fa = B.bilu_convert_f32(F) if fp32 else F
    apply = B.bilu_apply_f32 if fp32 else B.bilu_apply
    bad = rhs.clone()
    bits = bad.view(torch.int64)
    bits[7 * 3 + 1] = 0x7FF4DEADBEEF0001
    work = B.workspace(P.apply_workspace_bytes(3))
    x = apply(P, 3, Fa, bad, work=work).cpu().numpy()
    assert B.bilu_workspace_status(work) == 0
    clean = apply(P, 3, Fa, rhs).cpu().numpy()
    nan = np.isnan(x)
    assert nan.any() and not np.isnan(clean).any()
    assert np.array_equal(x[~nan], clean[~nan])


def test_compute_calls_never_rebuild_the_schedule(B):
    """Chunk settings take effect at set-up (bilu_pattern_upload /
    bilu_pattern_schedule) only: an apply, a factorization and a solve after a
    new setting run on the existing schedule and leave it as it is; the next
    bilu_pattern_schedule applies the setting.  Every schedule gives the
    oracle's x."""
    S = reservoir_system(12, 10, 6, 3, seed=4)
    o = OracleRun(S.n, 3, S.row_ptr, S.col_idx, S.vals, 1)
    rp, ci, vals, rhs = device_system(S, DEV)
    old_t, old_f = B.bilu_get_trisolve_chunk(), B.bilu_get_factor_chunk()
    try:
        B.bilu_set_trisolve_chunk(40)
        B.bilu_set_factor_chunk(60)
        P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, 1).upload()
        assert P.schedule_info() == {"solve_rows": 40, "factor_rows": 60}
        B.bilu_set_trisolve_chunk(13)
        B.bilu_set_factor_chunk(17)
        F, info = B.bilu_factor(P, 3, vals)
        x = B.bilu_apply(P, 3, F, rhs)
        _, si = B.bicgstab_solve(P, (S.n, 3, rp, ci, vals), F, rhs, tol=1e-10, maxit=300)
        assert info.status == 0 and si.status == 0
        assert P.schedule_info() == {"solve_rows": 40, "factor_rows": 60}
        assert rel_maxerr(x.cpu().numpy(), o.apply(S.rhs)) <= TOL_APPLY
        P.reschedule()
        assert P.schedule_info() == {"solve_rows": 13, "factor_rows": 17}
        F2, _ = B.bilu_factor(P, 3, vals)
        assert rel_maxerr(B.bilu_apply(P, 3, F2, rhs).cpu().numpy(), o.apply(S.rhs)) <= TOL_APPLY
    finally:
        B.bilu_set_trisolve_chunk(old_t)
        B.bilu_set_factor_chunk(old_f)


def test_compute_calls_need_an_uploaded_pattern(B):
    S = reservoir_system(6, 5, 4, 3, seed=1)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, 1)
    assert P.schedule_info() == {"solve_rows": 0, "factor_rows": 0}
    from paper_1703_01325_gb300 import _lib as L
    with pytest.raises(B.BiluError) as e:
        B.bilu_factor(P, 3, vals)
    assert e.value.status == L.BILU_ERR_STATE


@pytest.mark.parametrize("b", [2, 3, 8])
def test_apply_is_independent_of_residency(B, b):
    """The solves' result does not depend on how many CTAs share the chunks
    (each row's sum runs in a fixed order): FP64 and FP32 applies with one
    resident CTA per SM equal the default grid's bit for bit, and the oracle's
    x.  b = 2 prefetches two rows ahead, b = 3 and 8 one row ahead in FP64."""
    S = reservoir_system(20, 14, 9, b, seed=30 + b)
    o = OracleRun(S.n, b, S.row_ptr, S.col_idx, S.vals, 1)
    _, _, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, 1).upload()
    F, _ = B.bilu_factor(P, b, vals)
    F32 = B.bilu_convert_f32(F)
    x64 = B.bilu_apply(P, b, F, rhs).cpu().numpy()
    x32 = B.bilu_apply_f32(P, b, F32, rhs).cpu().numpy()
    try:
        B.bilu_set_trisolve_ctas_per_sm(1)
        y64 = B.bilu_apply(P, b, F, rhs).cpu().numpy()
        y32 = B.bilu_apply_f32(P, b, F32, rhs).cpu().numpy()
    finally:
        B.bilu_set_trisolve_ctas_per_sm(0)
    assert np.array_equal(x64.view(np.int64), y64.view(np.int64))
    assert np.array_equal(x32.view(np.int64), y32.view(np.int64))
    assert rel_maxerr(x64, o.apply(S.rhs)) <= TOL_APPLY
