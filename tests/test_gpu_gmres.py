"""GPU parity of the restarted GMRES(m) solver (the solver of the paper's
experiments) against the CPU oracle's GMRES on the same seeded inputs: fixed
step counts (one cycle and across restarts) element by element, solves to a
tolerance, and the edge cases."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1703_01325_gb300.reservoir import random_pattern, reservoir_system  # noqa: E402
from tests.gpu_util import TOL_X, OracleRun, device_system  # noqa: E402
from tests.oracle_helpers import diag_dominant_block_values  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def B(libbilu):
    import paper_1703_01325_gb300.bilu as B
    torch.cuda.set_device(0)
    return B


def _setup(B, S, k):
    o = OracleRun(S.n, S.b, S.row_ptr, S.col_idx, S.vals, k)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
    F, info = B.bilu_factor(P, S.b, vals)
    assert info.status == 0
    return o, P, F, (S.n, S.b, rp, ci, vals), rhs


@pytest.mark.parametrize("steps,restart", [(1, 20), (7, 20), (20, 20), (23, 5), (40, 20)])
@pytest.mark.parametrize("b,k", [(3, 1), (2, 0)])
def test_gmres_fixed_steps_match_oracle(B, steps, restart, b, k):
    S = reservoir_system(16, 12, 8, b, sigma=2.0, accum=1e-3, seed=7 + b)
    o, P, F, A, rhs = _setup(B, S, k)
    x, info = B.gmres_solve(P, A, F, rhs, tol=1e-30, maxit=steps, restart=restart)
    xo, ito, rro, sto = oracle.gmres(S.n, b, S.row_ptr, S.col_idx, S.vals, o.prp, o.pci, o.F, o.Dinv, S.rhs,
                                     tol=1e-30, maxit=steps, restart=restart)
    assert info.iters == ito == steps and info.status == 5 and sto == oracle.ERR_NOT_CONVERGED
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= TOL_X * np.linalg.norm(xo)
    assert info.true_relres == pytest.approx(rro, rel=1e-6)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_gmres_converges_like_oracle(B, k):
    S = reservoir_system(16, 16, 8, 3, sigma=1.0, accum=0.01)
    o, P, F, A, rhs = _setup(B, S, k)
    x, info = B.gmres_solve(P, A, F, rhs, tol=1e-10, maxit=2000, restart=20)
    xo, ito, rro, sto = oracle.gmres(S.n, 3, S.row_ptr, S.col_idx, S.vals, o.prp, o.pci, o.F, o.Dinv, S.rhs,
                                     tol=1e-10, maxit=2000, restart=20)
    assert info.status == 0 and sto == oracle.OK
    assert info.true_relres <= 1e-10 and abs(info.iters - ito) <= 1
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= TOL_X * np.linalg.norm(xo)
    res = np.linalg.norm(S.rhs - o.spmv(xg)) / np.linalg.norm(S.rhs)
    assert res == pytest.approx(info.true_relres, rel=1e-6)


def test_gmres_edge_cases(B):
    S = reservoir_system(6, 5, 4, 3, sigma=1.0, accum=0.01)
    o, P, F, A, rhs = _setup(B, S, 0)
    x, info = B.gmres_solve(P, A, F, torch.zeros_like(rhs), x=torch.ones_like(rhs))
    assert info.status == 0 and info.iters == 0 and not x.any()
    x, info = B.gmres_solve(P, A, F, rhs, maxit=0)
    assert info.status == 5 and info.iters == 0 and not x.any()
    for bad in (0, 65):
        with pytest.raises(B.BiluError):
            B.gmres_solve(P, A, F, rhs, restart=bad)
    # a start vector that already solves the system: no step
    xs, _ = B.gmres_solve(P, A, F, rhs, tol=1e-12, maxit=500)
    x, info = B.gmres_solve(P, A, F, rhs, x=xs.clone(), tol=1e-8)
    assert info.status == 0 and info.iters == 0


def test_gmres_exact_preconditioner_one_step(B):
    n, b = 60, 2
    rp, ci = random_pattern(n, density=0.08, seed=11)
    vals = diag_dominant_block_values(n, b, rp, ci, seed=12)
    o = OracleRun(n, b, rp, ci, vals, n)
    P = B.bilu_symbolic(n, rp, ci, n).upload()
    dvals = torch.from_numpy(vals.reshape(-1)).to(DEV)
    F, _ = B.bilu_factor(P, b, dvals)
    A = (n, b, torch.from_numpy(rp).to(DEV), torch.from_numpy(ci).to(DEV), dvals)
    rhs = torch.linspace(1, 2, n * b, dtype=torch.float64, device=DEV)
    x, info = B.gmres_solve(P, A, F, rhs, tol=1e-12, maxit=10)
    assert info.status == 0 and info.iters == 1 and info.true_relres <= 1e-12


@pytest.mark.parametrize("solver", ["gmres", "bicgstab"])
def test_non_finite_operator_is_a_breakdown(B, solver):
    """A NaN in A makes every Krylov scalar non-finite: both solvers report a
    breakdown and x keeps its (finite) start value."""
    S = reservoir_system(6, 5, 4, 3, sigma=1.0, accum=0.01)
    o, P, F, A, rhs = _setup(B, S, 0)
    n, b, rp, ci, vals = A
    bad = vals.clone()
    bad[5] = float("nan")
    fn = B.gmres_solve if solver == "gmres" else B.bicgstab_solve
    x, info = fn(P, (n, b, rp, ci, bad), F, rhs, tol=1e-8, maxit=20)
    assert info.status == 4 and torch.isfinite(x).all()
