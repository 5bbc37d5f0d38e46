"""The device symbolic phase (bilu_symbolic_gpu) against the CPU oracle: P'
(Algorithm 3, Eq. 1-2), the level of fill of every entry and both Eq. 4
level sets must agree bit for bit with oracle.symbolic / oracle.levels, and
with the library's host phase."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1703_01325_gb300.reservoir import grid_pattern, random_pattern  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(libbilu):
    import paper_1703_01325_gb300.bilu as B
    torch.cuda.set_device(0)
    return B


def _oracle_pattern(n, rp, ci, k):
    prp, pci, plev = oracle.symbolic(n, rp, ci, k)
    lo, up = oracle.levels(n, prp, pci)
    return dict(row_ptr=prp, col_idx=pci, lev=plev, lvl_lower=lo, lvl_upper=up)


def _same(B, n, rp, ci, k, cap=256, host=True):
    P = B.bilu_symbolic_gpu(n, rp, ci, k, row_capacity=cap)
    g = P.export()
    o = _oracle_pattern(n, rp, ci, k)
    for key in ("row_ptr", "col_idx", "lev", "lvl_lower", "lvl_upper"):
        assert np.array_equal(np.asarray(o[key], np.int32), g[key]), key
    info = P.info
    rows = np.repeat(np.arange(n), np.diff(o["row_ptr"]))
    assert info.nnz_p == len(o["col_idx"]) and info.nnz_a == rp[-1]
    assert info.nnz_l == int((o["col_idx"] < rows).sum()) and info.nnz_u == int((o["col_idx"] > rows).sum())
    assert info.nlev_l == (o["lvl_lower"].max() + 1 if n else 0)
    assert info.nlev_u == (o["lvl_upper"].max() + 1 if n else 0)
    if host:
        h = B.bilu_symbolic(n, rp, ci, k).export()
        for key in ("row_ptr", "col_idx", "lev", "lvl_lower", "lvl_upper"):
            assert np.array_equal(h[key], g[key]), key
    return P


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("k", [0, 1, 2, 3, 8])
def test_random_patterns(B, seed, k):
    n = 30 + 23 * seed
    rp, ci = random_pattern(n, density=3.0 / n + 0.01 * (seed % 3), seed=2000 + seed, symmetric=(seed % 2 == 0))
    _same(B, n, rp, ci, k, cap=n)


@pytest.mark.parametrize("grid", [(7, 5, 3), (16, 16, 8), (33, 9, 6)])
@pytest.mark.parametrize("stencil", [7, 27])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_grid_patterns(B, grid, stencil, k):
    rp, ci = grid_pattern(*grid, stencil)
    _same(B, int(np.prod(grid)), rp, ci, k)


def test_full_fill_and_empty(B):
    rp, ci = random_pattern(80, density=0.05, seed=77)
    _same(B, 80, rp, ci, 80, cap=80)
    P = B.bilu_symbolic_gpu(0, np.zeros(1, np.int32), np.zeros(0, np.int32), 1)
    assert P.info.n == 0 and P.info.nnz_p == 0


def test_capacity_and_pattern_errors(B):
    from paper_1703_01325_gb300 import _lib as L
    rp, ci = grid_pattern(8, 8, 4, 27)
    with pytest.raises(B.BiluError) as e:
        B.bilu_symbolic_gpu(256, rp, ci, 2, row_capacity=32)  # rows of P' hold far more than 32 blocks
    assert e.value.status == L.BILU_ERR_OOM
    _same(B, 256, rp, ci, 2, cap=512)  # the device is still usable
    with pytest.raises(B.BiluError) as e:
        B.bilu_symbolic_gpu(2, np.array([0, 1, 2]), np.array([0, 0]), 1)
    assert e.value.status == L.BILU_ERR_PATTERN
    with pytest.raises(B.BiluError) as e:
        B.bilu_symbolic_gpu(4, np.array([0, 1, 2, 3, 4]), np.arange(4), 1, row_capacity=0)
    assert e.value.status == L.BILU_ERR_ARG


def test_full_size_workload(B):
    """The 128 x 128 x 64 7-point pattern at ILU(1) (the bench workload)."""
    rp, ci = grid_pattern(128, 128, 64, 7)
    _same(B, 128 * 128 * 64, rp, ci, 1, cap=64, host=False)


def test_27pt_ilu2_workload(B):
    """A 64 x 64 x 32 27-point pattern at ILU(2): rows of P' up to 125 blocks,
    the fill structure of the 160 x 160 x 80 27-point ILU(2) case."""
    rp, ci = grid_pattern(64, 64, 32, 27)
    _same(B, 64 * 64 * 32, rp, ci, 2, cap=256, host=False)


@pytest.mark.parametrize("grid,stencil,k,b", [((13, 9, 6), 7, 1, 3), ((9, 8, 7), 27, 2, 2), ((40, 1, 1), 7, 0, 4)])
def test_device_pattern_factor_and_apply(B, grid, stencil, k, b):
    """A pattern completed on the device (L / U' split, Eq. 4 levels and the
    backfill map all built there) drives the factorization and the apply to
    the oracle's results; its upload builds the schedules without copying the
    structure again."""
    from paper_1703_01325_gb300.reservoir import reservoir_system
    from tests.gpu_util import TOL_APPLY, TOL_FACTOR, OracleRun, device_system, rel_maxerr
    S = reservoir_system(*grid, b, stencil=stencil, sigma=1.0, accum=0.01, seed=17)
    o = OracleRun(S.n, b, S.row_ptr, S.col_idx, S.vals, k)
    rp, ci, vals, rhs = device_system(S, "cuda:0")
    P = B.bilu_symbolic_gpu(S.n, S.row_ptr, S.col_idx, k, row_capacity=256).upload()
    H = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k)
    assert P.info.nlev_l == H.info.nlev_l and P.info.nlev_u == H.info.nlev_u
    assert B.bilu_auto_trisolve_chunk(P) == B.bilu_auto_trisolve_chunk(H)
    assert P.schedule(64)["ord_lower"].tolist() == H.schedule(64)["ord_lower"].tolist()
    F, info = B.bilu_factor(P, b, vals)
    assert info.status == 0
    Lg, Dg, Ug = (t.cpu().numpy() for t in B.factor_sections(P, b, F))
    assert rel_maxerr(Lg, o.L()) <= TOL_FACTOR
    assert rel_maxerr(Dg, o.Dinv) <= TOL_FACTOR
    assert rel_maxerr(Ug, o.U()) <= TOL_FACTOR
    x = B.bilu_apply(P, b, F, rhs)
    assert rel_maxerr(x.cpu().numpy(), o.apply(S.rhs)) <= TOL_APPLY


@pytest.mark.parametrize("grid,stencil,k,rows", [((16, 16, 8), 7, 1, 32), ((33, 9, 6), 27, 2, 64),
                                                 ((128, 128, 64), 7, 1, 256), ((24, 20, 10), 7, 0, 1024)])
def test_device_schedule_equals_host_schedule(B, grid, stencil, k, rows):
    """The schedule built for a pattern that lives on the device (per-row gaps,
    each chunk's local-level order, the chunk priorities and the predecessor
    lists on the device; cuts and list scheduling on the host from those) is
    the host builder's, bit for bit: chunk bounds, both row orders, both claim
    orders."""
    rp, ci = grid_pattern(*grid, stencil)
    n = int(np.prod(grid))
    g = B.bilu_symbolic_gpu(n, rp, ci, k, row_capacity=256).schedule(rows)
    h = B.bilu_symbolic(n, rp, ci, k).schedule(rows)
    for key in ("bounds", "ord_lower", "ord_upper", "tick_lower", "tick_upper"):
        assert np.array_equal(g[key], h[key]), key


def test_random_pattern_device_schedule(B):
    """Irregular patterns: many predecessor chunks per chunk."""
    for seed in range(3):
        n = 700 + 50 * seed
        rp, ci = random_pattern(n, density=0.006 + 0.002 * seed, seed=900 + seed, symmetric=seed == 1)
        for k in (0, 2):
            for rows in (7, 64):
                g = B.bilu_symbolic_gpu(n, rp, ci, k, row_capacity=n).schedule(rows)
                h = B.bilu_symbolic(n, rp, ci, k).schedule(rows)
                for key in ("bounds", "ord_lower", "ord_upper", "tick_lower", "tick_upper"):
                    assert np.array_equal(g[key], h[key]), (seed, k, rows, key)
