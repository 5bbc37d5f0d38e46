"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test computes the expected value by a route other than the oracle's
(dense Algorithm 2 bookkeeping, the fill-path theorem, hand-worked fixtures,
closed forms, ILU's defining property, dense LU and numpy solves), chosen so
that a dropped term, a wrong sign or index or a transposed operand in the
oracle fails at least one of them.  CPU only.
"""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1703_01325_gb300.reservoir import (grid_pattern, random_block_values, random_pattern,
                                              reservoir_system)
from tests.oracle_helpers import (block, dense_levels_alg2, diag_dominant_block_values,
                                  fill_path_levels, pattern_set, split_factors,
                                  symbolic_full_fill, to_dense)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def sym_dict(n, rp, ci, k):
    prp, pci, plev = oracle.symbolic(n, rp, ci, k)
    return {(i, int(pci[t])): int(plev[t]) for i in range(n) for t in range(prp[i], prp[i + 1])}, (prp, pci, plev)


# ----------------------------------------------------------------------------
# Symbolic phase (Algorithm 3, Eq. 1-2)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_symbolic_matches_dense_algorithm2(seed, k):
    n = 8 + (seed * 7) % 30
    rp, ci = random_pattern(n, density=0.12 + 0.02 * (seed % 4), seed=seed, symmetric=(seed % 3 == 0))
    got, _ = sym_dict(n, rp, ci, k)
    assert got == dense_levels_alg2(n, rp, ci, k, dropped_to_inf=True)
    # Dropped levels kept finite instead of infinite give the same pattern.
    assert got == dense_levels_alg2(n, rp, ci, k, dropped_to_inf=False)


@pytest.mark.parametrize("seed", range(10))
def test_symbolic_fill_path_theorem(seed):
    n = 10 + (seed * 5) % 20
    rp, ci = random_pattern(n, density=0.15, seed=100 + seed, symmetric=(seed % 2 == 0))
    fp = fill_path_levels(n, rp, ci)
    for k in (0, 1, 2, 4):
        got, _ = sym_dict(n, rp, ci, k)
        expect = {key: lv for key, lv in fp.items() if lv <= k}
        assert got == expect


def test_symbolic_k0_is_pattern_of_A():
    rp, ci = grid_pattern(5, 4, 3, 7)
    n = 60
    prp, pci, plev = oracle.symbolic(n, rp, ci, 0)
    assert np.array_equal(prp, rp) and np.array_equal(pci, ci) and not plev.any()


@pytest.mark.parametrize("seed", range(6))
def test_symbolic_full_fill_for_large_k(seed):
    n = 12 + 3 * seed
    rp, ci = random_pattern(n, density=0.1, seed=200 + seed)
    got, _ = sym_dict(n, rp, ci, n)
    assert set(got) == symbolic_full_fill(n, rp, ci)


@pytest.mark.parametrize("k", [0, 1, 2, 5, 50])
def test_symbolic_tridiagonal_has_no_fill(k):
    n = 40
    rows, cols = [], []
    rp = [0]
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                cols.append(j)
        rp.append(len(cols))
    rp, ci = np.array(rp, np.int32), np.array(cols, np.int32)
    prp, pci, plev = oracle.symbolic(n, rp, ci, k)
    assert np.array_equal(prp, rp) and np.array_equal(pci, ci) and not plev.any()


@pytest.mark.parametrize("seed", range(5))
def test_symbolic_nested_in_k(seed):
    n = 30
    rp, ci = random_pattern(n, density=0.1, seed=300 + seed)
    prev = None
    for k in range(5):
        cur, _ = sym_dict(n, rp, ci, k)
        if prev is not None:
            assert set(prev) <= set(cur)
            assert all(cur[key] == prev[key] for key in prev)
        prev = cur


def _read_arrow():
    blocks, cur = {}, None
    for line in open(os.path.join(GOLDEN, "arrow5_levels.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("k="):
            cur = int(line[2:])
            blocks[cur] = []
            continue
        blocks[cur].append({int(a): int(b) for a, b in (e.split(":") for e in line.split())})
    return blocks


def test_symbolic_golden_arrow():
    n = 5
    rows = [list(range(5))] + [[0, i] for i in range(1, 5)]
    rp = np.array([0] + list(np.cumsum([len(r) for r in rows])), np.int32)
    ci = np.array([c for r in rows for c in r], np.int32)
    for k, expect_rows in _read_arrow().items():
        got, _ = sym_dict(n, rp, ci, k)
        expect = {(i, j): lv for i, row in enumerate(expect_rows) for j, lv in row.items()}
        assert got == expect


def test_symbolic_golden_stencil7_k1():
    nx, ny, nz = 7, 6, 5
    rp, ci = grid_pattern(nx, ny, nz, 7)
    n = nx * ny * nz
    prp, pci, plev = oracle.symbolic(n, rp, ci, 1)
    rows = []
    for line in open(os.path.join(GOLDEN, "stencil7_k1_interior_row.txt")):
        if line.strip() and not line.startswith("#"):
            dz, dy, dx, lv = map(int, line.split())
            rows.append((dx + nx * dy + nx * ny * dz, lv))
    checked = 0
    for z in range(1, nz - 1):
        for y in range(1, ny - 1):
            for x in range(1, nx - 1):
                i = x + nx * (y + ny * z)
                got = [(int(pci[t]) - i, int(plev[t])) for t in range(prp[i], prp[i + 1])]
                assert got == rows
                checked += 1
    assert checked == (nx - 2) * (ny - 2) * (nz - 2)


def test_symbolic_rejects_bad_patterns():
    rp = np.array([0, 1, 2], np.int32)
    assert oracle.check_pattern(2, rp, np.array([0, 0], np.int32)) == oracle.ERR_PATTERN  # no diag row 1
    assert oracle.check_pattern(2, np.array([0, 2, 3], np.int32), np.array([1, 0, 1], np.int32)) == oracle.ERR_PATTERN
    assert oracle.check_pattern(2, np.array([0, 2, 3], np.int32), np.array([0, 0, 1], np.int32)) == oracle.ERR_PATTERN
    assert oracle.check_pattern(2, np.array([0, 1, 2], np.int32), np.array([0, 2], np.int32)) == oracle.ERR_PATTERN
    with pytest.raises(oracle.OracleError):
        oracle.symbolic(2, rp, np.array([0, 0], np.int32), 1)


# ----------------------------------------------------------------------------
# Dependency levels (Eq. 4)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_levels_characterisation(seed):
    """Every dependency sits in a strictly lower level and every row at level
    l > 0 has a dependency at level l - 1: that fixes the longest-path levels."""
    n = 60
    rp, ci = random_pattern(n, density=0.06, seed=400 + seed)
    prp, pci, _ = oracle.symbolic(n, rp, ci, seed % 3)
    lo, up = oracle.levels(n, prp, pci)
    for i in range(n):
        cols = pci[prp[i]:prp[i + 1]]
        low = [lo[j] for j in cols if j < i]
        high = [up[j] for j in cols if j > i]
        assert all(l < lo[i] for l in low)
        assert (lo[i] == 0) == (len(low) == 0)
        if low:
            assert max(low) == lo[i] - 1
        assert all(l < up[i] for l in high)
        if high:
            assert max(high) == up[i] - 1
        else:
            assert up[i] == 0


def test_levels_closed_form_7pt_k0():
    nx, ny, nz = 9, 7, 5
    rp, ci = grid_pattern(nx, ny, nz, 7)
    n = nx * ny * nz
    lo, up = oracle.levels(n, rp, ci)
    c = np.arange(n)
    x, y, z = c % nx, (c // nx) % ny, c // (nx * ny)
    assert np.array_equal(lo, x + y + z)
    assert np.array_equal(up, (nx - 1 - x) + (ny - 1 - y) + (nz - 1 - z))
    assert lo.max() + 1 == nx + ny + nz - 2


# ----------------------------------------------------------------------------
# Backfill (Algorithm 5) and factorisation (Algorithm 4, Eq. 5)
# ----------------------------------------------------------------------------

def test_backfill_copies_A_and_zeros_fills():
    S = reservoir_system(5, 4, 3, 2, sigma=1.0, accum=0.01)
    prp, pci, plev = oracle.symbolic(S.n, S.row_ptr, S.col_idx, 2)
    A1 = oracle.backfill(S.n, S.b, S.row_ptr, S.col_idx, S.vals, prp, pci)
    assert np.array_equal(to_dense(S.n, S.b, prp, pci, A1), to_dense(S.n, S.b, S.row_ptr, S.col_idx, S.vals))
    fills = plev > 0
    assert fills.any() and not A1[fills].any()


@pytest.mark.parametrize("b", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_factor_ilu_property_on_pattern(b, k):
    """(L D U')_ij = A'_ij for every (i, j) in P' (ILU's defining property)."""
    n = 24
    rp, ci = random_pattern(n, density=0.12, seed=500 + 7 * b + k)
    vals = diag_dominant_block_values(n, b, rp, ci, seed=b * 10 + k)
    prp, pci, _ = oracle.symbolic(n, rp, ci, k)
    A1 = oracle.backfill(n, b, rp, ci, vals, prp, pci)
    F, dinv = oracle.factor(n, b, prp, pci, A1)
    L, D, U = split_factors(n, b, prp, pci, F)
    M = L @ D @ U
    A = to_dense(n, b, rp, ci, vals)
    scale = np.abs(A).max()
    for (i, j) in pattern_set(n, prp, pci):
        si, sj = slice(i * b, (i + 1) * b), slice(j * b, (j + 1) * b)
        assert np.abs(M[si, sj] - A[si, sj]).max() <= 1e-12 * scale
    if k == 0:  # and the dropped fill is really missing somewhere
        assert np.abs(M - A).max() > 1e-6 * scale
    for i in range(n):
        t = [u for u in range(prp[i], prp[i + 1]) if pci[u] == i][0]
        assert np.allclose(block(dinv[i], b) @ block(F[t], b), np.eye(b), atol=1e-12)


@pytest.mark.parametrize("b", [1, 3, 4, 7])
def test_factor_full_fill_is_dense_block_lu(b):
    n = 14
    rp, ci = random_pattern(n, density=0.2, seed=600 + b)
    vals = diag_dominant_block_values(n, b, rp, ci, seed=b)
    prp, pci, _ = oracle.symbolic(n, rp, ci, n)
    A1 = oracle.backfill(n, b, rp, ci, vals, prp, pci)
    F, dinv = oracle.factor(n, b, prp, pci, A1)
    L, D, U = split_factors(n, b, prp, pci, F)
    A = to_dense(n, b, rp, ci, vals)
    assert np.abs(L @ D @ U - A).max() <= 1e-12 * np.abs(A).max()
    # and M^{-1} r = A^{-1} r
    r = random_block_values(n, b, seed=9)[:, 0] if b == 1 else random_block_values(n, b, seed=9)[:, :b].ravel()
    x = oracle.apply(n, b, prp, pci, F, dinv, r)
    assert np.allclose(x, np.linalg.solve(A, r), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("b", [1, 2, 3, 6])
def test_factor_block_tridiagonal_is_block_thomas(b):
    n = 12
    rp = [0]
    cols = []
    for i in range(n):
        cols += [j for j in (i - 1, i, i + 1) if 0 <= j < n]
        rp.append(len(cols))
    rp, ci = np.array(rp, np.int32), np.array(cols, np.int32)
    vals = diag_dominant_block_values(n, b, rp, ci, seed=700 + b, boost=3.0 * b)
    A = to_dense(n, b, rp, ci, vals)
    blk = lambda i, j: A[i * b:(i + 1) * b, j * b:(j + 1) * b]
    Dt = [blk(0, 0)]
    for i in range(1, n):
        Dt.append(blk(i, i) - blk(i, i - 1) @ np.linalg.solve(Dt[i - 1], blk(i - 1, i)))
    prp, pci, _ = oracle.symbolic(n, rp, ci, 0)
    F, dinv = oracle.factor(n, b, prp, pci, oracle.backfill(n, b, rp, ci, vals, prp, pci))
    for i in range(n):
        for t in range(prp[i], prp[i + 1]):
            j = pci[t]
            if j == i:
                expect = Dt[i]
            elif j == i - 1:
                expect = blk(i, i - 1) @ np.linalg.inv(Dt[i - 1])
            else:
                expect = np.linalg.solve(Dt[i], blk(i, i + 1))
            assert np.allclose(block(F[t], b), expect, rtol=1e-11, atol=1e-12)
        assert np.allclose(block(dinv[i], b), np.linalg.inv(Dt[i]), rtol=1e-11, atol=1e-12)


def test_factor_golden_tridiag():
    m = 8
    rp = [0]
    cols, vals = [], []
    for i in range(m):
        for j in (i - 1, i, i + 1):
            if 0 <= j < m:
                cols.append(j)
                vals.append(2.0 if i == j else -1.0)
        rp.append(len(cols))
    rp, ci = np.array(rp, np.int32), np.array(cols, np.int32)
    vals = np.array(vals)[:, None]
    prp, pci, _ = oracle.symbolic(m, rp, ci, 0)
    F, dinv = oracle.factor(m, 1, prp, pci, oracle.backfill(m, 1, rp, ci, vals, prp, pci))
    rows = [l.split() for l in open(os.path.join(GOLDEN, "tridiag8_ilu0.txt")) if l.strip() and not l.startswith("#")]
    for i, (idx, d, l) in enumerate(rows):
        assert int(idx) == i + 1
        tdiag = [t for t in range(prp[i], prp[i + 1]) if pci[t] == i][0]
        assert F[tdiag, 0] == pytest.approx(float(Fraction(d)), rel=1e-15)
        assert dinv[i, 0] == pytest.approx(1.0 / float(Fraction(d)), rel=1e-15)
        if l != "none":
            tl = [t for t in range(prp[i + 1], prp[i + 2]) if pci[t] == i][0]
            assert F[tl, 0] == pytest.approx(float(Fraction(l)), rel=1e-15)
            tu = [t for t in range(prp[i], prp[i + 1]) if pci[t] == i + 1][0]
            assert F[tu, 0] == pytest.approx(float(Fraction(l)), rel=1e-15)  # U' = D^-1 * (-1)


@pytest.mark.parametrize("b", [1, 2, 3, 5, 8])
def test_factor_block_diagonal(b):
    n = 9
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    vals = random_block_values(n, b, seed=800 + b)
    for q in range(b):
        vals[:, q * b + q] += 0.5 * b
    prp, pci, _ = oracle.symbolic(n, rp, ci, 3)
    F, dinv = oracle.factor(n, b, prp, pci, oracle.backfill(n, b, rp, ci, vals, prp, pci))
    assert len(pci) == n
    for i in range(n):
        assert np.allclose(block(dinv[i], b), np.linalg.inv(block(vals[i], b)), rtol=1e-12, atol=1e-13)
        assert np.array_equal(F[i], vals[i])


def test_factor_pivoting_inside_block():
    """A diagonal block with a zero (1,1) entry needs row pivoting inside the
    b x b inverse; the inverse must still be exact."""
    b = 3
    D = np.array([[0.0, 2.0, 1.0], [1.0, 0.0, 3.0], [4.0, 1.0, 0.0]])
    vals = D.T.reshape(1, 9)  # column-major storage
    rp, ci = np.array([0, 1], np.int32), np.array([0], np.int32)
    F, dinv = oracle.factor(1, b, rp, ci, vals)
    assert np.allclose(block(dinv[0], b), np.linalg.inv(D), rtol=1e-14, atol=1e-15)


def test_factor_reports_singular_row():
    b = 2
    n = 3
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    vals = np.tile(np.eye(2).T.ravel(), (n, 1))
    vals[1] = 0.0
    with pytest.raises(oracle.OracleError) as e:
        oracle.factor(n, b, rp, ci, vals)
    assert e.value.status == oracle.ERR_SINGULAR and e.value.row == 1
    vals[1] = np.eye(2).ravel()
    vals[2, 0] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.factor(n, b, rp, ci, vals)
    assert e.value.row == 2


# ----------------------------------------------------------------------------
# Apply (Eq. 6 / Algorithm 7), SpMV, BiCGSTAB
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("b", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_apply_inverts_LDU(b, k):
    S = reservoir_system(4, 3, 3, b, sigma=1.0, accum=0.01, seed=b + 10 * k)
    prp, pci, _ = oracle.symbolic(S.n, S.row_ptr, S.col_idx, k)
    F, dinv = oracle.factor(S.n, b, prp, pci, oracle.backfill(S.n, b, S.row_ptr, S.col_idx, S.vals, prp, pci))
    x = oracle.apply(S.n, b, prp, pci, F, dinv, S.rhs)
    L, D, U = split_factors(S.n, b, prp, pci, F)
    assert np.linalg.norm(L @ D @ U @ x - S.rhs) <= 1e-12 * np.linalg.norm(S.rhs) * np.linalg.cond(L @ D @ U)


@pytest.mark.parametrize("b", [1, 3, 8])
def test_spmv_dense(b):
    S = reservoir_system(5, 4, 3, b, stencil=27, seed=3)
    x = np.linspace(-1, 1, S.n * b)
    y = oracle.spmv(S.n, b, S.row_ptr, S.col_idx, S.vals, x)
    Ad = to_dense(S.n, b, S.row_ptr, S.col_idx, S.vals)
    assert np.allclose(y, Ad @ x, rtol=1e-13, atol=1e-13 * np.abs(Ad).max())


@pytest.mark.parametrize("k", [0, 1])
def test_bicgstab_solves_small_reservoir(k):
    S = reservoir_system(6, 5, 4, 3, sigma=1.0, accum=0.01)
    prp, pci, _ = oracle.symbolic(S.n, S.row_ptr, S.col_idx, k)
    F, dinv = oracle.factor(S.n, 3, prp, pci, oracle.backfill(S.n, 3, S.row_ptr, S.col_idx, S.vals, prp, pci))
    x, it, rr, st = oracle.bicgstab(S.n, 3, S.row_ptr, S.col_idx, S.vals, prp, pci, F, dinv, S.rhs,
                                    tol=1e-10, maxit=500)
    assert st == oracle.OK and rr <= 1e-10 and it > 0
    Ad = to_dense(S.n, 3, S.row_ptr, S.col_idx, S.vals)
    xd = np.linalg.solve(Ad, S.rhs)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.cond(Ad) * np.linalg.norm(xd)
    assert np.linalg.norm(Ad @ x - S.rhs) / np.linalg.norm(S.rhs) == pytest.approx(rr, rel=1e-6)


def test_bicgstab_exact_preconditioner_one_iteration():
    n, b = 10, 2
    rp, ci = random_pattern(n, density=0.3, seed=11)
    vals = diag_dominant_block_values(n, b, rp, ci, seed=12)
    prp, pci, _ = oracle.symbolic(n, rp, ci, n)
    F, dinv = oracle.factor(n, b, prp, pci, oracle.backfill(n, b, rp, ci, vals, prp, pci))
    rhs = np.linspace(1, 2, n * b)
    x, it, rr, st = oracle.bicgstab(n, b, rp, ci, vals, prp, pci, F, dinv, rhs, tol=1e-12, maxit=10)
    assert st == oracle.OK and it == 1 and rr <= 1e-12


def test_bicgstab_zero_rhs_and_maxit():
    S = reservoir_system(6, 5, 4, 3, sigma=1.0, accum=0.01)
    prp, pci, _ = oracle.symbolic(S.n, S.row_ptr, S.col_idx, 0)
    F, dinv = oracle.factor(S.n, 3, prp, pci, oracle.backfill(S.n, 3, S.row_ptr, S.col_idx, S.vals, prp, pci))
    x, it, rr, st = oracle.bicgstab(S.n, 3, S.row_ptr, S.col_idx, S.vals, prp, pci, F, dinv,
                                    np.zeros(S.n * 3), tol=1e-8, maxit=10)
    assert st == oracle.OK and it == 0 and not x.any()
    x, it, rr, st = oracle.bicgstab(S.n, 3, S.row_ptr, S.col_idx, S.vals, prp, pci, F, dinv, S.rhs,
                                    tol=1e-30, maxit=3)
    assert st == oracle.ERR_NOT_CONVERGED and it == 3


def test_bicgstab_first_step_properties():
    """One iteration from x0 = 0 must equal x1 = alpha p_hat + omega s_hat with
    alpha fixed by the BiCG condition (r_hat, s) = 0 and omega the minimiser of
    ||s - omega t|| (the local minimal-residual step), both computed here with
    dense numpy solves of M = L D U' and a least-squares fit."""
    S = reservoir_system(5, 4, 3, 2, sigma=1.0, accum=0.01, seed=21)
    prp, pci, _ = oracle.symbolic(S.n, S.row_ptr, S.col_idx, 0)
    F, dinv = oracle.factor(S.n, 2, prp, pci, oracle.backfill(S.n, 2, S.row_ptr, S.col_idx, S.vals, prp, pci))
    x1, it, rr, st = oracle.bicgstab(S.n, 2, S.row_ptr, S.col_idx, S.vals, prp, pci, F, dinv, S.rhs,
                                     tol=1e-30, maxit=1)
    assert it == 1 and st == oracle.ERR_NOT_CONVERGED
    L, D, U = split_factors(S.n, 2, prp, pci, F)
    M = L @ D @ U
    A = to_dense(S.n, 2, S.row_ptr, S.col_idx, S.vals)
    b = S.rhs
    p_hat = np.linalg.solve(M, b)
    v = A @ p_hat
    alpha = b @ b / (b @ v)
    s = b - alpha * v
    assert abs(b @ s) <= 1e-12 * np.linalg.norm(b) ** 2
    s_hat = np.linalg.solve(M, s)
    t = A @ s_hat
    omega = np.linalg.lstsq(t[:, None], s, rcond=None)[0][0]
    assert np.allclose(x1, alpha * p_hat + omega * s_hat, rtol=1e-10, atol=1e-12 * np.abs(x1).max())


# ----------------------------------------------------------------------------
# Restarted GMRES(m) (the solver of the paper's experiments, Section 4)
# ----------------------------------------------------------------------------

def _gmres_system(seed=31, b=2, k=0):
    S = reservoir_system(4, 4, 3, b, sigma=1.0, accum=0.01, seed=seed)
    prp, pci, _ = oracle.symbolic(S.n, S.row_ptr, S.col_idx, k)
    F, dinv = oracle.factor(S.n, b, prp, pci, oracle.backfill(S.n, b, S.row_ptr, S.col_idx, S.vals, prp, pci))
    L, D, U = split_factors(S.n, b, prp, pci, F)
    A = to_dense(S.n, b, S.row_ptr, S.col_idx, S.vals)
    return S, prp, pci, F, dinv, A, L @ D @ U


def _min_residual_point(A, Minv, x0, r0, j):
    """argmin ||b - A x|| over x0 + M^{-1} K_j(A M^{-1}, r0), by brute force:
    an orthonormal basis of the Krylov space (numpy QR) and least squares."""
    AM = A @ Minv
    K = np.empty((len(r0), j))
    v = r0.copy()
    for q in range(j):
        K[:, q] = v / np.linalg.norm(v)
        v = AM @ K[:, q]
    Q, _ = np.linalg.qr(K)
    c = np.linalg.lstsq(AM @ Q, r0, rcond=None)[0]
    return x0 + Minv @ (Q @ c)


@pytest.mark.parametrize("j", [1, 2, 4, 7])
def test_gmres_minimises_the_residual_over_the_krylov_space(j):
    """After j Arnoldi steps from x0 = 0 (no restart), x_j is the minimal
    residual point of x0 + M^{-1} K_j(A M^{-1}, b)."""
    S, prp, pci, F, dinv, A, M = _gmres_system()
    x, it, rr, st = oracle.gmres(S.n, S.b, S.row_ptr, S.col_idx, S.vals, prp, pci, F, dinv, S.rhs,
                                 tol=1e-30, maxit=j, restart=20)
    assert it == j and st == oracle.ERR_NOT_CONVERGED
    xm = _min_residual_point(A, np.linalg.inv(M), np.zeros_like(S.rhs), S.rhs, j)
    assert np.linalg.norm(x - xm) <= 1e-8 * np.linalg.norm(xm)
    assert np.linalg.norm(S.rhs - A @ x) / np.linalg.norm(S.rhs) == pytest.approx(rr, rel=1e-9)


def test_gmres_restart_starts_from_the_true_residual():
    """GMRES(3) with 5 steps: one full cycle (minimal residual over K_3), then a
    cycle of 2 steps from r_3 = b - A x_3."""
    S, prp, pci, F, dinv, A, M = _gmres_system(seed=32)
    Minv = np.linalg.inv(M)
    x, it, rr, st = oracle.gmres(S.n, S.b, S.row_ptr, S.col_idx, S.vals, prp, pci, F, dinv, S.rhs,
                                 tol=1e-30, maxit=5, restart=3)
    assert it == 5
    x3 = _min_residual_point(A, Minv, np.zeros_like(S.rhs), S.rhs, 3)
    x5 = _min_residual_point(A, Minv, x3, S.rhs - A @ x3, 2)
    assert np.linalg.norm(x - x5) <= 1e-8 * np.linalg.norm(x5)


@pytest.mark.parametrize("k", [0, 1])
def test_gmres_solves_small_reservoir(k):
    S = reservoir_system(6, 5, 4, 3, sigma=1.0, accum=0.01)
    prp, pci, _ = oracle.symbolic(S.n, S.row_ptr, S.col_idx, k)
    F, dinv = oracle.factor(S.n, 3, prp, pci, oracle.backfill(S.n, 3, S.row_ptr, S.col_idx, S.vals, prp, pci))
    x, it, rr, st = oracle.gmres(S.n, 3, S.row_ptr, S.col_idx, S.vals, prp, pci, F, dinv, S.rhs,
                                 tol=1e-10, maxit=2000, restart=20)
    assert st == oracle.OK and rr <= 1e-10 and it > 0
    Ad = to_dense(S.n, 3, S.row_ptr, S.col_idx, S.vals)
    xd = np.linalg.solve(Ad, S.rhs)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.cond(Ad) * np.linalg.norm(xd)
    assert np.linalg.norm(Ad @ x - S.rhs) / np.linalg.norm(S.rhs) == pytest.approx(rr, rel=1e-6)


def test_gmres_exact_preconditioner_one_step_and_edges():
    n, b = 10, 2
    rp, ci = random_pattern(n, density=0.3, seed=11)
    vals = diag_dominant_block_values(n, b, rp, ci, seed=12)
    prp, pci, _ = oracle.symbolic(n, rp, ci, n)
    F, dinv = oracle.factor(n, b, prp, pci, oracle.backfill(n, b, rp, ci, vals, prp, pci))
    rhs = np.linspace(1, 2, n * b)
    x, it, rr, st = oracle.gmres(n, b, rp, ci, vals, prp, pci, F, dinv, rhs, tol=1e-12, maxit=10)
    assert st == oracle.OK and it == 1 and rr <= 1e-12
    x, it, rr, st = oracle.gmres(n, b, rp, ci, vals, prp, pci, F, dinv, np.zeros(n * b), tol=1e-8, maxit=10)
    assert st == oracle.OK and it == 0 and not x.any()
    x, it, rr, st = oracle.gmres(n, b, rp, ci, vals, prp, pci, F, dinv, rhs, tol=1e-8, maxit=0)
    assert st == oracle.ERR_NOT_CONVERGED and it == 0 and not x.any()
