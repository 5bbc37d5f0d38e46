"""GPU parity of the mixed-precision calls (FP32-stored preconditioner and
SpMV, FP64 refinement) against the CPU oracle.

The FP32 kernels are compared with the oracle run on the same FP32-rounded
values (rounding done here with numpy), so what remains is FP32 arithmetic:
tolerances follow the standard bound |fl(sum) - sum| <= gamma_m sum|terms|
with gamma_m = m u / (1 - m u), u = 2^-24, m = terms in the sum."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1703_01325_gb300.reservoir import reservoir_system  # noqa: E402
from tests.gpu_util import OracleRun, device_system, rel_maxerr  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U32 = 2.0 ** -24


def gamma(m):
    return m * U32 / (1 - m * U32)


@pytest.fixture(scope="module")
def B(libbilu):
    import paper_1703_01325_gb300.bilu as B
    torch.cuda.set_device(0)
    return B


@pytest.mark.parametrize("b", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("stencil", [7, 27])
def test_spmv_f32(B, b, stencil):
    S = reservoir_system(11, 7, 5, b, stencil=stencil, seed=b)
    rp, ci, vals, _ = device_system(S, DEV)
    vals32 = B.bilu_convert_f32(vals)
    x = np.linspace(-1.0, 1.0, S.n * b)
    y = B.bsr_spmv_f32(S.n, b, rp, ci, vals32, torch.from_numpy(x).to(DEV)).cpu().numpy()
    v32 = S.vals.astype(np.float32).astype(np.float64)
    x32 = x.astype(np.float32).astype(np.float64)
    yo = oracle.spmv(S.n, b, S.row_ptr, S.col_idx, v32, x32)
    absy = oracle.spmv(S.n, b, S.row_ptr, S.col_idx, np.abs(v32), np.abs(x32))
    terms = stencil * b
    assert np.all(np.abs(y - yo) <= 2 * gamma(terms) * absy + 1e-300)


def test_convert_f32_rounds_to_nearest(B):
    """FP64 -> FP32 rounding to nearest even (IEEE 754, numpy's cast) on the
    integer path: exact ties both ways, the carry into the exponent, the
    overflow boundary, the smallest normal, subnormals, signed zeros, and
    random values over the whole float range."""
    edge = [1.0, 1.0 + 2.0 ** -30, np.pi, -1e-40, 3.4e38, 1e300, 0.0, -0.0,
            1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, 1 + 2.0 ** -24 + 2.0 ** -50, 1 - 2.0 ** -25,
            3.4028234663852886e38, 3.4028235677973362e38, 3.4028235677973366e38, 2.0 ** 127 * (2 - 2.0 ** -24),
            2.0 ** -126, 2.0 ** -126 * (1 - 2.0 ** -24), 2.0 ** -126 * (1 - 2.0 ** -25), -1e-45, -np.inf, np.inf]
    rng = np.random.default_rng(5)
    rand = rng.standard_normal(100000) * np.exp(rng.uniform(-90, 90, 100000))
    x = np.concatenate([np.array(edge), rand, [np.nan]])
    got = B.bilu_convert_f32(torch.from_numpy(x).to(DEV)).cpu().numpy()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    assert np.array_equal(got[:-1].view(np.uint32), ref[:-1].view(np.uint32)) and np.isnan(got[-1])


@pytest.mark.parametrize("b,k", [(3, 0), (3, 1), (4, 2), (8, 1)])
def test_apply_f32_matches_rounded_factors(B, b, k):
    S = reservoir_system(12, 9, 7, b, sigma=1.0, accum=0.01, seed=3 * b + k)
    o = OracleRun(S.n, b, S.row_ptr, S.col_idx, S.vals, k)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
    F, _ = B.bilu_factor(P, b, vals)
    F32 = B.bilu_convert_f32(F)
    x = B.bilu_apply_f32(P, b, F32, rhs).cpu().numpy()
    # the oracle on the FP32-rounded factors and right-hand side
    F_r = o.F.astype(np.float32).astype(np.float64)
    D_r = o.Dinv.astype(np.float32).astype(np.float64)
    r_r = S.rhs.astype(np.float32).astype(np.float64)
    xo = oracle.apply(S.n, b, o.prp, o.pci, F_r, D_r, r_r)
    # FP32 arithmetic through two triangular sweeps: relative error a few
    # hundred units of u for these well-conditioned factors
    assert rel_maxerr(x, xo) <= 1e-4
    # and the FP32 preconditioner is close to the FP64 one
    assert rel_maxerr(x, o.apply(S.rhs)) <= 1e-3


@pytest.mark.parametrize("k", [0, 1])
def test_bicgstab_mixed_reaches_fp64_accuracy(B, k):
    S = reservoir_system(16, 16, 8, 3, sigma=1.0, accum=0.01)
    o = OracleRun(S.n, 3, S.row_ptr, S.col_idx, S.vals, k)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
    F, _ = B.bilu_factor(P, 3, vals)
    F32 = B.bilu_convert_f32(F)
    vals32 = B.bilu_convert_f32(vals)
    A = (S.n, 3, rp, ci, vals)
    x, info = B.bicgstab_solve_mixed(P, A, vals32, F32, rhs, tol=1e-10, maxit=2000, inner_tol=1e-4,
                                     inner_maxit=200)
    assert info.status == 0 and info.true_relres <= 1e-10
    xg = x.cpu().numpy()
    res = np.linalg.norm(S.rhs - o.spmv(xg)) / np.linalg.norm(S.rhs)
    assert res <= 1e-10 * (1 + 1e-6)
    assert res == pytest.approx(info.true_relres, rel=1e-5, abs=1e-16)
    xo, _, _, st = oracle.bicgstab(S.n, 3, S.row_ptr, S.col_idx, S.vals, o.prp, o.pci, o.F, o.Dinv, S.rhs,
                                   tol=1e-12, maxit=2000)
    assert st == 0
    assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)


def test_bicgstab_mixed_edge_cases(B):
    S = reservoir_system(6, 5, 4, 3, sigma=1.0, accum=0.01)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, 0).upload()
    F, _ = B.bilu_factor(P, 3, vals)
    F32, vals32 = B.bilu_convert_f32(F), B.bilu_convert_f32(vals)
    A = (S.n, 3, rp, ci, vals)
    x, info = B.bicgstab_solve_mixed(P, A, vals32, F32, torch.zeros_like(rhs), x=torch.ones_like(rhs))
    assert info.status == 0 and info.iters == 0 and not x.any()
    x, info = B.bicgstab_solve_mixed(P, A, vals32, F32, rhs, tol=1e-14, maxit=3, inner_maxit=2)
    assert info.status == 5 and info.iters == 3
    with pytest.raises(B.BiluError):
        B.bicgstab_solve_mixed(P, A, vals32, F32, rhs, inner_tol=1.5)


@pytest.mark.parametrize("b,k", [(3, 1), (4, 2), (8, 0)])
def test_factor_f32_close_to_fp64(B, b, k):
    """The factorization computed in FP32 stays within FP32 rounding growth of
    the oracle's FP64 factors on these well-conditioned systems."""
    S = reservoir_system(10, 8, 6, b, sigma=1.0, accum=0.01, seed=b + k)
    o = OracleRun(S.n, b, S.row_ptr, S.col_idx, S.vals, k)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
    F32, info = B.bilu_factor_f32(P, b, vals)
    assert info.status == 0
    Lg, Dg, Ug = (t.double().cpu().numpy() for t in B.factor_sections(P, b, F32))
    assert rel_maxerr(Lg, o.L()) <= 1e-4
    assert rel_maxerr(Dg, o.Dinv) <= 1e-4
    assert rel_maxerr(Ug, o.U()) <= 1e-4


def test_mixed_overflowing_fp32_copy_is_a_breakdown(B):
    """A system whose values overflow FP32 (|a| > 3.4e38) has an infinite FP32
    copy: the refinement reports a breakdown and leaves x finite."""
    S = reservoir_system(6, 5, 4, 3, sigma=1.0, accum=0.01)
    rp, ci, vals, rhs = device_system(S, DEV)
    vals = vals * 1e39
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, 0).upload()
    F, _ = B.bilu_factor(P, 3, vals)
    F32, vals32 = B.bilu_convert_f32(F), B.bilu_convert_f32(vals)
    assert not torch.isfinite(vals32).all()
    x, info = B.bicgstab_solve_mixed(P, (S.n, 3, rp, ci, vals), vals32, F32, rhs, tol=1e-8, maxit=50)
    assert info.status == 4 and torch.isfinite(x).all()


@pytest.mark.parametrize("k", [0, 1])
def test_bicgstab_f32prec_reaches_fp64_accuracy(B, k):
    """FP64 BiCGSTAB with the FP32-stored preconditioner reaches the FP64
    tolerance, its solution matches the oracle's FP64 solve, and it needs
    about as many iterations as the FP64 preconditioner."""
    S = reservoir_system(16, 16, 8, 3, sigma=1.0, accum=0.01)
    o = OracleRun(S.n, 3, S.row_ptr, S.col_idx, S.vals, k)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
    F32, _ = B.bilu_factor_f32(P, 3, vals)
    F, _ = B.bilu_factor(P, 3, vals)
    A = (S.n, 3, rp, ci, vals)
    x, info = B.bicgstab_solve_f32prec(P, A, F32, rhs, tol=1e-10, maxit=2000)
    assert info.status == 0 and info.true_relres <= 1e-10
    _, info64 = B.bicgstab_solve(P, A, F, rhs, tol=1e-10, maxit=2000)
    assert info.iters <= 1.5 * info64.iters + 2
    xg = x.cpu().numpy()
    res = np.linalg.norm(S.rhs - o.spmv(xg)) / np.linalg.norm(S.rhs)
    assert res <= 1e-10 * (1 + 1e-6)
    xo, _, _, st = oracle.bicgstab(S.n, 3, S.row_ptr, S.col_idx, S.vals, o.prp, o.pci, o.F, o.Dinv, S.rhs,
                                   tol=1e-12, maxit=2000)
    assert st == 0 and np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)


def test_convert_f32_bit_exact_on_many_values(B):
    """bilu_convert_f32 (integer-pipe rounding with a hardware fallback at the
    edges) agrees bit for bit with round-to-nearest-even: a million values over
    80 decades, values exactly halfway between floats, and the edge cases."""
    rng = np.random.default_rng(7)
    parts = [rng.standard_normal(1_000_000) * 10.0 ** rng.integers(-40, 40, 1_000_000)]
    f = rng.standard_normal(100_000).astype(np.float32)
    half_ulp = np.spacing(f).astype(np.float64) / 2
    parts += [f.astype(np.float64) + half_ulp, f.astype(np.float64) - half_ulp]
    parts.append(np.array([0.0, -0.0, 1e-40, -1e-45, 3.4028234663852886e38, 3.4028235677973366e38, 3.5e38,
                           -1e300, np.inf, -np.inf, 1.1754943508222875e-38, 1.1754942e-38]))
    x = np.concatenate(parts)
    got = B.bilu_convert_f32(torch.from_numpy(x).to(DEV)).cpu().numpy()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_apply_f32_conversions_bit_exact(B):
    """FP32 apply on a b = 1 block-diagonal system: x_i = double(float(d_i *
    float(r_i))), one rounding of one product, so every conversion on the way
    (r to float, y and z through the FP64 vectors and back, x to double) must
    be exact or correctly rounded: the result equals numpy bit for bit.  The
    values span 60 decades, with zeros of both signs, products that underflow
    to float subnormals and products that overflow to infinity."""
    rng = np.random.default_rng(11)
    n = 200_000
    r = rng.standard_normal(n) * 10.0 ** rng.integers(-20, 20, n)
    r[:1000] = 0.0
    r[1000:2000] = -0.0
    a = rng.choice([-1.0, 1.0], n) * rng.uniform(0.5, 2.0, n) * 10.0 ** rng.integers(-10, 10, n)
    r[2000:2100], a[2000:2100] = 1e-30, 1e12       # |d r| ~ 1e-42: float subnormal
    r[2100:2200], a[2100:2200] = -3e25, -1e-16     # |d r| ~ 3e41: float infinity
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    P = B.bilu_symbolic(n, rp, ci, 0).upload()
    F, info = B.bilu_factor(P, 1, torch.from_numpy(a).to(DEV))
    assert info.status == 0
    F32 = B.bilu_convert_f32(F)
    x = B.bilu_apply_f32(P, 1, F32, torch.from_numpy(r).to(DEV)).cpu().numpy()
    d32 = F32.cpu().numpy()
    with np.errstate(over="ignore", under="ignore"):
        z = d32 * r.astype(np.float32) + np.float32(0.0)  # fma(d, r, +0): a zero product is +0
    ref = z.astype(np.float64)
    assert np.array_equal(x.view(np.uint64), ref.view(np.uint64))
    assert np.isinf(ref[2100:2200]).all() and (np.abs(ref[2000:2100]) < 1.2e-38).all()
