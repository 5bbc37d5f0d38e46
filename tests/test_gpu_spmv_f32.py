"""GPU parity of the FP32 SpMV against the CPU oracle at sizes from a single
block row to the 128 x 128 x 64 matrix of the timed solve.

The oracle runs on the FP32-rounded values and x, so the remaining difference
is FP32 arithmetic, bounded by |fl(sum) - sum| <= gamma_m sum|terms| with
gamma_m = m u / (1 - m u), u = 2^-24 and m the terms of a row's sum."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1703_01325_gb300.reservoir import reservoir_system  # noqa: E402
from tests.gpu_util import device_system  # noqa: E402

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


def spmv_f32_against_oracle(B, S, seed):
    rp, ci, vals, _ = device_system(S, DEV)
    vals32 = B.bilu_convert_f32(vals)
    x = np.random.default_rng(seed).uniform(-1.0, 1.0, S.n * S.b)
    y = B.bsr_spmv_f32(S.n, S.b, rp, ci, vals32, torch.from_numpy(x).to(DEV)).cpu().numpy()
    v32 = S.vals.reshape(-1).astype(np.float32).astype(np.float64)
    x32 = x.astype(np.float32).astype(np.float64)
    yo = oracle.spmv(S.n, S.b, S.row_ptr, S.col_idx, v32, x32)
    absy = oracle.spmv(S.n, S.b, S.row_ptr, S.col_idx, np.abs(v32), np.abs(x32))
    terms = int(np.diff(S.row_ptr).max()) * S.b
    assert np.all(np.isfinite(y))
    assert np.all(np.abs(y - yo) <= 2 * gamma(terms) * absy + 1e-300)
    return rp, ci, vals32, x, y


# Tens of thousands of rows and more, every block size class, both stencils.
@pytest.mark.parametrize("nx,ny,nz,b,stencil", [
    (64, 64, 32, 3, 7), (64, 48, 32, 1, 7), (48, 40, 24, 2, 7), (48, 40, 24, 4, 7),
    (40, 32, 24, 5, 7), (40, 32, 16, 8, 7), (32, 32, 16, 3, 27), (24, 20, 12, 8, 27)])
def test_spmv_f32_matches_oracle_large(B, nx, ny, nz, b, stencil):
    S = reservoir_system(nx, ny, nz, b, stencil=stencil, sigma=1.0, accum=0.01, seed=nx + b)
    spmv_f32_against_oracle(B, S, seed=b)


@pytest.mark.parametrize("n_rows", [1, 2, 3, 5, 11, 97])
def test_spmv_f32_tiny_and_ragged(B, n_rows):
    """A 1-D chain of n_rows block rows: one row, fewer rows than a warp
    holds, and row lengths 1 to 3 (ragged batches of the loads)."""
    S = reservoir_system(n_rows, 1, 1, 3, stencil=7, seed=n_rows)
    spmv_f32_against_oracle(B, S, seed=n_rows)


def test_spmv_f32_full_size_128x128x64(B):
    """The 128 x 128 x 64 seven-point b = 3 matrix of the timed solve, every
    row against the oracle."""
    from paper_1703_01325_gb300.reservoir import WORKLOADS
    S = reservoir_system(**WORKLOADS["grid128x128x64_7pt_b3"])
    spmv_f32_against_oracle(B, S, seed=7)


@pytest.mark.parametrize("b", [1, 2, 3, 5])
@pytest.mark.parametrize("stencil", [7, 27])
def test_staged_equals_direct_kernel_bitwise(B, b, stencil):
    """For b <= 5 the FP32 SpMV stages each warp's matrix range in shared
    memory; values at an address that is not 16-byte aligned take the direct
    kernel.  Both sum each row in the same order, so y is bit-identical (the
    27-point groups overflow the stage buffer and read global memory)."""
    S = reservoir_system(40, 30, 20, b, stencil=stencil, seed=b)
    rp, ci, vals32, x, y = spmv_f32_against_oracle(B, S, seed=3)
    buf = torch.empty(vals32.numel() + 1, dtype=torch.float32, device=DEV)
    buf[1:].copy_(vals32)
    shifted = buf[1:]
    assert shifted.data_ptr() % 16 != 0
    y2 = B.bsr_spmv_f32(S.n, b, rp, ci, shifted, torch.from_numpy(x).to(DEV)).cpu().numpy()
    assert np.array_equal(y.view(np.int64), y2.view(np.int64))


@pytest.mark.parametrize("b", [1, 2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("stencil", [7, 27])
def test_spmv_f32x_matches_oracle_and_f32(B, b, stencil):
    """bsr_spmv_f32x (x in FP32) against the oracle on the same FP32 values,
    and bit-identical to bsr_spmv_f32 on x widened to FP64 (the rounding of
    (double) x32 back to FP32 is exact): the mixed solve relies on this."""
    S = reservoir_system(36, 28, 14, b, stencil=stencil, seed=10 + b)
    rp, ci, vals, _ = device_system(S, DEV)
    vals32 = B.bilu_convert_f32(vals)
    x32 = np.random.default_rng(b).uniform(-1.0, 1.0, S.n * b).astype(np.float32)
    y = B.bsr_spmv_f32x(S.n, b, rp, ci, vals32, torch.from_numpy(x32).to(DEV)).cpu().numpy()
    v32 = S.vals.reshape(-1).astype(np.float32).astype(np.float64)
    xo = x32.astype(np.float64)
    yo = oracle.spmv(S.n, b, S.row_ptr, S.col_idx, v32, xo)
    absy = oracle.spmv(S.n, b, S.row_ptr, S.col_idx, np.abs(v32), np.abs(xo))
    terms = int(np.diff(S.row_ptr).max()) * b
    assert np.all(np.abs(y - yo) <= 2 * gamma(terms) * absy + 1e-300)
    y64 = B.bsr_spmv_f32(S.n, b, rp, ci, vals32, torch.from_numpy(xo).to(DEV)).cpu().numpy()
    assert np.array_equal(y.view(np.int64), y64.view(np.int64))
