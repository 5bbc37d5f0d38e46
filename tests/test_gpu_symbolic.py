"""The device symbolic phase (bilu_symbolic_gpu) against the host one: P', the
level of every entry and both Eq. 4 level sets must agree bit for bit (the
host phase is itself bit-exact with the oracle, test_symbolic_lib.py)."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1703_01325_gb300.reservoir import grid_pattern, random_pattern  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(libbilu):
    import paper_1703_01325_gb300.bilu as B
    torch.cuda.set_device(0)
    return B


def _same(B, n, rp, ci, k, cap=256):
    h = B.bilu_symbolic(n, rp, ci, k).export()
    g = B.bilu_symbolic_gpu(n, rp, ci, k, row_capacity=cap).export()
    for key in ("row_ptr", "col_idx", "lev", "lvl_lower", "lvl_upper"):
        assert np.array_equal(h[key], g[key]), key


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
    """The 128 x 128 x 64 7-point pattern at ILU(1)."""
    rp, ci = grid_pattern(128, 128, 64, 7)
    _same(B, 128 * 128 * 64, rp, ci, 1, cap=64)
