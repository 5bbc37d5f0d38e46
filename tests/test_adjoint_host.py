"""Host side of the adjoint: the block CSR transpose and the transposed
pattern P'^T against plain numpy transposes and the oracle's Eq. 4 levels.
CPU only."""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1703_01325_gb300.reservoir import grid_pattern, random_pattern


def _np_transpose(n, rp, ci, vals=None):
    rows = np.repeat(np.arange(n), np.diff(rp))
    order = np.lexsort((rows, ci))  # by column, then row
    rpt = np.zeros(n + 1, np.int64)
    np.add.at(rpt, ci + 1, 1)
    return np.cumsum(rpt), rows[order], order


@pytest.mark.parametrize("seed", range(6))
def test_bsr_transpose_pattern(libbilu, seed):
    import paper_1703_01325_gb300.bilu as B
    n = 17 + 13 * seed
    rp, ci = random_pattern(n, density=0.05 + 0.02 * seed, seed=300 + seed, symmetric=False)
    rpt, cit, perm = B.bsr_transpose_pattern(n, rp, ci)
    ert, ecit, eperm = _np_transpose(n, rp, ci)
    assert np.array_equal(rpt, ert) and np.array_equal(cit, ecit) and np.array_equal(perm, eperm)
    # transposing twice gives A back
    rpt2, cit2, perm2 = B.bsr_transpose_pattern(n, rpt, cit)
    assert np.array_equal(rpt2, rp) and np.array_equal(cit2, ci)
    assert np.array_equal(perm[perm2], np.arange(len(ci)))


def test_bsr_transpose_pattern_edges(libbilu):
    import paper_1703_01325_gb300.bilu as B
    rpt, cit, perm = B.bsr_transpose_pattern(0, np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert rpt.tolist() == [0] and len(cit) == 0
    # rows with no blocks
    rpt, cit, perm = B.bsr_transpose_pattern(3, np.array([0, 0, 2, 2]), np.array([0, 2]))
    assert rpt.tolist() == [0, 1, 1, 2] and cit.tolist() == [1, 1] and perm.tolist() == [0, 1]
    with pytest.raises(B.BiluError):
        B.bsr_transpose_pattern(2, np.array([0, 1, 2]), np.array([0, 5]))


@pytest.mark.parametrize("k", [0, 1, 2])
@pytest.mark.parametrize("case", ["grid7", "grid27", "random"])
def test_pattern_transpose(libbilu, k, case):
    """P'^T is the transpose of P' (entries and their fill levels), its Eq. 4
    levels are the oracle's levels of the transposed pattern, and its L / U'
    counts swap."""
    import paper_1703_01325_gb300.bilu as B
    if case == "grid7":
        rp, ci = grid_pattern(7, 5, 4, 7)
    elif case == "grid27":
        rp, ci = grid_pattern(5, 4, 3, 27)
    else:
        rp, ci = random_pattern(90, density=0.04, seed=91 + k, symmetric=False)
    n = len(rp) - 1
    P = B.bilu_symbolic(n, rp, ci, k)
    e = P.export()
    PT = P.transpose(upload=False)
    t = PT.export()
    ert, ecit, order = _np_transpose(n, e["row_ptr"], e["col_idx"])
    assert np.array_equal(t["row_ptr"], ert)
    assert np.array_equal(t["col_idx"], ecit)
    assert np.array_equal(t["lev"], e["lev"][order])
    lo, up = oracle.levels(n, ert.astype(np.int32), ecit.astype(np.int32))
    assert np.array_equal(t["lvl_lower"], lo) and np.array_equal(t["lvl_upper"], up)
    assert PT.info.nnz_l == P.info.nnz_u and PT.info.nnz_u == P.info.nnz_l
    assert PT.info.nnz_p == P.info.nnz_p


def test_transposed_pattern_refuses_factor_and_transpose(libbilu):
    import paper_1703_01325_gb300.bilu as B
    from paper_1703_01325_gb300 import _lib as L
    rp, ci = grid_pattern(4, 3, 2, 7)
    P = B.bilu_symbolic(24, rp, ci, 1)
    PT = P.transpose(upload=False)
    h = C.c_void_p()
    assert libbilu.bilu_pattern_transpose(PT.handle, C.byref(h)) == L.BILU_ERR_ARG
    info = L.FactorInfo()
    assert libbilu.bilu_factor(PT.handle, 3, None, None, None, 0, None, C.byref(info)) == L.BILU_ERR_ARG
    assert libbilu.bilu_factor_transpose(P.handle, 3, None, None, None) == L.BILU_ERR_ARG
