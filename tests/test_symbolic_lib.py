"""The library's host symbolic phase against the oracle: P', the level of
every entry and both Eq. 4 level sets must agree bit for bit.  CPU only."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1703_01325_gb300.reservoir import grid_pattern, random_pattern


def _compare(B, n, rp, ci, k):
    P = B.bilu_symbolic(n, rp, ci, k)
    e = P.export()
    prp, pci, plev = oracle.symbolic(n, rp, ci, k)
    lo, up = oracle.levels(n, prp, pci)
    assert np.array_equal(e["row_ptr"], prp)
    assert np.array_equal(e["col_idx"], pci)
    assert np.array_equal(e["lev"], plev)
    assert np.array_equal(e["lvl_lower"], lo)
    assert np.array_equal(e["lvl_upper"], up)
    info = P.info
    assert info.nnz_p == len(pci) and info.nnz_a == rp[-1]
    rows = np.repeat(np.arange(n), np.diff(prp))
    assert info.nnz_l == int((pci < rows).sum()) and info.nnz_u == int((pci > rows).sum())
    assert info.nlev_l == (lo.max() + 1 if n else 0) and info.nlev_u == (up.max() + 1 if n else 0)
    P.close()


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("k", [0, 1, 2, 3, 8])
def test_random_patterns(libbilu, seed, k):
    import paper_1703_01325_gb300.bilu as B
    n = 20 + 9 * seed
    rp, ci = random_pattern(n, density=3.0 / n + 0.01 * (seed % 3), seed=1000 + seed,
                            symmetric=(seed % 2 == 0))
    _compare(B, n, rp, ci, k)


@pytest.mark.parametrize("grid", [(7, 5, 3), (16, 16, 8), (9, 4, 11)])
@pytest.mark.parametrize("stencil", [7, 27])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_grid_patterns(libbilu, grid, stencil, k):
    import paper_1703_01325_gb300.bilu as B
    rp, ci = grid_pattern(*grid, stencil)
    _compare(B, int(np.prod(grid)), rp, ci, k)


def test_full_fill_and_empty(libbilu):
    import paper_1703_01325_gb300.bilu as B
    rp, ci = random_pattern(60, density=0.05, seed=77)
    _compare(B, 60, rp, ci, 60)
    P = B.bilu_symbolic(0, np.zeros(1, np.int32), np.zeros(0, np.int32), 1)
    assert P.info.n == 0 and P.info.nnz_p == 0


def test_error_codes(libbilu):
    import paper_1703_01325_gb300.bilu as B
    from paper_1703_01325_gb300 import _lib as L
    bad = [
        (2, [0, 1, 2], [0, 0]),          # row 1 lacks its diagonal
        (2, [0, 2, 3], [1, 0, 1]),       # unsorted
        (2, [0, 2, 3], [0, 0, 1]),       # duplicate
        (2, [0, 1, 2], [0, 2]),          # out of range
        (2, [1, 2, 3], [0, 1]),          # row_ptr[0] != 0
    ]
    for n, rp, ci in bad:
        with pytest.raises(B.BiluError) as e:
            B.bilu_symbolic(n, np.array(rp), np.array(ci), 1)
        assert e.value.status == L.BILU_ERR_PATTERN
    with pytest.raises(B.BiluError) as e:
        B.bilu_symbolic(2, np.array([0, 1, 2]), np.array([0, 1]), -1)
    assert e.value.status == L.BILU_ERR_ARG
    assert libbilu.bilu_status_string(L.BILU_ERR_TIMEOUT).decode().startswith("a bounded")


@pytest.mark.parametrize("rows", [1, 5, 64, 1024])
@pytest.mark.parametrize("k", [0, 2])
def test_solve_schedule_is_a_valid_chunk_order(libbilu, rows, k):
    """Each chunk of the sync-free solves lists exactly its rows, and every
    dependency of a row inside the same chunk comes earlier in the list."""
    import paper_1703_01325_gb300.bilu as B
    from paper_1703_01325_gb300.reservoir import reservoir_system
    S = reservoir_system(11, 9, 7, 2, stencil=7 if k else 27)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k)
    e = P.export()
    rp, ci = e["row_ptr"], e["col_idx"]
    ordl, ordu = P.schedule(rows)
    n = S.n
    nch = (n + rows - 1) // rows
    for c in range(nch):
        for upper in (False, True):
            if not upper:
                lo, hi = c * rows, min(n, (c + 1) * rows)
                seq = ordl[c * rows:c * rows + hi - lo]
            else:
                hi = n - c * rows
                lo = max(0, hi - rows)
                seq = ordu[c * rows:c * rows + hi - lo]
            assert sorted(seq.tolist()) == list(range(lo, hi))
            where = {int(i): q for q, i in enumerate(seq)}
            for i in seq:
                for t in range(rp[i], rp[i + 1]):
                    j = int(ci[t])
                    dep = (j > i) if upper else (j < i)
                    if dep and lo <= j < hi:
                        assert where[j] < where[int(i)]


@pytest.mark.parametrize("rows", [1, 7, 64, 256])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_chunk_tickets_are_a_topological_order(libbilu, rows, k):
    """The claim tickets list every chunk once, and every chunk a chunk depends
    on (through any row) has a smaller ticket: no claimed chunk can wait on an
    unclaimed one, whatever number of CTAs is resident."""
    import paper_1703_01325_gb300.bilu as B
    from paper_1703_01325_gb300.reservoir import reservoir_system
    S = reservoir_system(13, 11, 6, 2, stencil=7 if k < 2 else 27)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k)
    e = P.export()
    rp, ci = e["row_ptr"], e["col_idx"]
    n = S.n
    nch = (n + rows - 1) // rows
    _, _, tl, tu = P.schedule(rows, tickets=True)
    for upper, tick in ((False, tl), (True, tu)):
        assert sorted(tick.tolist()) == list(range(nch))
        pos = np.empty(nch, np.int64)
        pos[tick] = np.arange(nch)
        chunk_of = (lambda j: (n - 1 - j) // rows) if upper else (lambda j: j // rows)
        for i in range(n):
            for t in range(rp[i], rp[i + 1]):
                j = int(ci[t])
                if (j > i) if upper else (j < i):
                    a, b_ = chunk_of(i), chunk_of(j)
                    assert a == b_ or pos[b_] < pos[a]
