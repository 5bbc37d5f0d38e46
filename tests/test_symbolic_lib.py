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


def _chunk_ranges(sched):
    bnd = sched["bounds"]
    return [(int(bnd[c]), int(bnd[c + 1])) for c in range(len(bnd) - 1)]


@pytest.mark.parametrize("rows", [1, 5, 64, 1024])
@pytest.mark.parametrize("k", [0, 2])
def test_solve_schedule_is_a_valid_chunk_order(libbilu, rows, k):
    """The chunks partition the rows into consecutive ranges of at most 1024
    rows; each chunk lists exactly its rows, and every dependency of a row
    inside the same chunk comes earlier in the list."""
    import paper_1703_01325_gb300.bilu as B
    from paper_1703_01325_gb300.reservoir import reservoir_system
    S = reservoir_system(11, 9, 7, 2, stencil=7 if k else 27)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k)
    e = P.export()
    rp, ci = e["row_ptr"], e["col_idx"]
    sch = P.schedule(rows)
    n = S.n
    ranges = _chunk_ranges(sch)
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    assert all(a < b_ <= a + 1024 for a, b_ in ranges)
    assert all(ranges[c][1] == ranges[c + 1][0] for c in range(len(ranges) - 1))
    for lo, hi in ranges:
        for upper in (False, True):
            seq = (sch["ord_upper"] if upper else sch["ord_lower"])[lo:hi]
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
    sch = P.schedule(rows)
    ranges = _chunk_ranges(sch)
    nch = len(ranges)
    chunk_of = np.empty(n, np.int64)
    for c, (lo, hi) in enumerate(ranges):
        chunk_of[lo:hi] = c
    for upper, tick in ((False, sch["tick_lower"]), (True, sch["tick_upper"])):
        assert sorted(tick.tolist()) == list(range(nch))
        pos = np.empty(nch, np.int64)
        pos[tick] = np.arange(nch)
        num = (lambda j: nch - 1 - chunk_of[j]) if upper else (lambda j: chunk_of[j])
        for i in range(n):
            for t in range(rp[i], rp[i + 1]):
                j = int(ci[t])
                if (j > i) if upper else (j < i):
                    a, b_ = num(i), num(j)
                    assert a == b_ or pos[b_] < pos[a]


@pytest.mark.parametrize("nx,rows,want", [(96, 256, 288), (128, 256, 256), (160, 256, 320), (96, 512, 576),
                                          (40, 100, 80)])
@pytest.mark.parametrize("k", [0, 1])
def test_chunks_hold_whole_grid_lines(libbilu, nx, rows, want, k):
    """On a natural-order grid the cuts fall at line starts (rows that do not
    depend on their predecessor), at the multiple of the line length nearest
    the target (a tie goes to the shorter chunk), and at every plane start
    (the largest dependency gap) that a chunk's window reaches, so no chunk
    straddles two planes."""
    import paper_1703_01325_gb300.bilu as B
    ny, nz = 6, 4
    rp, ci = grid_pattern(nx, ny, nz, 7)
    n = nx * ny * nz
    P = B.bilu_symbolic(n, rp, ci, k)
    bnd = P.schedule(rows)["bounds"]
    assert all(int(x) % nx == 0 for x in bnd)
    assert int(bnd[1]) == want
    assert set(range(0, n, nx * ny)) <= set(bnd.tolist())


def test_chunks_without_line_structure_use_the_target(libbilu):
    """A tridiagonal chain has no clean cut: every chunk has the target size."""
    import paper_1703_01325_gb300.bilu as B
    n = 1000
    rows_ = [[j for j in (i - 1, i, i + 1) if 0 <= j < n] for i in range(n)]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows_])]).astype(np.int32)
    ci = np.concatenate(rows_).astype(np.int32)
    P = B.bilu_symbolic(n, rp, ci, 0)
    bnd = P.schedule(64)["bounds"]
    assert bnd.tolist() == list(range(0, n, 64)) + [n]


@pytest.mark.parametrize("dims,stencil,k,want", [
    ((96, 96, 48), 7, 1, 288),     # three 96-row grid lines
    ((128, 128, 24), 7, 1, 384),   # three 128-row grid lines
    ((160, 160, 16), 27, 0, 256),  # lines longer than 128 rows: the size rule's cap
])
def test_auto_factor_chunk_target_is_three_grid_lines(libbilu, dims, stencil, k, want):
    """Large systems (n / (2 * SMs) >= 256 rows) factor in chunks of three grid
    lines, from the same line length as the solves' chunks."""
    import paper_1703_01325_gb300.bilu as B
    from paper_1703_01325_gb300.reservoir import reservoir_system
    S = reservoir_system(*dims, 1, stencil=stencil, sigma=1.0, accum=0.01)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k)
    assert B.bilu_auto_factor_chunk(P) == want


@pytest.mark.parametrize("dims,stencil,k,want,chunk", [
    ((96, 96, 48), 7, 1, 192, 192),     # two 96-row grid lines
    ((128, 128, 24), 7, 1, 256, 256),   # two 128-row grid lines
    ((160, 160, 16), 27, 0, 320, 320),  # two 160-row grid lines of a 27-point grid
    ((300, 300, 5), 7, 0, 256, 300),    # lines longer than 192 rows: the size rule's cap,
])                                      # cut at the nearest line start
def test_auto_chunk_target_is_two_grid_lines(libbilu, dims, stencil, k, want, chunk):
    """Large systems (n / (10 * SMs) >= 256 rows, on any part with up to 152
    SMs) get two grid lines per chunk: the pattern's line length is the most
    common distance between rows that do not depend on their predecessor."""
    import paper_1703_01325_gb300.bilu as B
    from paper_1703_01325_gb300.reservoir import reservoir_system
    S = reservoir_system(*dims, 1, stencil=stencil, sigma=1.0, accum=0.01)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k)
    assert B.bilu_auto_trisolve_chunk(P) == want
    # and the schedule cut at that target holds whole lines (plane ends aside)
    lens = np.diff(P.schedule(want)["bounds"])
    assert np.bincount(lens).argmax() == chunk


@pytest.mark.parametrize("n,seed", [(3000, 1), (20000, 2)])
def test_auto_chunk_targets_without_grid_lines(libbilu, n, seed):
    """A pattern without recurring line starts falls back to the size rules:
    n / (10 * SMs) in [32, 256] for the solves, n / (2 * SMs) in [64, 256]
    for the factorization (SMs = 1 when the library sees no GPU)."""
    import paper_1703_01325_gb300.bilu as B
    torch = pytest.importorskip("torch")
    sms = torch.cuda.get_device_properties(0).multi_processor_count if torch.cuda.is_available() else 1
    rp, ci = random_pattern(n, density=4.0 / n, seed=seed)
    P = B.bilu_symbolic(n, rp, ci, 0)
    assert B.bilu_auto_trisolve_chunk(P) == max(32, min(256, n // (10 * sms)))
    assert B.bilu_auto_factor_chunk(P) == max(64, min(256, n // (2 * sms)))
