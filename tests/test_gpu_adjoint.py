"""GPU checks of the adjoint: block gather-transposes and -lambda x^T against
numpy, the transposed preconditioner against a dense M^{-T} built from the
oracle's factors and against the adjoint identity <M^{-T} r, s> = <r, M^{-1} s>
(oracle M^{-1}), and the autograd gradients against a dense reference
(4 x 4 x 4) and central finite differences (64 x 64 x 32, h = 1e-6)."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1703_01325_gb300.reservoir import loss_weights, random_pattern, reservoir_system  # noqa: E402
from tests.gpu_util import OracleRun, device_system, rel_maxerr  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def B(libbilu):
    import paper_1703_01325_gb300.bilu as B
    torch.cuda.set_device(0)
    return B


def _blocks(vals, b):
    """(nblocks, b, b) array [block][row][col] from column-major b*b blocks."""
    return np.asarray(vals).reshape(-1, b, b).transpose(0, 2, 1)


def _dense(n, b, rp, ci, vals):
    A = np.zeros((n * b, n * b))
    blk = _blocks(vals, b)
    for i in range(n):
        for t in range(rp[i], rp[i + 1]):
            j = ci[t]
            A[i * b:(i + 1) * b, j * b:(j + 1) * b] = blk[t]
    return A


def _dense_M(o):
    """M = L D U' from the oracle's factors (L, U' unit block triangular)."""
    n, b = o.n, o.b
    rows = np.repeat(np.arange(n), np.diff(o.prp))
    Ld = np.eye(n * b)
    Ud = np.eye(n * b)
    blk = _blocks(o.F, b)
    for t in range(len(o.pci)):
        i, j = rows[t], o.pci[t]
        if j < i:
            Ld[i * b:(i + 1) * b, j * b:(j + 1) * b] = blk[t]
        elif j > i:
            Ud[i * b:(i + 1) * b, j * b:(j + 1) * b] = blk[t]
    D = np.zeros((n * b, n * b))
    dinv = _blocks(o.Dinv, b)
    for i in range(n):
        D[i * b:(i + 1) * b, i * b:(i + 1) * b] = np.linalg.inv(dinv[i])
    return Ld @ D @ Ud


@pytest.mark.parametrize("b", [1, 2, 3, 5, 8])
def test_gather_transpose_and_outer_grad(B, b):
    n = 40
    rp, ci = random_pattern(n, density=0.1, seed=7 + b, symmetric=False)
    nnz = len(ci)
    rng = np.random.default_rng(b)
    vals = rng.standard_normal(nnz * b * b)
    rpt, cit, perm = B.bsr_transpose_pattern(n, rp, ci)
    got = B.bsr_gather_transpose(b, torch.from_numpy(perm).to(DEV), torch.from_numpy(vals).to(DEV)).cpu().numpy()
    want = _blocks(vals, b)[perm].transpose(0, 2, 1)  # [block][row][col] of A^T blocks
    assert np.array_equal(_blocks(got, b), want)
    lam, x = rng.standard_normal(n * b), rng.standard_normal(n * b)
    g = B.bsr_outer_grad(n, b, torch.from_numpy(rp).to(DEV), torch.from_numpy(ci).to(DEV),
                         torch.from_numpy(lam).to(DEV), torch.from_numpy(x).to(DEV)).cpu().numpy()
    rows = np.repeat(np.arange(n), np.diff(rp))
    ref = -np.einsum("tr,tc->trc", lam.reshape(n, b)[rows], x.reshape(n, b)[ci])
    assert np.array_equal(_blocks(g, b), ref)


@pytest.mark.parametrize("b,k", [(1, 1), (3, 0), (3, 2), (4, 1)])
def test_transposed_apply_small_dense(B, b, k):
    S = reservoir_system(5, 4, 3, b, sigma=1.0, accum=0.01, seed=20 + b + k)
    o = OracleRun(S.n, b, S.row_ptr, S.col_idx, S.vals, k)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
    F, info = B.bilu_factor(P, b, vals)
    PT = P.transpose()
    FT = B.bilu_factor_transpose(PT, b, F)
    z = B.bilu_apply(PT, b, FT, rhs).cpu().numpy()
    M = _dense_M(o)
    assert rel_maxerr(z, np.linalg.solve(M.T, S.rhs)) <= 1e-10
    # the D section of the transposed factors is D^{-T}, exactly
    _, Dg, _ = (t.cpu().numpy() for t in B.factor_sections(P, b, F))
    _, Dt, _ = (t.cpu().numpy() for t in B.factor_sections(PT, b, FT))
    assert np.array_equal(_blocks(Dt, b), _blocks(Dg, b).transpose(0, 2, 1))


@pytest.mark.parametrize("grid,k", [((24, 20, 10), 1), ((13, 9, 7), 2)])
def test_transposed_apply_adjoint_identity(B, grid, k):
    """<M^{-T} r, s> = <r, M^{-1} s> with M^{-1} s from the oracle, and the
    transposed factors hold exactly F's blocks transposed."""
    S = reservoir_system(*grid, 3, sigma=1.0, accum=0.01, seed=11)
    o = OracleRun(S.n, 3, S.row_ptr, S.col_idx, S.vals, k)
    rp, ci, vals, rhs = device_system(S, DEV)
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
    F, _ = B.bilu_factor(P, 3, vals)
    PT = P.transpose()
    FT = B.bilu_factor_transpose(PT, 3, F)
    Lg, Dg, Ug = (t.cpu().numpy() for t in B.factor_sections(P, 3, F))
    Lt, Dt, Ut = (t.cpu().numpy() for t in B.factor_sections(PT, 3, FT))
    assert np.array_equal(_blocks(Dt, 3), _blocks(Dg, 3).transpose(0, 2, 1))
    e, et = P.export(), PT.export()
    _, _, order = _transpose_order(S.n, e["row_ptr"], e["col_idx"])
    rows = np.repeat(np.arange(S.n), np.diff(e["row_ptr"]))
    up = e["col_idx"] > rows
    # U'^T blocks in P'^T row order are U' blocks in P' column order, transposed
    src_u = np.cumsum(up) - 1
    rows_t = np.repeat(np.arange(S.n), np.diff(et["row_ptr"]))
    low_t = et["col_idx"] < rows_t
    assert np.array_equal(_blocks(Lt, 3), _blocks(Ug, 3)[src_u[order[low_t]]].transpose(0, 2, 1))
    rng = np.random.default_rng(5)
    r, s = rng.standard_normal(S.n * 3), rng.standard_normal(S.n * 3)
    z = B.bilu_apply(PT, 3, FT, torch.from_numpy(r).to(DEV)).cpu().numpy()
    lhs, rhs_ = z @ s, r @ o.apply(s)
    assert abs(lhs - rhs_) <= 1e-10 * np.linalg.norm(z) * np.linalg.norm(s)


def _transpose_order(n, rp, ci):
    rows = np.repeat(np.arange(n), np.diff(rp))
    order = np.lexsort((rows, ci))
    return None, None, order


def test_autograd_matches_dense_gradient(B):
    """4 x 4 x 4 cells, b = 3, ILU(1): dL/dvals and dL/drhs of L = ||W x||^2
    against x = A^{-1} b, lambda = A^{-T} (2 W^2 x) computed densely."""
    from paper_1703_01325_gb300.adjoint import BlockILUSolver
    S = reservoir_system(4, 4, 4, 3, sigma=1.0, accum=0.01, seed=4)
    w = loss_weights(S.n, 3, seed=4)
    solver = BlockILUSolver(S.n, 3, S.row_ptr, S.col_idx, 1, tol=1e-13, device=DEV)
    vals = torch.from_numpy(S.vals.reshape(-1).copy()).to(DEV).requires_grad_(True)
    rhs = torch.from_numpy(S.rhs.copy()).to(DEV).requires_grad_(True)
    W = torch.from_numpy(w).to(DEV)
    x = solver.solve(vals, rhs)
    loss = ((W * x) ** 2).sum()
    loss.backward()
    A = _dense(S.n, 3, S.row_ptr, S.col_idx, S.vals.reshape(-1))
    xd = np.linalg.solve(A, S.rhs)
    lam = np.linalg.solve(A.T, 2 * w * w * xd)
    rows = np.repeat(np.arange(S.n), np.diff(S.row_ptr))
    gref = -np.einsum("tr,tc->trc", lam.reshape(-1, 3)[rows], xd.reshape(-1, 3)[S.col_idx])
    assert rel_maxerr(x.detach().cpu().numpy(), xd) <= 1e-10
    assert rel_maxerr(rhs.grad.cpu().numpy(), lam) <= 1e-9
    assert rel_maxerr(_blocks(vals.grad.cpu().numpy(), 3), gref) <= 1e-9


def _fd_check(B, S, k, entries, tol, stable):
    """Central differences (h = 1e-6) of L = ||W x||^2 on `entries` random
    entries of the values and of the right-hand side against the adjoint
    gradient.  With `stable`, L(+h) - L(-h) is formed as
    sum W^2 (x+ - x-)(x+ + x-), the difference x+ - x- of the two perturbed
    solutions taken from one more solve with A (A (x+ - x-) = -h E (x+ + x-)
    for a value entry E, = 2h e_q for a right-hand side entry): an identity,
    not a linearisation.  Subtracting the two losses directly keeps only about
    cond(A) * solve tolerance / h of relative accuracy, too little on a
    131,072-cell system."""
    from paper_1703_01325_gb300.adjoint import BlockILUSolver
    b = S.b
    w = torch.from_numpy(loss_weights(S.n, b, seed=1703)).to(DEV)
    solver = BlockILUSolver(S.n, b, S.row_ptr, S.col_idx, k, tol=1e-13, device=DEV)
    vals0 = torch.from_numpy(S.vals.reshape(-1).copy()).to(DEV)
    rhs0 = torch.from_numpy(S.rhs.copy()).to(DEV)
    vals = vals0.clone().requires_grad_(True)
    rhs = rhs0.clone().requires_grad_(True)
    loss = ((w * solver.solve(vals, rhs)) ** 2).sum()
    loss.backward()
    gv, gr = vals.grad.cpu().numpy(), rhs.grad.cpu().numpy()
    sol = lambda v, r: solver.solve(v, r).detach()
    x0 = sol(vals0, rhs0)
    rows = np.repeat(np.arange(S.n), np.diff(S.row_ptr))
    rng = np.random.default_rng(64)
    h = 1e-6
    for which, g, base in (("vals", gv, vals0), ("rhs", gr, rhs0)):
        idx = rng.choice(base.numel(), entries, replace=False)
        fd = []
        with torch.no_grad():
            for q in idx:
                p, m = base.clone(), base.clone()
                p[q] += h
                m[q] -= h
                xp, xm = (sol(p, rhs0), sol(m, rhs0)) if which == "vals" else (sol(vals0, p), sol(vals0, m))
                if not stable:
                    fd.append(float(((w * xp) ** 2).sum() - ((w * xm) ** 2).sum()) / (2 * h))
                    continue
                f = torch.zeros_like(rhs0)
                if which == "vals":
                    t, e = divmod(int(q), b * b)
                    r, c = e % b, e // b
                    f[rows[t] * b + r] = -h * (xp + xm)[S.col_idx[t] * b + c]
                else:
                    f[int(q)] = 2 * h
                d = sol(vals0, f)
                fd.append(float((w * w * d * (xp + xm)).sum()) / (2 * h))
        fd = np.array(fd)
        assert np.abs(fd - g[idx]).max() <= tol * np.abs(g).max(), (which, np.abs(fd - g[idx]).max())
    return x0


def test_autograd_matches_finite_differences(B):
    """64 x 64 x 32 cells, b = 3, ILU(1): 64 random entries (32 values, 32
    right-hand side), central differences with h = 1e-6, agreement to 1e-5."""
    S = reservoir_system(64, 64, 32, 3, sigma=1.0, accum=0.01, seed=1703)
    _fd_check(B, S, 1, 32, 1e-5, stable=True)


def test_autograd_matches_plain_finite_differences_small(B):
    """8 x 8 x 8 cells, b = 3, ILU(1): the plain difference of the two losses
    already agrees to 1e-5 on a well-conditioned small system."""
    S = reservoir_system(8, 8, 8, 3, sigma=1.0, accum=0.1, seed=17)
    _fd_check(B, S, 1, 16, 1e-5, stable=False)


def test_autograd_matches_plain_central_differences_64x64x32(B):
    """64 x 64 x 32 cells, b = 3, ILU(1): plain central differences (h = 1e-6)
    of L = ||W x||^2 on 32 entries (16 block values, 16 right-hand side
    components) -- two independent evaluations L(+h) and L(-h), subtracted --
    against the adjoint gradient, entry by entry:
    |fd - g_q| <= 1e-5 * max(|g_q|, 1e-3 max|g|).  Each perturbed system is
    solved to 1e-13 by one refinement step from the unperturbed solution x0
    (x = x0 + d, A(+-h) d = rhs(+-h) - A(+-h) x0), so the solver's error in x0
    is common to both evaluations instead of swamping their O(h) difference."""
    from paper_1703_01325_gb300.adjoint import BlockILUSolver
    S = reservoir_system(64, 64, 32, 3, sigma=1.0, accum=0.01, seed=1703)
    b = S.b
    w = torch.from_numpy(loss_weights(S.n, b, seed=1703)).to(DEV)
    solver = BlockILUSolver(S.n, b, S.row_ptr, S.col_idx, 1, tol=1e-13, device=DEV)
    vals0 = torch.from_numpy(S.vals.reshape(-1).copy()).to(DEV)
    rhs0 = torch.from_numpy(S.rhs.copy()).to(DEV)
    vals = vals0.clone().requires_grad_(True)
    rhs = rhs0.clone().requires_grad_(True)
    ((w * solver.solve(vals, rhs)) ** 2).sum().backward()
    gv, gr = vals.grad.cpu().numpy(), rhs.grad.cpu().numpy()
    rp, ci = (torch.from_numpy(a).to(DEV) for a in (S.row_ptr, S.col_idx))
    with torch.no_grad():
        x0 = solver.solve(vals0, rhs0).detach()

        def loss(v, r):
            d = solver.solve(v, r - B.bsr_spmv(S.n, b, rp, ci, v, x0)).detach()
            return float(((w * (x0 + d)) ** 2).sum())

        rng = np.random.default_rng(32)
        h = 1e-6
        for which, g, base in (("vals", gv, vals0), ("rhs", gr, rhs0)):
            idx = rng.choice(base.numel(), 16, replace=False)
            gmax = np.abs(g).max()
            for q in idx:
                p, m = base.clone(), base.clone()
                p[q] += h
                m[q] -= h
                if which == "vals":
                    fd = (loss(p, rhs0) - loss(m, rhs0)) / (2 * h)
                else:
                    fd = (loss(vals0, p) - loss(vals0, m)) / (2 * h)
                bound = 1e-5 * max(abs(g[q]), 1e-3 * gmax)
                assert abs(fd - g[q]) <= bound, (which, int(q), fd, g[q], bound)
