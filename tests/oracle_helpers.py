"""Independent dense/brute-force references used to pin the oracle.

These are not restatements of the oracle's code: each computes the same
quantity by a different route (dense n x n level matrices with the paper's
full j loop, shortest fill paths, dense LU, numpy linear algebra).
"""
from __future__ import annotations

from collections import deque

import numpy as np

INF = 1 << 40


def block(vals_row: np.ndarray, b: int) -> np.ndarray:
    """b x b block from its column-major storage (element (r,c) at c*b + r)."""
    return np.asarray(vals_row, dtype=np.float64).reshape(b, b).T


def to_dense(n, b, rp, ci, vals) -> np.ndarray:
    M = np.zeros((n * b, n * b))
    for i in range(n):
        for t in range(rp[i], rp[i + 1]):
            j = ci[t]
            M[i * b:(i + 1) * b, j * b:(j + 1) * b] = block(vals[t], b)
    return M


def pattern_set(n, rp, ci):
    return {(i, int(ci[t])) for i in range(n) for t in range(rp[i], rp[i + 1])}


def dense_levels_alg2(n, rp, ci, k, dropped_to_inf=True):
    """Level bookkeeping of Algorithms 2/3 literally: dense n x n levels, the
    full j = p+1..n loop, the drop test after the row.  Returns {(i,j): lev}."""
    lev = np.full((n, n), INF, dtype=np.int64)
    for i in range(n):
        for t in range(rp[i], rp[i + 1]):
            lev[i, ci[t]] = 0
    for i in range(1, n):
        for p in range(i):
            if lev[i, p] <= k:
                for j in range(p + 1, n):
                    cand = lev[i, p] + lev[p, j] + 1
                    if cand < lev[i, j]:
                        lev[i, j] = cand
        if dropped_to_inf:
            row = lev[i]
            row[row > k] = INF
    return {(i, j): int(lev[i, j]) for i in range(n) for j in range(n) if lev[i, j] <= k}


def fill_path_levels(n, rp, ci):
    """Fill-path theorem (Hysom and Pothen): the level of fill of (i, j) is
    one less than the length of the shortest path i -> j in the graph of A
    whose interior vertices are all numbered below min(i, j)."""
    adj = [list(ci[rp[u]:rp[u + 1]]) for u in range(n)]
    out = {}
    for i in range(n):
        out[(i, i)] = 0
        for j in range(n):
            if j == i:
                continue
            m = min(i, j)
            dist = {i: 0}
            q = deque([i])
            found = None
            while q and found is None:
                u = q.popleft()
                for v in adj[u]:
                    if v == j:
                        found = dist[u] + 1
                        break
                    if v < m and v not in dist:
                        dist[v] = dist[u] + 1
                        q.append(v)
            if found is not None:
                out[(i, j)] = found - 1
    return out


def symbolic_full_fill(n, rp, ci):
    """Pattern of Gaussian elimination without dropping (boolean)."""
    F = np.zeros((n, n), dtype=bool)
    for i in range(n):
        F[i, ci[rp[i]:rp[i + 1]]] = True
    for p in range(n):
        rows = np.nonzero(F[p + 1:, p])[0] + p + 1
        cols = np.nonzero(F[p, p + 1:])[0] + p + 1
        for i in rows:
            F[i, cols] = True
    return {(i, j) for i in range(n) for j in range(n) if F[i, j]}


def split_factors(n, b, prp, pci, F):
    """Dense unit-lower L, block-diagonal D and unit-upper U' from the
    oracle's P'-layout factor array."""
    N = n * b
    L = np.eye(N)
    U = np.eye(N)
    D = np.zeros((N, N))
    for i in range(n):
        for t in range(prp[i], prp[i + 1]):
            j = pci[t]
            blk = block(F[t], b)
            sl_i, sl_j = slice(i * b, (i + 1) * b), slice(j * b, (j + 1) * b)
            if j < i:
                L[sl_i, sl_j] = blk
            elif j > i:
                U[sl_i, sl_j] = blk
            else:
                D[sl_i, sl_j] = blk
    return L, D, U


def diag_dominant_block_values(n, b, rp, ci, seed, boost=None):
    """Random blocks with a strongly dominant diagonal (well-posed pivots)."""
    from paper_1703_01325_gb300.reservoir import random_block_values
    vals = random_block_values(int(rp[-1]), b, seed)
    row_len = np.diff(rp)
    for i in range(n):
        for t in range(rp[i], rp[i + 1]):
            if ci[t] == i:
                d = (boost if boost is not None else 2.0 * b * row_len[i])
                for q in range(b):
                    vals[t, q * b + q] += d
    return vals
