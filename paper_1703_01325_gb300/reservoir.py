"""Seeded synthetic reservoir-style block matrices -- inputs only.

This module draws the inputs that both the CUDA library and the CPU oracle are
fed; it holds none of the ILU(k) method's arithmetic.  The matrices stand in
for the paper's workloads (a 3-D 7-point Poisson matrix and two SuiteSparse
matrices with about seven nonzeros per row, Section 3), which are not
available here.

Recipe (a cell-centred finite-volume discretisation with b unknowns per cell):

* cells on an nx x ny x nz grid, numbered c = x + nx*(y + ny*z) (natural
  lexicographic order); one b x b block row per cell;
* 7-point (faces) or 27-point (all 26 neighbours) stencil, block columns
  sorted ascending;
* permeability K_c = exp(sigma * g_c), g_c ~ N(0, 1) by Box-Muller;
* transmissibility T_cd = 2 K_c K_d / (K_c + K_d) (harmonic mean);
* off-diagonal block A_cd = -T_cd (I + 0.1 R_cd), R_cd uniform in
  [-1, 1]^{b x b}, drawn independently for every ordered pair, so A is
  nonsymmetric;
* diagonal block A_cc = (sum_d T_cd) I + accum (I + 0.1 R'_c);
* right-hand side uniform in [-1, 1]^{n b}.

Random numbers come from a counter-based generator: u = splitmix64 of a
per-(seed, stream) key plus the element index, top 53 bits scaled to [0, 1).
The same numbers result whatever order elements are drawn in.

Blocks are stored column by column (element (r, c) of block t at
``vals[t, c*b + r]``), as the paper's block CSR format prescribes.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

STREAM_PERM = 1
STREAM_R = 2
STREAM_RDIAG = 3
STREAM_RHS = 4
STREAM_W = 5
STREAM_PATTERN = 6

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on uint64 arrays."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, stream: int, idx) -> np.ndarray:
    """Counter-based uniforms in [0, 1) with 53 random bits."""
    key = splitmix64(np.array([(seed & 0xFFFFFFFFFFFF) | (stream << 56)], dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        z = splitmix64(np.asarray(idx, dtype=np.uint64) + key)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, stream: int, idx, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, stream, idx)


def stencil_offsets(stencil: int):
    """(dx, dy, dz) neighbour offsets, sorted by the column they address."""
    if stencil == 7:
        offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    elif stencil == 27:
        offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    else:
        raise ValueError("stencil must be 7 or 27")
    return offs


def grid_pattern(nx: int, ny: int, nz: int, stencil: int = 7):
    """Block CSR pattern (row_ptr, col_idx) of the grid stencil, int32."""
    n = nx * ny * nz
    c = np.arange(n, dtype=np.int64)
    x = c % nx
    y = (c // nx) % ny
    z = c // (nx * ny)
    offs = stencil_offsets(stencil)
    valid = np.empty((n, len(offs)), dtype=bool)
    delta = np.empty(len(offs), dtype=np.int64)
    for o, (dx, dy, dz) in enumerate(offs):
        valid[:, o] = ((x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
                       & (z + dz >= 0) & (z + dz < nz))
        delta[o] = dx + nx * dy + nx * ny * dz
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    cols = (c[:, None] + delta[None, :])[valid]
    return row_ptr.astype(np.int32), cols.astype(np.int32)


@dataclass
class BlockSystem:
    """A block CSR system A x = rhs with b x b column-major blocks."""
    n: int
    b: int
    row_ptr: np.ndarray  # int32 [n+1]
    col_idx: np.ndarray  # int32 [nnzb]
    vals: np.ndarray     # float64 [nnzb, b*b]
    rhs: np.ndarray      # float64 [n*b]
    grid: tuple = ()
    stencil: int = 7

    @property
    def nnzb(self) -> int:
        return int(self.row_ptr[-1])


def reservoir_system(nx: int, ny: int, nz: int, b: int, stencil: int = 7, sigma: float = 1.0,
                     accum: float = 0.01, seed: int = 1703) -> BlockSystem:
    """The seeded reservoir-style matrix and right-hand side described above."""
    n = nx * ny * nz
    row_ptr, col_idx = grid_pattern(nx, ny, nz, stencil)
    nnzb = int(row_ptr[-1])
    bb = b * b
    cells = np.arange(n, dtype=np.uint64)
    u1 = uniform01(seed, STREAM_PERM, 2 * cells)
    u2 = uniform01(seed, STREAM_PERM, 2 * cells + np.uint64(1))
    g = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    K = np.exp(sigma * g)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    cols = col_idx.astype(np.int64)
    Kr, Kc = K[rows], K[cols]
    T = 2.0 * Kr * Kc / (Kr + Kc)
    off = rows != cols
    eye = np.zeros(bb, dtype=np.float64)
    eye[[q * b + q for q in range(b)]] = 1.0
    vals = uniform(seed, STREAM_R, np.arange(nnzb * bb, dtype=np.uint64), -1.0, 1.0).reshape(nnzb, bb)
    vals *= 0.1
    vals += eye[None, :]
    vals[off] *= -T[off, None]
    diag = np.nonzero(~off)[0]
    sumT = np.bincount(rows[off], weights=T[off], minlength=n)
    rdiag = uniform(seed, STREAM_RDIAG, np.arange(n * bb, dtype=np.uint64), -1.0, 1.0).reshape(n, bb)
    vals[diag] = sumT[:, None] * eye[None, :] + accum * (eye[None, :] + 0.1 * rdiag)
    rhs = uniform(seed, STREAM_RHS, np.arange(n * b, dtype=np.uint64), -1.0, 1.0)
    return BlockSystem(n=n, b=b, row_ptr=row_ptr, col_idx=col_idx, vals=vals, rhs=rhs,
                       grid=(nx, ny, nz), stencil=stencil)


def random_pattern(n: int, density: float, seed: int, symmetric: bool = False):
    """Random sparse pattern with a full diagonal (for tiny structural tests)."""
    u = uniform01(seed, STREAM_PATTERN, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    M = u < density
    if symmetric:
        M = M | M.T
    np.fill_diagonal(M, True)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum(M.sum(axis=1))
    col_idx = np.nonzero(M)[1].astype(np.int32)
    return row_ptr, col_idx


def random_block_values(nnzb: int, b: int, seed: int, stream: int = STREAM_R) -> np.ndarray:
    """Uniform [-1, 1] block values (for tiny structural tests)."""
    return uniform(seed, stream, np.arange(nnzb * b * b, dtype=np.uint64), -1.0, 1.0).reshape(nnzb, b * b)


def loss_weights(n: int, b: int, seed: int = 1703) -> np.ndarray:
    """Diagonal loss weights W uniform in [0.5, 1.5] (differentiation workload)."""
    return uniform(seed, STREAM_W, np.arange(n * b, dtype=np.uint64), 0.5, 1.5)


# The workloads, named by what they are.
WORKLOADS = {
    "grid16x16x8_7pt_b3": dict(nx=16, ny=16, nz=8, b=3, stencil=7, sigma=1.0, accum=0.01),
    "grid128x128x64_7pt_b3": dict(nx=128, ny=128, nz=64, b=3, stencil=7, sigma=2.0, accum=1e-3),
    "grid96x96x48_7pt": dict(nx=96, ny=96, nz=48, stencil=7, sigma=1.0, accum=0.01),
    "grid160x160x80_27pt_b3": dict(nx=160, ny=160, nz=80, b=3, stencil=27, sigma=2.5, accum=1e-4),
    "grid64x64x32_7pt_b3": dict(nx=64, ny=64, nz=32, b=3, stencil=7, sigma=1.0, accum=0.01),
}
