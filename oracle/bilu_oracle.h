/*
 * bilu_oracle.h -- CPU oracle for the decoupled block-wise ILU(k) method
 * (Yang, Liu, Zhong, Chen, "Decoupled Block-Wise ILU(k) Preconditioner on GPU").
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, single-threaded fp64
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header or constant with the CUDA library and must never serve as a
 * fallback for it.
 *
 * Storage (Section 2.1): block CSR.  rp[n+1] row starts (in blocks), ci[nnzb]
 * block column indices (sorted, unique, diagonal present), values hold nnzb
 * blocks of b*b doubles, each block stored column by column: element (r,c) of
 * block t is vals[t*b*b + c*b + r].
 *
 * Readings of the paper that this oracle follows (each is also listed in the
 * design notes):
 *   - level symbol of Eq. 1-2 is a level of fill, not the factor L;
 *   - an entry is kept iff its level <= k (k = 0 gives ILU(0));
 *   - Algorithm 3's drop test is applied once the row is complete;
 *   - Algorithm 3's full n x n start pattern is realised as a sparse sorted
 *     row merge that produces the identical set; only j in P'(p) are visited
 *     because every other j gets a level > k;
 *   - "nonzero block" is structural (listed in Ap/Aj), whatever its values;
 *   - Algorithm 4's A_pp^{-1} is row p's already-updated diagonal block D_p,
 *     with no block pivoting; the b x b inverse uses Gauss-Jordan with partial
 *     pivoting inside the block;
 *   - dependency levels (Eq. 4) are exported 0-based (paper level - 1).
 */
#ifndef BILU_ORACLE_H
#define BILU_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  OR_OK = 0,
  OR_ERR_ARG = 1,
  OR_ERR_PATTERN = 2,
  OR_ERR_SINGULAR = 3,
  OR_ERR_BREAKDOWN = 4,
  OR_ERR_NOT_CONVERGED = 5,
  OR_ERR_OOM = 6
};

/* Structural checks on (rp, ci): rp monotone from 0, columns in range, strictly
 * increasing per row, diagonal present in every row.  Returns OR_OK or
 * OR_ERR_PATTERN / OR_ERR_ARG. */
int or_check_pattern(int32_t n, const int32_t* rp, const int32_t* ci);

/* Symbolic phase, Algorithm 3 with Eq. 1 (initial levels) and Eq. 2 (level
 * update).  Output: the level-<=k pattern P' as CSR with the level of every
 * entry.  *prp, *pci, *plev are malloc'd here; free with or_free. */
int or_symbolic(int32_t n, const int32_t* rp, const int32_t* ci, int32_t k,
                int32_t** prp, int32_t** pci, int32_t** plev);

/* Eq. 4: lvl_lower[i] over P'(i) columns j < i (rows ascending), lvl_upper[i]
 * over columns j > i (rows descending, the reversed graph).  0-based. */
int or_levels(int32_t n, const int32_t* prp, const int32_t* pci,
              int32_t* lvl_lower, int32_t* lvl_upper);

/* Algorithm 5 steps 3-4: copy A's blocks into A' (pattern P'), zero blocks at
 * the fill positions.  Every A position must be in P'. */
int or_backfill(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci,
                const double* vals, const int32_t* prp, const int32_t* pci,
                double* fvals);

/* Algorithm 4 on A' in place, then Eq. 5.  On return fvals holds, per block:
 * L_ij (j < i), D_i = the factored pivot block (j = i), U'_ij = D_i^{-1} U_ij
 * (j > i); dinv holds D_i^{-1} for every row (n*b*b doubles).  On a singular
 * or non-finite pivot block returns OR_ERR_SINGULAR with *bad_row set. */
int or_factor(int32_t n, int32_t b, const int32_t* prp, const int32_t* pci,
              double* fvals, double* dinv, int32_t* bad_row);

/* Eq. 6 / Algorithm 7: L y = r, z = D^{-1} y, U' x = z.  r and x: n*b. */
int or_apply(int32_t n, int32_t b, const int32_t* prp, const int32_t* pci,
             const double* fvals, const double* dinv, const double* r, double* x);

/* y = A x, each block row summed in column order. */
int or_spmv(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci,
            const double* vals, const double* x, double* y);

/* Right-preconditioned BiCGSTAB (the Templates book, cited in Section 1),
 * preconditioner M = L D U' from or_factor.  x holds x0 on entry.  Stops when
 * the recurrence residual ||r||/||b|| <= tol and the recomputed true residual
 * confirms it; otherwise restarts from r = b - A x until maxit iterations are
 * spent.  *iters counts full or half iterations; *relres is the true relative
 * residual of the returned x. */
int or_bicgstab(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci,
                const double* vals, const int32_t* prp, const int32_t* pci,
                const double* fvals, const double* dinv, const double* rhs,
                double* x, double tol, int32_t maxit, int32_t* iters,
                double* relres);

/* Restarted GMRES(m) preconditioned on the right with M = L D U' -- the
 * solver of the paper's experiments (Section 4: GMRES restarted every 20
 * iterations).  Each cycle: r0 = b - A x, beta = ||r0||, v_1 = r0 / beta;
 * for j = 1..m the Arnoldi step w = A M^{-1} v_j orthogonalised by modified
 * Gram-Schmidt (h_ij = (w, v_i), w -= h_ij v_i for i = 1..j, in order),
 * h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}; Givens rotations reduce H to
 * upper triangular form and |g_{j+1}| is the residual norm of the least
 * squares problem min ||beta e_1 - H y||.  The cycle ends when |g_{j+1}| <=
 * tol ||b||, when h_{j+1,j} = 0, after m steps, or when maxit steps have been
 * taken in all; then y solves the triangular system and x += M^{-1} (V y).
 * The solve stops once the recomputed true residual ||b - A x|| / ||b|| <=
 * tol, otherwise the next cycle starts from it.  *iters counts Arnoldi steps;
 * *relres is the true relative residual of the returned x.  1 <= m <= 64. */
int or_gmres(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci,
             const double* vals, const int32_t* prp, const int32_t* pci,
             const double* fvals, const double* dinv, const double* rhs,
             double* x, double tol, int32_t maxit, int32_t m, int32_t* iters,
             double* relres);

void or_free(void* p);

#ifdef __cplusplus
}
#endif
#endif
