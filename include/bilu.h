/*
 * bilu.h -- C ABI of the GB300 (sm_103a) block ILU(k) library.
 *
 * The method is the decoupled block-wise ILU(k) preconditioner of Yang, Liu,
 * Zhong and Chen ("Decoupled Block-Wise ILU(k) Preconditioner on GPU"):
 *   symbolic phase   -- level-of-fill pattern P' of the block graph (Section
 *                       2.2, Algorithm 3, Eq. 1-2) and dependency levels
 *                       (Section 2.4, Eq. 4);
 *   factorization    -- A' = A backfilled onto P' (Algorithm 5), block ILU(0)
 *                       on A' (Algorithm 4) and U = D U' (Eq. 5), D^{-1} stored;
 *   preconditioning  -- L y = r, z = D^{-1} y, U' x = z (Eq. 6, Algorithm 7);
 *   Krylov solve     -- BiCGSTAB (Section 1 names it among the Krylov methods)
 *                       with the block SpMV y = A x.
 *
 * Conventions shared by every call:
 *  - Block CSR (Section 2.1): row_ptr[n+1] and col_idx[nnzb] count blocks;
 *    columns strictly increasing in every row; every row holds its diagonal
 *    block.  Values hold nnzb blocks of b*b doubles, each block stored column
 *    by column: element (r, c) of block t is vals[t*b*b + c*b + r].
 *  - 1 <= b <= 8.  Block rows n < 2^31, pattern sizes < 2^31 blocks.
 *  - "stream" is a cudaStream_t (NULL = legacy default stream).  Every device
 *    call is stream ordered and returns once its work is enqueued unless the
 *    call says it synchronises.
 *  - The caller owns every device buffer passed in (vectors, values, factor
 *    buffer, workspace).  The library allocates device memory only in the
 *    set-up calls bilu_pattern_upload, bilu_pattern_schedule and
 *    bilu_symbolic_gpu, never in factor, apply, SpMV or solve; those read the
 *    pattern's device copy and schedules and modify nothing in the handle, so
 *    several host threads may run them on one pattern at once (set-up calls
 *    on that pattern must not overlap them).
 *  - Pointers prefixed d_ are device pointers on the current device; the
 *    others are host pointers.  Input and output vectors must not alias.
 *  - Every call returns a bilu_status code; no call aborts the process and no
 *    kernel traps: device-side failures are written to an error word in the
 *    workspace and reported by the next call that synchronises.
 */
#ifndef BILU_H
#define BILU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum bilu_status {
  BILU_OK = 0,
  BILU_ERR_ARG = 1,           /* invalid argument (null pointer, bad size, b out of range) */
  BILU_ERR_PATTERN = 2,       /* unsorted/duplicate/out-of-range column or missing diagonal */
  BILU_ERR_SINGULAR = 3,      /* zero or non-finite pivot block D_i; row in the info struct */
  BILU_ERR_BREAKDOWN = 4,     /* BiCGSTAB breakdown: rho, (r_hat, v) or omega became 0 */
  BILU_ERR_NOT_CONVERGED = 5, /* maxit iterations without reaching tol */
  BILU_ERR_TIMEOUT = 6,       /* a bounded dependency wait inside a kernel ran out */
  BILU_ERR_CUDA = 7,          /* a CUDA runtime call failed */
  BILU_ERR_OOM = 8,           /* host or device allocation failed, or a size overflowed */
  BILU_ERR_STATE = 9          /* pattern not uploaded, or workspace too small */
};

/* Static message for a status code; never NULL. */
const char* bilu_status_string(int status);

/* ------------------------------------------------------------------------ */
/* Symbolic phase (host)                                                     */
/* ------------------------------------------------------------------------ */

typedef struct bilu_pattern bilu_pattern; /* opaque, library-owned */

/*
 * bilu_symbolic -- level-of-fill pattern P' of ILU(k) on the block graph.
 * Section 2.3: every listed block of A is one point of the abstract point
 * matrix, whatever its values.  Section 2.2, Algorithm 3 with Eq. 1 (level 0
 * on A's pattern) and Eq. 2 (lev_ij = min(lev_ij, lev_ip + lev_pj + 1) over
 * pivots p < i of level <= k); entries of level <= k are kept.  Also computes
 * the dependency levels of Eq. 4 for the lower and the upper part.
 *   n        number of block rows (>= 0)
 *   row_ptr  host, n+1 entries, row_ptr[0] = 0
 *   col_idx  host, row_ptr[n] entries
 *   k        level of fill, >= 0 (k >= n means complete fill)
 *   out      receives a new handle; free it with bilu_destroy_pattern
 * Returns BILU_ERR_PATTERN for a malformed pattern, BILU_ERR_OOM if P' would
 * exceed 2^31 - 1 blocks.  Host only; touches no GPU state.
 */
int bilu_symbolic(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t k,
                  bilu_pattern** out);

typedef struct {
  int32_t n;       /* block rows */
  int32_t k;       /* level of fill */
  int64_t nnz_a;   /* blocks of A */
  int64_t nnz_p;   /* blocks of P' (lower + diagonal + upper) */
  int64_t nnz_l;   /* strictly lower blocks of P' */
  int64_t nnz_u;   /* strictly upper blocks of P' */
  int32_t nlev_l;  /* number of dependency levels of L (Eq. 4) */
  int32_t nlev_u;  /* number of dependency levels of U' (reversed graph) */
} bilu_pattern_info;

/* Sizes of a pattern.  Host only. */
int bilu_pattern_query(const bilu_pattern* p, bilu_pattern_info* info);

/*
 * bilu_pattern_export -- copy P' out to caller-allocated host arrays:
 *   row_ptr[n+1], col_idx[nnz_p], lev[nnz_p] (level of fill of each entry),
 *   lvl_lower[n], lvl_upper[n] (Eq. 4 levels, 0-based: the paper's l(i) - 1).
 * Any output pointer may be NULL to skip it.  Host only.
 */
int bilu_pattern_export(const bilu_pattern* p, int32_t* row_ptr, int32_t* col_idx, int32_t* lev,
                        int32_t* lvl_lower, int32_t* lvl_upper);

/*
 * bilu_pattern_upload -- copy the pattern's integer structure to the current
 * device and build the schedules of the sync-free factorization and solves
 * (set-up; allocates device memory owned by the handle, about
 * 4*(4n + nnz_l + nnz_u + nnz_a) bytes).  Synchronises the stream.  Needed
 * before bilu_factor, bilu_apply and the solvers, which return
 * BILU_ERR_STATE without it.
 */
int bilu_pattern_upload(bilu_pattern* p, void* stream);

/*
 * bilu_pattern_schedule -- rebuild the uploaded pattern's schedules with the
 * current tuning settings (the chunk targets of include/bilu_tuning.h take
 * effect here and in bilu_pattern_upload, nowhere else).  The paper has no
 * counterpart: a schedule is how the sync-free kernels walk the Eq. 4
 * dependency graph, not what they compute.  Set-up: synchronises the stream,
 * allocates the new schedules before freeing the old ones (on failure the old
 * ones stay), and must not overlap a compute call on the same pattern.
 * BILU_ERR_STATE if the pattern is not uploaded to the current device.
 */
int bilu_pattern_schedule(bilu_pattern* p, void* stream);

/* Rows per chunk of the current solve and factorization schedules (0 when
 * there is none, e.g. before bilu_pattern_upload).  Either output may be
 * NULL.  Host only. */
int bilu_pattern_schedule_info(const bilu_pattern* p, int32_t* solve_rows, int32_t* factor_rows);

/* Frees the handle and its device copy.  NULL is ignored. */
void bilu_destroy_pattern(bilu_pattern* p);

/* ------------------------------------------------------------------------ */
/* Factor buffer layout                                                      */
/* ------------------------------------------------------------------------ */
/*
 * The factors live in ONE caller-allocated device buffer of
 * bilu_factor_bytes(p, b) bytes, b*b doubles per block, in three sections:
 *   [0, nnz_l)                  L_ij, j < i, rows ascending, columns ascending
 *                               (the strictly lower blocks of P');
 *   [nnz_l, nnz_l + n)          D_i^{-1}, one block per row (Eq. 5);
 *   [nnz_l + n, nnz_l + n + nnz_u)  U'_ij = D_i^{-1} U_ij, j > i, rows
 *                               ascending, columns ascending.
 * L and U' have identity diagonal blocks, which are not stored.
 */
size_t bilu_factor_bytes(const bilu_pattern* p, int32_t b);

/* ------------------------------------------------------------------------ */
/* Factorization (device)                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t status;       /* bilu_status of the factorization */
  int32_t bad_row;      /* first block row whose pivot block was singular, else -1 */
  double ms;            /* device time of the factorization (CUDA events) */
} bilu_factor_info;

/* Scratch bytes bilu_factor needs (per-row ready flags and counters). */
size_t bilu_factor_workspace_bytes(const bilu_pattern* p, int32_t b);

/*
 * bilu_factor -- numeric factorization A ~ L D U' on the pattern P'.
 * Algorithm 5 steps 3-5: A' = A with zero fill blocks (backfill), then
 * Algorithm 4 in place, rows ascending, pivots p ascending:
 *   A_ip <- A_ip D_p^{-1};  A_ij <- A_ij - A_ip U_pj  for (i,j),(p,j) in P';
 * then D_i^{-1} (Gauss-Jordan with partial pivoting inside the b x b block)
 * and U'_ij = D_i^{-1} U_ij (Eq. 5).
 *   d_a_vals   device, nnz_a*b*b doubles: A's values on the pattern given to
 *              bilu_symbolic
 *   d_factors  device, bilu_factor_bytes(p, b) bytes, written (layout above)
 *   d_work     device scratch of at least bilu_factor_workspace_bytes bytes;
 *              contents on entry are ignored
 *   info       may be NULL
 * Synchronises the stream to read the device error word.  Returns
 * BILU_ERR_SINGULAR (info->bad_row set) for a zero or non-finite pivot block.
 */
int bilu_factor(const bilu_pattern* p, int32_t b, const double* d_a_vals, double* d_factors,
                void* d_work, size_t work_bytes, void* stream, bilu_factor_info* info);

/* ------------------------------------------------------------------------ */
/* Preconditioner apply (device)                                             */
/* ------------------------------------------------------------------------ */

/* Scratch bytes bilu_apply needs (the intermediate y = L^{-1} r, overwritten
 * by z = D^{-1} y, and counters). */
size_t bilu_apply_workspace_bytes(const bilu_pattern* p, int32_t b);

/*
 * bilu_apply -- x = M^{-1} r with M = L D U' (Eq. 6, Algorithm 7):
 *   L y = r (rows ascending), z = D^{-1} y, U' x = z (rows descending).
 * z = D^{-1} y is a pass of its own between the two solves, in place in the
 * workspace.  Both triangular solves run as single sync-free kernels: each
 * row waits, with a bounded spin, for the rows it depends on.  Allocates
 * nothing and builds nothing: it runs on the schedule of the last
 * bilu_pattern_upload / bilu_pattern_schedule (BILU_ERR_STATE if none).
 *   d_factors  device, output of bilu_factor with the same b
 *   d_r, d_x   device, n*b doubles each; must not alias
 *   d_work     device scratch of at least bilu_apply_workspace_bytes bytes
 * Asynchronous: a dependency wait that times out is recorded in the workspace
 * error word (read it with bilu_workspace_status).
 */
int bilu_apply(const bilu_pattern* p, int32_t b, const double* d_factors, const double* d_r,
               double* d_x, void* d_work, size_t work_bytes, void* stream);

/*
 * bilu_workspace_status -- synchronises the stream and returns the status the
 * most recent bilu_apply on this workspace recorded in its device error word
 * (BILU_OK or BILU_ERR_TIMEOUT).  Every bilu_apply clears the word first.
 */
int bilu_workspace_status(const void* d_work, void* stream);

/*
 * bilu_apply_noalloc -- the same x = M^{-1} r as bilu_apply, for callers that
 * must not allocate device memory: a host program that owns all device memory
 * and gives plugins none of it, or code that cannot afford the device-wide
 * synchronisation a cudaMalloc or cudaFree may cause, so it has no workspace
 * to pass.  The paper has no counterpart; this is a deployment variant.
 *   Scratch: a fixed 32 MiB array inside the library (every GPU that loads
 *   the library holds it until the process exits).  The call allocates
 *   nothing and calls no allocating routine.
 *   Limit: n*b*8 + 256 bytes must fit in 32 MiB (n*b <= 4,194,272);
 *   larger systems return BILU_ERR_STATE without launching anything.
 *   Set-up: the first call on each device looks up the array's device
 *   address (with that device current); make that first call before any
 *   stream capture begins.  The pattern must have been uploaded
 *   (bilu_pattern_upload / bilu_pattern_schedule build the solve order this
 *   call reuses, as bilu_apply does).
 *   Sharing: every call uses the same array, whose contents persist between
 *   calls; each call resets what must start cleared before use.  Calls whose
 *   work overlaps on the GPU (different streams, other threads) race on the
 *   array and give wrong results: serialise them.
 *   Arguments as for bilu_apply, without the workspace.  Asynchronous; a
 *   bounded dependency wait that runs out (which correct use never causes)
 *   is recorded in the scratch's error word: bilu_apply_noalloc_status
 *   reads it.
 */
int bilu_apply_noalloc(const bilu_pattern* p, int32_t b, const double* d_factors, const double* d_r,
                       double* d_x, void* stream);

/*
 * bilu_apply_noalloc_status -- synchronises the stream and returns the status
 * the most recent bilu_apply_noalloc on the current device recorded in the
 * fixed scratch's error word: BILU_OK, or BILU_ERR_TIMEOUT when a bounded
 * dependency wait ran out (x then holds NaN where rows were not solved).
 * Allocates nothing; reads 4 bytes through the scratch address the first
 * bilu_apply_noalloc on this device looked up (BILU_ERR_STATE before any
 * such call).  The paper has no counterpart.
 */
int bilu_apply_noalloc_status(void* stream);

/* ------------------------------------------------------------------------ */
/* Block SpMV (device)                                                       */
/* ------------------------------------------------------------------------ */

/*
 * bsr_spmv -- y = A x for a block CSR matrix (the SpMV Section 2.4 relies
 * on; each block row summed over its blocks in column order).
 *   n, b                 block rows and block size
 *   d_row_ptr, d_col_idx device pattern (as for bilu_symbolic; the diagonal is
 *                        not required here)
 *   d_vals               device, nnzb*b*b doubles
 *   d_x, d_y             device, n*b doubles each; must not alias
 * Asynchronous.
 */
int bsr_spmv(int32_t n, int32_t b, const int32_t* d_row_ptr, const int32_t* d_col_idx,
             const double* d_vals, const double* d_x, double* d_y, void* stream);

/* ------------------------------------------------------------------------ */
/* BiCGSTAB (device)                                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t n;                /* block rows */
  int32_t b;                /* block size */
  const int32_t* row_ptr;   /* device, n+1 */
  const int32_t* col_idx;   /* device, nnzb */
  const double* vals;       /* device, nnzb*b*b, column-major blocks */
} bilu_bsr;

typedef struct {
  int32_t status;           /* bilu_status of the solve */
  int32_t iters;            /* BiCGSTAB iterations (a half iteration counts as one) */
  double true_relres;       /* ||rhs - A x|| / ||rhs|| of the returned x */
  double ms;                /* device time of the solve (CUDA events) */
} bilu_solve_info;

/* Scratch bytes bicgstab_solve needs (eight Krylov vectors, reductions and
 * the apply workspace). */
size_t bicgstab_workspace_bytes(const bilu_pattern* p, int32_t b);

/*
 * bicgstab_solve -- right-preconditioned BiCGSTAB (van der Vorst, as in the
 * Templates book the paper cites) for A x = rhs with M = L D U' from
 * bilu_factor:
 *   r = rhs - A x0, r_hat = r;  each iteration: rho = (r_hat, r);
 *   p = r + beta (p - omega v); p_hat = M^{-1} p; v = A p_hat;
 *   alpha = rho / (r_hat, v); s = r - alpha v (stop if ||s||/||rhs|| <= tol);
 *   s_hat = M^{-1} s; t = A s_hat; omega = (t, s)/(t, t);
 *   x += alpha p_hat + omega s_hat; r = s - omega t.
 * Convergence is declared when the recurrence residual drops below tol AND
 * the recomputed true residual ||rhs - A x||/||rhs|| confirms it; otherwise
 * the iteration restarts from the true residual until maxit is spent.
 *   A          device matrix; A->n and A->b must match the pattern and b
 *   d_factors  output of bilu_factor for the same pattern and b
 *   d_rhs      device, n*b doubles
 *   d_x        device, n*b doubles: x0 on entry, the solution on return
 *   tol        relative residual target (> 0)
 *   maxit      iteration limit (>= 0)
 *   d_work     device scratch of at least bicgstab_workspace_bytes bytes
 *   info       may be NULL
 * Synchronises the stream a few times per iteration batch to test
 * convergence.  Returns BILU_OK, BILU_ERR_NOT_CONVERGED, BILU_ERR_BREAKDOWN or
 * BILU_ERR_TIMEOUT; x holds the last iterate in every case.
 */
int bicgstab_solve(const bilu_pattern* p, const bilu_bsr* A, const double* d_factors,
                   const double* d_rhs, double* d_x, double tol, int32_t maxit, void* d_work,
                   size_t work_bytes, void* stream, bilu_solve_info* info);

/* ------------------------------------------------------------------------ */
/* Mixed precision: FP32-stored preconditioner, FP64 refinement             */
/* ------------------------------------------------------------------------ */
/*
 * The paper works in FP64 throughout (Section 3).  These calls keep L, U' and
 * D^{-1} (and a copy of A for the inner SpMV) in FP32 and apply them in FP32
 * arithmetic, while every Krylov vector, scalar, dot product and the outer
 * residual stay FP64.  Layouts are those of the FP64 calls with float in
 * place of double.
 */

/* Bytes of an FP32 factor buffer (same three sections as bilu_factor_bytes). */
size_t bilu_factor_bytes_f32(const bilu_pattern* p, int32_t b);

/* bilu_factor with every step in FP32: A's FP64 values are rounded to FP32
 * as they are backfilled, and Algorithm 4, the D^{-1} inversion and Eq. 5 run
 * in FP32 arithmetic into an FP32 factor buffer of bilu_factor_bytes_f32
 * bytes.  Same workspace, status and info as bilu_factor. */
int bilu_factor_f32(const bilu_pattern* p, int32_t b, const double* d_a_vals, float* d_factors32,
                    void* d_work, size_t work_bytes, void* stream, bilu_factor_info* info);

/* d_dst[q] = (float)d_src[q] for q < count (device; round to nearest).  Makes
 * the FP32 factor buffer from bilu_factor's output (count = nslots*b*b, i.e.
 * bilu_factor_bytes / 8) and the FP32 copy of A's values.  Asynchronous. */
int bilu_convert_f32(const double* d_src, float* d_dst, int64_t count, void* stream);

/* x = M^{-1} r with the FP32 factors (Eq. 6, Algorithm 7; FP32 products and
 * sums, r read and x written in FP64).  Workspace as for bilu_apply.
 * Asynchronous; status of the bounded waits via bilu_workspace_status. */
int bilu_apply_f32(const bilu_pattern* p, int32_t b, const float* d_factors32, const double* d_r,
                   double* d_x, void* d_work, size_t work_bytes, void* stream);

/* y = A x with A's values in FP32 (FP32 products and sums, each block row
 * summed over its blocks in column order; x read and y written in FP64, x
 * rounded to FP32 to nearest).  Asynchronous. */
int bsr_spmv_f32(int32_t n, int32_t b, const int32_t* d_row_ptr, const int32_t* d_col_idx,
                 const float* d_vals32, const double* d_x, double* d_y, void* stream);

/* y = A x with A's values and x in FP32 (d_x32: device, n*b floats; y in
 * FP64): the products and sums of bsr_spmv_f32, so its y for x equals this
 * call's y for x rounded to FP32.  bicgstab_solve_mixed uses it on the FP32
 * preconditioner's own FP32 result.  Asynchronous. */
int bsr_spmv_f32x(int32_t n, int32_t b, const int32_t* d_row_ptr, const int32_t* d_col_idx,
                  const float* d_vals32, const float* d_x32, double* d_y, void* stream);

/* Scratch bytes bicgstab_solve_mixed needs. */
size_t bicgstab_mixed_workspace_bytes(const bilu_pattern* p, int32_t b);

/*
 * bicgstab_solve_mixed -- iterative refinement around FP32-preconditioned
 * BiCGSTAB:  repeat  r = rhs - A x (FP64 SpMV, A->vals);  stop when
 * ||r||/||rhs|| <= tol;  solve A d = r by BiCGSTAB (the algorithm of
 * bicgstab_solve) with the FP32 SpMV (d_vals32) and the FP32 preconditioner
 * (d_factors32) until its recurrence residual drops by inner_tol or
 * inner_maxit iterations pass;  x += d.
 *   tol in (0, 1), inner_tol in (0, 1), maxit >= 0 (total inner iterations),
 *   inner_maxit >= 1; other arguments as for bicgstab_solve.
 * info->iters counts inner iterations, info->true_relres is the FP64 residual
 * of the returned x.  Synchronises the stream between refinement steps.
 */
int bicgstab_solve_mixed(const bilu_pattern* p, const bilu_bsr* A, const float* d_vals32,
                         const float* d_factors32, const double* d_rhs, double* d_x, double tol,
                         int32_t maxit, double inner_tol, int32_t inner_maxit, void* d_work,
                         size_t work_bytes, void* stream, bilu_solve_info* info);

/*
 * bicgstab_solve_f32prec -- the BiCGSTAB of bicgstab_solve (FP64 SpMV with
 * A->vals, FP64 vectors, scalars, dot products and true residual) with the
 * preconditioner stored and applied in FP32 (d_factors32 from
 * bilu_factor_f32 or bilu_convert_f32).  One Krylov space, no restarts: the
 * FP32 preconditioner changes only how fast the FP64 iteration converges,
 * not the accuracy it reaches.  Workspace: bicgstab_workspace_bytes.  Other
 * arguments and results as for bicgstab_solve.
 */
int bicgstab_solve_f32prec(const bilu_pattern* p, const bilu_bsr* A, const float* d_factors32, const double* d_rhs,
                           double* d_x, double tol, int32_t maxit, void* d_work, size_t work_bytes, void* stream,
                           bilu_solve_info* info);

/* Scratch bytes gmres_solve needs for restart length `restart` (0 for invalid
 * arguments). */
size_t gmres_workspace_bytes(const bilu_pattern* p, int32_t b, int32_t restart);

/*
 * gmres_solve -- restarted GMRES(restart) preconditioned on the right with
 * M = L D U', the solver of the paper's experiments (Section 4 restarts it
 * every 20 iterations).  Each cycle starts from r0 = rhs - A x, builds an
 * Arnoldi basis of A M^{-1} by modified Gram-Schmidt, reduces the Hessenberg
 * matrix with Givens rotations and ends when the least-squares residual is
 * <= tol ||rhs||, when the Krylov space is invariant, after `restart` steps or
 * when maxit steps have been taken in all; then x += M^{-1} V y.  The solve
 * returns BILU_OK once the recomputed true residual ||rhs - A x|| / ||rhs|| <=
 * tol, else starts the next cycle (BILU_ERR_NOT_CONVERGED after maxit steps,
 * BILU_ERR_BREAKDOWN when a cycle makes no step).
 *   restart in [1, 64]; tol in (0, 1); maxit >= 0 counts Arnoldi steps.
 *   Other arguments as for bicgstab_solve; d_work holds
 *   gmres_workspace_bytes(p, A->b, restart) bytes.  info->iters counts
 *   Arnoldi steps.  Synchronises the stream every few steps.
 */
int gmres_solve(const bilu_pattern* p, const bilu_bsr* A, const double* d_factors, const double* d_rhs,
                double* d_x, double tol, int32_t maxit, int32_t restart, void* d_work, size_t work_bytes,
                void* stream, bilu_solve_info* info);

/*
 * bilu_symbolic_gpu -- the same P', fill levels and Eq. 4 levels as
 * bilu_symbolic (bit for bit), computed on the current device: Algorithm 3's
 * row merges with one warp per row (rows in ascending order, row i waiting,
 * bounded, for each pivot row p < i it merges), then the completion of the
 * pattern -- row pointers (device scans), the L / U' split, the Eq. 4 levels
 * (a sync-free longest-path pass per triangle, one warp per row) and the
 * backfill map of Algorithm 5 -- also on the device, straight into the
 * handle's device copy.  Inputs are host arrays as for bilu_symbolic.  The
 * returned handle lives on this device; bilu_pattern_upload on the same
 * device then only builds the schedules.  Its host copy of P' is filled from
 * the device only when a host-side call needs it (bilu_pattern_export,
 * bilu_pattern_transpose, bilu_schedule_export, an upload to another device).
 *   row_capacity in [1, 8192]: the most entries any row of P' may hold; a row
 *   that outgrows it returns BILU_ERR_OOM (retry with a larger capacity).
 *   Device scratch of about 8 * n * row_capacity bytes is allocated and freed
 *   inside the call; the stream is synchronised.  BILU_ERR_TIMEOUT if a wait
 *   exceeds the spin limit (bilu_set_spin_limit_ns).
 */
int bilu_symbolic_gpu(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t k, int32_t row_capacity,
                      void* stream, bilu_pattern** out);

/* ---- adjoint: A^T lambda = g with the transposed factors ----
 *
 * A loss L(x) through x = A^{-1} b has dL/db = lambda and dL/dA_IJ =
 * -lambda_I x_J^T (on A's block pattern), where A^T lambda = dL/dx.  With
 * M = L D U' (Eq. 5-6), M^T = U'^T D^T L^T: the preconditioner of the adjoint
 * solve is the apply of Eq. 6 / Algorithm 7 on the transposed pattern P'^T
 * (whose strictly lower part is U'^T and strictly upper part L^T) with every
 * block transposed, so bilu_apply, bicgstab_solve and bsr_spmv serve the
 * adjoint unchanged once the transposes below exist.
 */

/* The transposed pattern P'^T of p (host; library-owned handle, freed by
 * bilu_destroy_pattern; upload it before use).  It serves bilu_apply,
 * bicgstab_solve and bilu_factor_transpose, not bilu_factor
 * (BILU_ERR_ARG).  p must not itself be a transposed pattern (BILU_ERR_ARG). */
int bilu_pattern_transpose(const bilu_pattern* p, bilu_pattern** out);

/* d_factors_t (device, bilu_factor_bytes(pt, b) bytes, laid out for pt) <-
 * the factors of the source pattern of pt (d_factors, laid out for it) with
 * every block transposed: [U'^T | D^{-T} | L^T].  pt must come from
 * bilu_pattern_transpose and be uploaded (else BILU_ERR_ARG / BILU_ERR_STATE).
 * Asynchronous; d_factors and d_factors_t must not overlap. */
int bilu_factor_transpose(const bilu_pattern* pt, int32_t b, const double* d_factors, double* d_factors_t,
                          void* stream);

/* Transpose of a block CSR pattern (host, caller-allocated): row_ptr_t[n+1],
 * col_idx_t[nnzb] (sorted rows) and perm[nnzb], the block of A that block t
 * of A^T transposes.  BILU_ERR_PATTERN for an invalid row_ptr or column. */
int bsr_transpose_pattern(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* row_ptr_t,
                          int32_t* col_idx_t, int32_t* perm);

/* d_dst block t <- (d_src block d_perm[t])^T for t < nblocks (device arrays;
 * b x b column-major blocks; A^T's values from A's with perm from
 * bsr_transpose_pattern).  Indices are not checked on the device.
 * Asynchronous; d_src and d_dst must not overlap. */
int bsr_gather_transpose(int64_t nblocks, int32_t b, const int32_t* d_perm, const double* d_src, double* d_dst,
                         void* stream);

/* d_grad block t (row I, column J = col_idx[t]) <- -lambda_I x_J^T: the
 * gradient of a loss with respect to A's blocks, given the adjoint solution
 * lambda and the solution x (device arrays, n*b doubles each; d_grad has
 * nnzb*b*b doubles).  Asynchronous. */
int bsr_outer_grad(int32_t n, int32_t b, const int32_t* d_row_ptr, const int32_t* d_col_idx,
                   const double* d_lambda, const double* d_x, double* d_grad, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BILU_H */
