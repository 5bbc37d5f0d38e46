/*
 * bilu_oracle.c -- CPU oracle (TEST INFRASTRUCTURE ONLY; see bilu_oracle.h).
 *
 * Plain single-threaded C in fp64, compiled with -ffp-contract=off so that no
 * multiply-add is fused and results do not depend on the host ISA.  Each
 * function follows one passage of the paper in the paper's order of
 * operations; nothing is blocked, fused or reordered.
 */
#include "bilu_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

void or_free(void* p) { free(p); }

int or_check_pattern(int32_t n, const int32_t* rp, const int32_t* ci) {
  if (n < 0 || (n > 0 && (!rp || !ci))) return OR_ERR_ARG;
  if (n == 0) return OR_OK;
  if (rp[0] != 0) return OR_ERR_PATTERN;
  for (int32_t i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return OR_ERR_PATTERN;
    int has_diag = 0;
    for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
      if (ci[t] < 0 || ci[t] >= n) return OR_ERR_PATTERN;
      if (t > rp[i] && ci[t] <= ci[t - 1]) return OR_ERR_PATTERN;
      if (ci[t] == i) has_diag = 1;
    }
    if (!has_diag) return OR_ERR_PATTERN;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Symbolic phase: Algorithm 3, Eq. 1 and Eq. 2.                              */
/*                                                                           */
/* Row i starts from Eq. 1: level 0 on A's pattern, "infinity" elsewhere.    */
/* Columns p < i are taken in ascending order; those with level <= k act as   */
/* pivots and apply Eq. 2 to every j > p: lev_ij = min(lev_ij, lev_ip +       */
/* lev_pj + 1).  Only j in the final P'(p) can give a value <= k, so only     */
/* those are visited, and a candidate above k is never recorded (it could     */
/* only be dropped at the end).  A fill j with p < j < i joins the row and is */
/* itself visited as a pivot later, exactly as in the dense loop over p.      */
/* The row kept is {j : lev_ij <= k}.  The current row is a sorted linked     */
/* list over column indices (next[]), the sparse stand-in for the paper's     */
/* full n x n starting pattern.                                               */
/* ------------------------------------------------------------------------- */
int or_symbolic(int32_t n, const int32_t* rp, const int32_t* ci, int32_t k,
                int32_t** prp_out, int32_t** pci_out, int32_t** plev_out) {
  if (!prp_out || !pci_out || !plev_out || k < 0) return OR_ERR_ARG;
  int st = or_check_pattern(n, rp, ci);
  if (st != OR_OK) return st;
  int32_t* prp = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  size_t cap = (n > 0 ? (size_t)rp[n] : 0) * 2 + 16;
  int32_t* pci = (int32_t*)malloc(sizeof(int32_t) * cap);
  int32_t* plev = (int32_t*)malloc(sizeof(int32_t) * cap);
  int32_t* lev = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  if (!prp || !pci || !plev || !lev || !next) {
    free(prp); free(pci); free(plev); free(lev); free(next);
    return OR_ERR_OOM;
  }
  size_t nnz = 0;
  prp[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    /* Eq. 1: the row of A, all at level 0, as a sorted list. */
    int32_t head = -1, tail = -1;
    for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
      int32_t j = ci[t];
      lev[j] = 0;
      next[j] = -1;
      if (tail < 0) head = j; else next[tail] = j;
      tail = j;
    }
    /* Pivots p < i in ascending order (the list grows behind p). */
    for (int32_t p = head; p != -1 && p < i; p = next[p]) {
      if (lev[p] > k) continue; /* never true: only levels <= k are listed */
      int32_t cursor = p;       /* list node with column < every j below */
      for (int32_t t = prp[p]; t < prp[p + 1]; ++t) {
        int32_t j = pci[t];
        if (j <= p) continue;
        int64_t cand = (int64_t)lev[p] + (int64_t)plev[t] + 1; /* Eq. 2 */
        if (cand > k) continue;
        while (next[cursor] != -1 && next[cursor] < j) cursor = next[cursor];
        if (next[cursor] == j) {
          if (cand < lev[j]) lev[j] = (int32_t)cand;
        } else { /* new fill position */
          next[j] = next[cursor];
          next[cursor] = j;
          lev[j] = (int32_t)cand;
        }
        cursor = j;
      }
    }
    /* Emit P'(i) = {j : lev_ij <= k}, sorted. */
    for (int32_t j = head; j != -1; j = next[j]) {
      if (nnz == cap) {
        cap *= 2;
        int32_t* a = (int32_t*)realloc(pci, sizeof(int32_t) * cap);
        if (!a) { free(prp); free(pci); free(plev); free(lev); free(next); return OR_ERR_OOM; }
        pci = a;
        int32_t* c = (int32_t*)realloc(plev, sizeof(int32_t) * cap);
        if (!c) { free(prp); free(pci); free(plev); free(lev); free(next); return OR_ERR_OOM; }
        plev = c;
      }
      pci[nnz] = j;
      plev[nnz] = lev[j];
      ++nnz;
    }
    if (nnz > (size_t)INT32_MAX) {
      free(prp); free(pci); free(plev); free(lev); free(next);
      return OR_ERR_OOM;
    }
    prp[i + 1] = (int32_t)nnz;
  }
  free(lev);
  free(next);
  *prp_out = prp;
  *pci_out = pci;
  *plev_out = plev;
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Eq. 4: l(i) = 1 + max_j l(j) over j with L_ij != 0 (structurally), level   */
/* of a row with no such j is the starting value.  Stored 0-based.  The upper */
/* solve uses the same rule on the reversed graph (rows descending, j > i).   */
/* ------------------------------------------------------------------------- */
int or_levels(int32_t n, const int32_t* prp, const int32_t* pci,
              int32_t* lvl_lower, int32_t* lvl_upper) {
  if (n < 0 || (n > 0 && (!prp || !pci || !lvl_lower || !lvl_upper))) return OR_ERR_ARG;
  for (int32_t i = 0; i < n; ++i) {
    int32_t l = 0;
    for (int32_t t = prp[i]; t < prp[i + 1]; ++t) {
      int32_t j = pci[t];
      if (j < i && lvl_lower[j] + 1 > l) l = lvl_lower[j] + 1;
    }
    lvl_lower[i] = l;
  }
  for (int32_t i = n - 1; i >= 0; --i) {
    int32_t l = 0;
    for (int32_t t = prp[i]; t < prp[i + 1]; ++t) {
      int32_t j = pci[t];
      if (j > i && lvl_upper[j] + 1 > l) l = lvl_upper[j] + 1;
    }
    lvl_upper[i] = l;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 5, steps 3-4: backfill A into A' and zero the fill positions.   */
/* ------------------------------------------------------------------------- */
int or_backfill(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci,
                const double* vals, const int32_t* prp, const int32_t* pci,
                double* fvals) {
  if (n < 0 || b < 1) return OR_ERR_ARG;
  size_t bb = (size_t)b * b;
  for (int32_t i = 0; i < n; ++i) {
    for (int32_t u = prp[i]; u < prp[i + 1]; ++u)
      for (size_t e = 0; e < bb; ++e) fvals[(size_t)u * bb + e] = 0.0;
    for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
      int32_t u = prp[i];
      while (u < prp[i + 1] && pci[u] != ci[t]) ++u;
      if (u == prp[i + 1]) return OR_ERR_PATTERN; /* A entry missing from P' */
      for (size_t e = 0; e < bb; ++e) fvals[(size_t)u * bb + e] = vals[(size_t)t * bb + e];
    }
  }
  return OR_OK;
}

/* Dense b x b helpers, column-major, sums over the inner index ascending. */
static void blk_copy(int32_t b, const double* x, double* z) {
  for (int32_t e = 0; e < b * b; ++e) z[e] = x[e];
}

/* z = x * y */
static void blk_mul(int32_t b, const double* x, const double* y, double* z) {
  for (int32_t c = 0; c < b; ++c)
    for (int32_t r = 0; r < b; ++r) {
      double s = 0.0;
      for (int32_t m = 0; m < b; ++m) s += x[m * b + r] * y[c * b + m];
      z[c * b + r] = s;
    }
}

/* z = z - x * y */
static void blk_sub_mul(int32_t b, const double* x, const double* y, double* z) {
  for (int32_t c = 0; c < b; ++c)
    for (int32_t r = 0; r < b; ++r) {
      double s = 0.0;
      for (int32_t m = 0; m < b; ++m) s += x[m * b + r] * y[c * b + m];
      z[c * b + r] -= s;
    }
}

/* Inverse by Gauss-Jordan elimination with partial (row) pivoting on [D | I].
 * Returns 1 if a pivot is zero or any value is not finite. */
static int blk_inverse(int32_t b, const double* d, double* dinv) {
  double m[64], w[64];
  for (int32_t e = 0; e < b * b; ++e) {
    if (!isfinite(d[e])) return 1;
    m[e] = d[e];
    w[e] = 0.0;
  }
  for (int32_t r = 0; r < b; ++r) w[r * b + r] = 1.0;
  for (int32_t c = 0; c < b; ++c) {
    int32_t pr = c;
    double best = fabs(m[c * b + c]);
    for (int32_t r = c + 1; r < b; ++r)
      if (fabs(m[c * b + r]) > best) { best = fabs(m[c * b + r]); pr = r; }
    if (!(best > 0.0)) return 1;
    if (pr != c)
      for (int32_t q = 0; q < b; ++q) {
        double t = m[q * b + c]; m[q * b + c] = m[q * b + pr]; m[q * b + pr] = t;
        t = w[q * b + c]; w[q * b + c] = w[q * b + pr]; w[q * b + pr] = t;
      }
    double piv = m[c * b + c];
    for (int32_t q = 0; q < b; ++q) {
      m[q * b + c] /= piv;
      w[q * b + c] /= piv;
    }
    for (int32_t r = 0; r < b; ++r) {
      if (r == c) continue;
      double f = m[c * b + r];
      if (f == 0.0) continue;
      for (int32_t q = 0; q < b; ++q) {
        m[q * b + r] -= f * m[q * b + c];
        w[q * b + r] -= f * w[q * b + c];
      }
    }
  }
  for (int32_t e = 0; e < b * b; ++e) {
    if (!isfinite(w[e])) return 1;
    dinv[e] = w[e];
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 4 (block ILU(0) on A' over P'), then Eq. 5 (U = D U').          */
/*   for i ascending:                                                        */
/*     for p < i in P'(i), ascending:                                        */
/*       A_ip <- A_ip * A_pp^{-1}           (A_pp = row p's final pivot D_p) */
/*       for j > p with (i,j) in P' and (p,j) in P':                          */
/*         A_ij <- A_ij - A_ip * A_pj        (A_pj = row p's unscaled U)      */
/*     D_i = A_ii, store D_i^{-1}                                            */
/*   then U'_ij = D_i^{-1} U_ij for every j > i (after all rows, because     */
/*   later rows need the unscaled U_pj).                                      */
/* ------------------------------------------------------------------------- */
int or_factor(int32_t n, int32_t b, const int32_t* prp, const int32_t* pci,
              double* fvals, double* dinv, int32_t* bad_row) {
  if (n < 0 || b < 1 || b > 8) return OR_ERR_ARG;
  if (bad_row) *bad_row = -1;
  size_t bb = (size_t)b * b;
  int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  if (!pos) return OR_ERR_OOM;
  for (int32_t j = 0; j < n; ++j) pos[j] = -1;
  double tmp[64];
  for (int32_t i = 0; i < n; ++i) {
    for (int32_t u = prp[i]; u < prp[i + 1]; ++u) pos[pci[u]] = u;
    int32_t diag = pos[i];
    for (int32_t t = prp[i]; t < prp[i + 1] && pci[t] < i; ++t) {
      int32_t p = pci[t];
      double* aip = fvals + (size_t)t * bb;
      blk_mul(b, aip, dinv + (size_t)p * bb, tmp);
      blk_copy(b, tmp, aip);
      for (int32_t s = prp[p]; s < prp[p + 1]; ++s) {
        int32_t j = pci[s];
        if (j <= p) continue;
        int32_t u = pos[j];
        if (u < 0) continue;
        blk_sub_mul(b, aip, fvals + (size_t)s * bb, fvals + (size_t)u * bb);
      }
    }
    if (diag < 0 || blk_inverse(b, fvals + (size_t)diag * bb, dinv + (size_t)i * bb)) {
      if (bad_row) *bad_row = i;
      for (int32_t u = prp[i]; u < prp[i + 1]; ++u) pos[pci[u]] = -1;
      free(pos);
      return OR_ERR_SINGULAR;
    }
    for (int32_t u = prp[i]; u < prp[i + 1]; ++u) pos[pci[u]] = -1;
  }
  free(pos);
  /* Eq. 5: U' = D^{-1} U. */
  for (int32_t i = 0; i < n; ++i)
    for (int32_t u = prp[i]; u < prp[i + 1]; ++u) {
      if (pci[u] <= i) continue;
      blk_mul(b, dinv + (size_t)i * bb, fvals + (size_t)u * bb, tmp);
      blk_copy(b, tmp, fvals + (size_t)u * bb);
    }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Eq. 6 / Algorithm 7: three separate steps.                                */
/* ------------------------------------------------------------------------- */
int or_apply(int32_t n, int32_t b, const int32_t* prp, const int32_t* pci,
             const double* fvals, const double* dinv, const double* r, double* x) {
  if (n < 0 || b < 1 || b > 8) return OR_ERR_ARG;
  size_t bb = (size_t)b * b;
  double* y = (double*)malloc(sizeof(double) * ((size_t)n * b + 1));
  double* z = (double*)malloc(sizeof(double) * ((size_t)n * b + 1));
  if (!y || !z) { free(y); free(z); return OR_ERR_OOM; }
  /* L y = r, rows ascending (L has identity diagonal blocks). */
  for (int32_t i = 0; i < n; ++i) {
    double* yi = y + (size_t)i * b;
    for (int32_t r0 = 0; r0 < b; ++r0) yi[r0] = r[(size_t)i * b + r0];
    for (int32_t t = prp[i]; t < prp[i + 1] && pci[t] < i; ++t) {
      const double* l = fvals + (size_t)t * bb;
      const double* yj = y + (size_t)pci[t] * b;
      for (int32_t r0 = 0; r0 < b; ++r0) {
        double s = 0.0;
        for (int32_t c = 0; c < b; ++c) s += l[c * b + r0] * yj[c];
        yi[r0] -= s;
      }
    }
  }
  /* z = D^{-1} y. */
  for (int32_t i = 0; i < n; ++i) {
    const double* d = dinv + (size_t)i * bb;
    for (int32_t r0 = 0; r0 < b; ++r0) {
      double s = 0.0;
      for (int32_t c = 0; c < b; ++c) s += d[c * b + r0] * y[(size_t)i * b + c];
      z[(size_t)i * b + r0] = s;
    }
  }
  /* U' x = z, rows descending (U' has identity diagonal blocks). */
  for (int32_t i = n - 1; i >= 0; --i) {
    double* xi = x + (size_t)i * b;
    for (int32_t r0 = 0; r0 < b; ++r0) xi[r0] = z[(size_t)i * b + r0];
    for (int32_t t = prp[i]; t < prp[i + 1]; ++t) {
      if (pci[t] <= i) continue;
      const double* u = fvals + (size_t)t * bb;
      const double* xj = x + (size_t)pci[t] * b;
      for (int32_t r0 = 0; r0 < b; ++r0) {
        double s = 0.0;
        for (int32_t c = 0; c < b; ++c) s += u[c * b + r0] * xj[c];
        xi[r0] -= s;
      }
    }
  }
  free(y);
  free(z);
  return OR_OK;
}

int or_spmv(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci,
            const double* vals, const double* x, double* y) {
  if (n < 0 || b < 1) return OR_ERR_ARG;
  size_t bb = (size_t)b * b;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t r0 = 0; r0 < b; ++r0) {
      double s = 0.0;
      for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
        const double* a = vals + (size_t)t * bb;
        const double* xj = x + (size_t)ci[t] * b;
        for (int32_t c = 0; c < b; ++c) s += a[c * b + r0] * xj[c];
      }
      y[(size_t)i * b + r0] = s;
    }
  return OR_OK;
}

static double vdot(size_t m, const double* a, const double* c) {
  double s = 0.0;
  for (size_t q = 0; q < m; ++q) s += a[q] * c[q];
  return s;
}

/* ------------------------------------------------------------------------- */
/* Preconditioned BiCGSTAB (van der Vorst), as printed in the Templates book */
/* that Section 1 cites for it, with the preconditioner applied on the right  */
/* (p_hat = M^{-1} p, s_hat = M^{-1} s, x updated with p_hat and s_hat).       */
/* ------------------------------------------------------------------------- */
int or_bicgstab(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci,
                const double* vals, const int32_t* prp, const int32_t* pci,
                const double* fvals, const double* dinv, const double* rhs,
                double* x, double tol, int32_t maxit, int32_t* iters,
                double* relres) {
  if (n < 0 || b < 1 || b > 8 || maxit < 0 || !(tol >= 0.0)) return OR_ERR_ARG;
  size_t m = (size_t)n * b;
  *iters = 0;
  *relres = 0.0;
  double bnorm = sqrt(vdot(m, rhs, rhs));
  if (bnorm == 0.0) {
    for (size_t q = 0; q < m; ++q) x[q] = 0.0;
    return OR_OK;
  }
  double* buf = (double*)malloc(sizeof(double) * (8 * m + 8));
  if (!buf) return OR_ERR_OOM;
  double *r = buf, *rh = r + m, *p = rh + m, *v = p + m, *ph = v + m, *s = ph + m,
         *sh = s + m, *t = sh + m;
  int status = OR_ERR_NOT_CONVERGED;
  int32_t it = 0;
  for (;;) { /* (re)start from the true residual */
    or_spmv(n, b, rp, ci, vals, x, r);
    for (size_t q = 0; q < m; ++q) { r[q] = rhs[q] - r[q]; rh[q] = r[q]; p[q] = 0.0; v[q] = 0.0; }
    double rnorm = sqrt(vdot(m, r, r));
    *relres = rnorm / bnorm;
    if (*relres <= tol) { status = OR_OK; break; }
    if (it >= maxit) { status = OR_ERR_NOT_CONVERGED; break; }
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    int converged = 0, broke = 0;
    while (it < maxit) {
      double rho = vdot(m, rh, r);
      if (rho == 0.0) { broke = 1; break; }
      double beta = (rho / rho_prev) * (alpha / omega);
      for (size_t q = 0; q < m; ++q) p[q] = r[q] + beta * (p[q] - omega * v[q]);
      or_apply(n, b, prp, pci, fvals, dinv, p, ph);
      or_spmv(n, b, rp, ci, vals, ph, v);
      double rv = vdot(m, rh, v);
      if (rv == 0.0) { broke = 1; break; }
      alpha = rho / rv;
      for (size_t q = 0; q < m; ++q) s[q] = r[q] - alpha * v[q];
      ++it;
      if (sqrt(vdot(m, s, s)) / bnorm <= tol) {
        for (size_t q = 0; q < m; ++q) x[q] += alpha * ph[q];
        converged = 1;
        break;
      }
      or_apply(n, b, prp, pci, fvals, dinv, s, sh);
      or_spmv(n, b, rp, ci, vals, sh, t);
      double tt = vdot(m, t, t);
      if (tt == 0.0) { broke = 1; break; }
      omega = vdot(m, t, s) / tt;
      for (size_t q = 0; q < m; ++q) x[q] += alpha * ph[q] + omega * sh[q];
      for (size_t q = 0; q < m; ++q) r[q] = s[q] - omega * t[q];
      if (sqrt(vdot(m, r, r)) / bnorm <= tol) { converged = 1; break; }
      if (omega == 0.0) { broke = 1; break; }
      rho_prev = rho;
    }
    /* True residual of the current x. */
    or_spmv(n, b, rp, ci, vals, x, t);
    for (size_t q = 0; q < m; ++q) t[q] = rhs[q] - t[q];
    *relres = sqrt(vdot(m, t, t)) / bnorm;
    if (*relres <= tol) { status = OR_OK; break; }
    if (broke && !converged) { status = OR_ERR_BREAKDOWN; break; }
    if (it >= maxit) { status = OR_ERR_NOT_CONVERGED; break; }
    /* recurrence said converged but the true residual did not: restart */
  }
  *iters = it;
  free(buf);
  return status;
}

/* ------------------------------------------------------------------------- */
/* Restarted GMRES(m), right preconditioning (see bilu_oracle.h).             */
/* ------------------------------------------------------------------------- */
int or_gmres(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci,
             const double* vals, const int32_t* prp, const int32_t* pci,
             const double* fvals, const double* dinv, const double* rhs,
             double* x, double tol, int32_t maxit, int32_t m, int32_t* iters,
             double* relres) {
  if (n < 0 || b < 1 || b > 8 || maxit < 0 || m < 1 || m > 64 || !(tol >= 0.0)) return OR_ERR_ARG;
  size_t len = (size_t)n * b;
  *iters = 0;
  *relres = 0.0;
  double bnorm = sqrt(vdot(len, rhs, rhs));
  if (bnorm == 0.0) {
    for (size_t q = 0; q < len; ++q) x[q] = 0.0;
    return OR_OK;
  }
  /* V: m+1 basis vectors; w, z, u: work vectors; H column-major (m+1) x m */
  double* buf = (double*)malloc(sizeof(double) * ((size_t)(m + 4) * len + 8));
  double* H = (double*)malloc(sizeof(double) * (size_t)(m + 1) * m);
  double* cs = (double*)malloc(sizeof(double) * (size_t)m);
  double* sn = (double*)malloc(sizeof(double) * (size_t)m);
  double* g = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* y = (double*)malloc(sizeof(double) * (size_t)m);
  if (!buf || !H || !cs || !sn || !g || !y) {
    free(buf); free(H); free(cs); free(sn); free(g); free(y);
    return OR_ERR_OOM;
  }
  double* V = buf;
  double* w = V + (size_t)(m + 1) * len;
  double* z = w + len;
  double* u = z + len;
  int status = OR_ERR_NOT_CONVERGED;
  int32_t it = 0;
  for (;;) {
    /* r0 = b - A x */
    or_spmv(n, b, rp, ci, vals, x, w);
    for (size_t q = 0; q < len; ++q) w[q] = rhs[q] - w[q];
    double beta = sqrt(vdot(len, w, w));
    *relres = beta / bnorm;
    if (*relres <= tol) { status = OR_OK; break; }
    if (it >= maxit) { status = OR_ERR_NOT_CONVERGED; break; }
    for (size_t q = 0; q < len; ++q) V[q] = w[q] / beta;
    for (int32_t q = 0; q <= m; ++q) g[q] = 0.0;
    g[0] = beta;
    int32_t k = 0; /* columns of this cycle */
    while (k < m && it < maxit) {
      int32_t j = k;
      double* vj = V + (size_t)j * len;
      or_apply(n, b, prp, pci, fvals, dinv, vj, z);
      or_spmv(n, b, rp, ci, vals, z, w);
      double* hj = H + (size_t)j * (m + 1);
      for (int32_t i = 0; i <= j; ++i) { /* modified Gram-Schmidt */
        const double* vi = V + (size_t)i * len;
        hj[i] = vdot(len, w, vi);
        for (size_t q = 0; q < len; ++q) w[q] -= hj[i] * vi[q];
      }
      hj[j + 1] = sqrt(vdot(len, w, w));
      /* previous rotations on column j, then the new one */
      for (int32_t i = 0; i < j; ++i) {
        double a = hj[i], c = hj[i + 1];
        hj[i] = cs[i] * a + sn[i] * c;
        hj[i + 1] = -sn[i] * a + cs[i] * c;
      }
      double a = hj[j], c = hj[j + 1];
      double rho = sqrt(a * a + c * c);
      ++it;
      k = j + 1;
      if (rho == 0.0) { k = j; break; } /* w and v_j both vanish: no progress */
      cs[j] = a / rho;
      sn[j] = c / rho;
      hj[j] = rho;
      hj[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      if (fabs(g[j + 1]) <= tol * bnorm) break;
      if (c == 0.0) break; /* h_{j+1,j} = 0: the Krylov space is invariant */
      double* vn = V + (size_t)(j + 1) * len;
      for (size_t q = 0; q < len; ++q) vn[q] = w[q] / c;
    }
    if (k == 0) { status = OR_ERR_BREAKDOWN; break; }
    /* y = R^{-1} g by back substitution; u = V y; x += M^{-1} u */
    for (int32_t i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int32_t l = i + 1; l < k; ++l) s -= H[(size_t)l * (m + 1) + i] * y[l];
      y[i] = s / H[(size_t)i * (m + 1) + i];
    }
    for (size_t q = 0; q < len; ++q) u[q] = 0.0;
    for (int32_t i = 0; i < k; ++i) {
      const double* vi = V + (size_t)i * len;
      for (size_t q = 0; q < len; ++q) u[q] += y[i] * vi[q];
    }
    or_apply(n, b, prp, pci, fvals, dinv, u, z);
    for (size_t q = 0; q < len; ++q) x[q] += z[q];
  }
  *iters = it;
  free(buf); free(H); free(cs); free(sn); free(g); free(y);
  return status;
}
