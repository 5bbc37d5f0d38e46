// krylov.cu -- right-preconditioned BiCGSTAB on the device.
//
// The iteration is van der Vorst's BiCGSTAB as printed in the Templates book
// (the paper cites it for BiCGSTAB in Section 1), preconditioned on the right
// with M = L D U':
//   r = rhs - A x0, r_hat = r, rho_prev = alpha = omega = 1, p = v = 0
//   loop: rho = (r_hat, r); beta = (rho/rho_prev)(alpha/omega)
//         p = r + beta (p - omega v); p_hat = M^{-1} p; v = A p_hat
//         alpha = rho / (r_hat, v); s = r - alpha v; x += alpha p_hat
//         stop if ||s|| <= tol ||rhs||
//         s_hat = M^{-1} s; t = A s_hat; omega = (t, s)/(t, t)
//         x += omega s_hat; r = s - omega t; stop if ||r|| <= tol ||rhs||
// (x is advanced in two halves, alpha p_hat then omega s_hat, which equals the
// book's single update up to rounding.)  Scalars live in device memory; every
// kernel of an iteration returns at once when the device stop word is set, so
// the host can enqueue several iterations and look at the state only between
// batches.  Dot products reduce in two deterministic stages (fixed grid of
// per-block partial sums, then one block), so a run is bitwise reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <functional>

#include "device_common.cuh"

namespace bilu {
namespace {

constexpr int kRedBlocks = 608;  // partial sums per dot product
constexpr int kRedThreads = 256;

enum Reason : int { kRunning = 0, kConverged = 1, kBreakdown = 2, kMaxit = 3 };

struct KState {
  double rho, rho_prev, alpha, omega;
  double bnorm2, thresh2;  // ||rhs||^2 and (tol ||rhs||)^2
  double last2;            // last squared residual norm the recurrences produced
  double true2;            // squared true residual norm (after the loop)
  int stop, reason, iters, maxit;
};

__device__ __forceinline__ bool stopped(const KState* st) {
  return ld_volatile_s32(&st->stop) != 0;
}

template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* partials) {
  __shared__ double red[NV][kRedThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v[q] += __shfl_down_sync(kFull, v[q], d);
    if (lane == 0) red[q][wid] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int k = 0; k < kRedThreads / 32; ++k) s += red[threadIdx.x][k];
    partials[threadIdx.x * kRedBlocks + blockIdx.x] = s;
  }
}

// r = rhs - t, r_hat = r, p = v = 0; partials: (r, r), (rhs, rhs)
__global__ void k_init(long long m, const double* rhs, const double* t, double* r, double* rh,
                       double* p, double* v, double* partials) {
  double acc[2] = {0.0, 0.0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (long long)gridDim.x * blockDim.x) {
    const double b = rhs[q];
    const double rq = b - t[q];
    r[q] = rq;
    rh[q] = rq;
    p[q] = 0.0;
    v[q] = 0.0;
    acc[0] = fma(rq, rq, acc[0]);
    acc[1] = fma(b, b, acc[1]);
  }
  block_reduce_store<2>(acc, partials);
}

// p = r + beta (p - omega v)
__global__ void k_update_p(long long m, const KState* st, const double* r, double* p,
                           const double* v) {
  if (stopped(st)) return;
  const double beta = (st->rho / st->rho_prev) * (st->alpha / st->omega);
  const double omega = st->omega;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (long long)gridDim.x * blockDim.x)
    p[q] = r[q] + beta * (p[q] - omega * v[q]);
}

// partial (a, c)
__global__ void k_dot(long long m, const KState* st, const double* a, const double* c,
                      double* partials) {
  if (stopped(st)) return;
  double acc[1] = {0.0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (long long)gridDim.x * blockDim.x)
    acc[0] = fma(a[q], c[q], acc[0]);
  block_reduce_store<1>(acc, partials);
}

// s = r - alpha v; x += alpha p_hat; partial (s, s)
__global__ void k_s(long long m, const KState* st, const double* r, const double* v,
                    const double* ph, double* s, double* x, double* partials) {
  if (stopped(st)) return;
  const double alpha = st->alpha;
  double acc[1] = {0.0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (long long)gridDim.x * blockDim.x) {
    const double sq = r[q] - alpha * v[q];
    s[q] = sq;
    x[q] += alpha * ph[q];
    acc[0] = fma(sq, sq, acc[0]);
  }
  block_reduce_store<1>(acc, partials);
}

// partials (t, s), (t, t)
__global__ void k_dot_ts(long long m, const KState* st, const double* t, const double* s,
                         double* partials) {
  if (stopped(st)) return;
  double acc[2] = {0.0, 0.0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (long long)gridDim.x * blockDim.x) {
    const double tq = t[q];
    acc[0] = fma(tq, s[q], acc[0]);
    acc[1] = fma(tq, tq, acc[1]);
  }
  block_reduce_store<2>(acc, partials);
}

// x += omega s_hat; r = s - omega t; partials (r, r), (r_hat, r)
__global__ void k_xr(long long m, const KState* st, const double* sh, const double* s,
                     const double* t, const double* rh, double* x, double* r, double* partials) {
  if (stopped(st)) return;
  const double omega = st->omega;
  double acc[2] = {0.0, 0.0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (long long)gridDim.x * blockDim.x) {
    x[q] += omega * sh[q];
    const double rq = s[q] - omega * t[q];
    r[q] = rq;
    acc[0] = fma(rq, rq, acc[0]);
    acc[1] = fma(rh[q], rq, acc[1]);
  }
  block_reduce_store<2>(acc, partials);
}

// t = rhs - t; partial (t, t)
__global__ void k_resid(long long m, const double* rhs, double* t, double* partials) {
  double acc[1] = {0.0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (long long)gridDim.x * blockDim.x) {
    const double d = rhs[q] - t[q];
    t[q] = d;
    acc[0] = fma(d, d, acc[0]);
  }
  block_reduce_store<1>(acc, partials);
}

__global__ void k_zero(long long m, double* x) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (long long)gridDim.x * blockDim.x)
    x[q] = 0.0;
}

enum FinStep : int { kFinInit, kFinAlpha, kFinS, kFinOmega, kFinR, kFinTrue };

// Sums the partials of one step (fixed order) and advances the scalar state.
__global__ void k_fin(KState* st, const double* partials, int step, int nv, double tol) {
  __shared__ double tot[2][kRedThreads / 32];
  double v[2] = {0.0, 0.0};
  for (int q = 0; q < nv; ++q)
    for (int k = threadIdx.x; k < kRedBlocks; k += blockDim.x) v[q] += partials[q * kRedBlocks + k];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 2; ++q) {
    for (int d = 16; d >= 1; d >>= 1) v[q] += __shfl_down_sync(kFull, v[q], d);
    if (lane == 0) tot[q][wid] = v[q];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double a = 0.0, c = 0.0;
  for (int k = 0; k < kRedThreads / 32; ++k) {
    a += tot[0][k];
    c += tot[1][k];
  }
  if (step == kFinTrue) {
    st->true2 = a;
    return;
  }
  if (step == kFinInit) {  // a = (r, r), c = (rhs, rhs)
    st->bnorm2 = c;
    st->thresh2 = (tol * sqrt(c)) * (tol * sqrt(c));
    st->rho = a;  // r_hat = r
    st->rho_prev = st->alpha = st->omega = 1.0;
    st->last2 = a;
    st->reason = kRunning;
    st->stop = 0;
    if (c == 0.0) { st->reason = kConverged; st->stop = 1; }  // rhs = 0: the host returns x = 0
    else if (sqrt(a) <= tol * sqrt(c)) { st->reason = kConverged; st->stop = 1; }
    else if (st->iters >= st->maxit) { st->reason = kMaxit; st->stop = 1; }
    else if (a == 0.0) { st->reason = kBreakdown; st->stop = 1; }
    return;
  }
  if (st->stop) return;
  const double bn = sqrt(st->bnorm2);
  switch (step) {
    // A non-finite scalar (an overflowing operator, e.g. an FP32 preconditioner
    // on an ill-conditioned system) ends the run as a breakdown before it can
    // reach x: the kernels that update x run only after the check.
    case kFinAlpha:  // a = (r_hat, v)
      if (a == 0.0 || !isfinite(a)) { st->reason = kBreakdown; st->stop = 1; break; }
      st->alpha = st->rho / a;
      break;
    case kFinS:  // a = (s, s)
      st->iters += 1;
      if (!isfinite(a)) { st->reason = kBreakdown; st->stop = 1; break; }
      st->last2 = a;
      if (sqrt(a) / bn <= tol) { st->reason = kConverged; st->stop = 1; }
      break;
    case kFinOmega:  // a = (t, s), c = (t, t)
      if (c == 0.0 || !isfinite(a) || !isfinite(c)) { st->reason = kBreakdown; st->stop = 1; break; }
      st->omega = a / c;
      break;
    case kFinR:  // a = (r, r), c = (r_hat, r)
      if (!isfinite(a) || !isfinite(c)) { st->reason = kBreakdown; st->stop = 1; break; }
      st->last2 = a;
      if (sqrt(a) / bn <= tol) { st->reason = kConverged; st->stop = 1; break; }
      if (st->omega == 0.0) { st->reason = kBreakdown; st->stop = 1; break; }
      st->rho_prev = st->rho;
      st->rho = c;
      if (c == 0.0) { st->reason = kBreakdown; st->stop = 1; break; }
      if (st->iters >= st->maxit) { st->reason = kMaxit; st->stop = 1; }
      break;
    default:
      break;
  }
}

__global__ void k_state_reset(KState* st, int maxit) {
  st->iters = 0;
  st->maxit = maxit;
  st->stop = 0;
  st->reason = kRunning;
}


// x += d
__global__ void k_axpy1(long long m, double* x, const double* d) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (long long)gridDim.x * blockDim.x)
    x[q] += d[q];
}

// t = rhs - t; partials (t, t), (rhs, rhs)
__global__ void k_resid2(long long m, const double* rhs, double* t, double* partials) {
  double acc[2] = {0.0, 0.0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (long long)gridDim.x * blockDim.x) {
    const double b = rhs[q];
    const double d = b - t[q];
    t[q] = d;
    acc[0] = fma(d, d, acc[0]);
    acc[1] = fma(b, b, acc[1]);
  }
  block_reduce_store<2>(acc, partials);
}

// sums of two partial arrays into out[0..1] (fixed order)
__global__ void k_sum2(const double* partials, double* out) {
  __shared__ double tot[2][kRedThreads / 32];
  double v[2] = {0.0, 0.0};
  for (int q = 0; q < 2; ++q)
    for (int k = threadIdx.x; k < kRedBlocks; k += blockDim.x) v[q] += partials[q * kRedBlocks + k];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 2; ++q) {
    for (int d = 16; d >= 1; d >>= 1) v[q] += __shfl_down_sync(kFull, v[q], d);
    if (lane == 0) tot[q][wid] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < kRedThreads / 32; ++k) {
      a += tot[0][k];
      c += tot[1][k];
    }
    out[0] = a;
    out[1] = c;
  }
}

}  // namespace

size_t krylov_workspace_bytes(int32_t n, int32_t b) {
  const size_t vec = align256((size_t)n * b * sizeof(double));
  return align256(sizeof(KState)) + align256(2 * kRedBlocks * sizeof(double)) + 8 * vec +
         apply_workspace_bytes(n, b);
}

size_t krylov_mixed_workspace_bytes(int32_t n, int32_t b) {
  const size_t vec = align256((size_t)n * b * sizeof(double));
  return krylov_workspace_bytes(n, b) + 2 * vec + 256;
}

// BiCGSTAB on the operators of `ops`; `x` holds the start vector.  With
// confirm, convergence is declared only when the recomputed true residual
// (ops.spmv) confirms it, restarting otherwise; without confirm the loop ends
// on the recurrence residual (used for the inner solves of the refinement).
int bicgstab_core(const KOps& ops, long long m, const double* rhs, double* x, double tol, int32_t maxit,
                  bool confirm, void* work, void* stream, int batch, int32_t* iters_out, double* relres_out,
                  double* bnorm2_out) {
  cudaStream_t s = (cudaStream_t)stream;
  const size_t vec = align256((size_t)m * sizeof(double));
  char* base = reinterpret_cast<char*>(work);
  KState* st = reinterpret_cast<KState*>(base);
  base += align256(sizeof(KState));
  double* partials = reinterpret_cast<double*>(base);
  base += align256(2 * kRedBlocks * sizeof(double));
  double* r = reinterpret_cast<double*>(base + 0 * vec);
  double* rh = reinterpret_cast<double*>(base + 1 * vec);
  double* pv = reinterpret_cast<double*>(base + 2 * vec);
  double* v = reinterpret_cast<double*>(base + 3 * vec);
  double* ph = reinterpret_cast<double*>(base + 4 * vec);
  double* sv = reinterpret_cast<double*>(base + 5 * vec);
  double* sh = reinterpret_cast<double*>(base + 6 * vec);
  double* t = reinterpret_cast<double*>(base + 7 * vec);
  void* awork = base + 8 * vec;
  int32_t* aheader = reinterpret_cast<int32_t*>(awork);
  int32_t* stop = &st->stop;
  const int vb = kRedBlocks, vt = kRedThreads;
  const auto& spmv_applied = ops.spmv_applied ? ops.spmv_applied : ops.spmv;

  cudaMemsetAsync(aheader, 0, kHeaderBytes, s);
  int status = BILU_OK;
  KState hs{};
  { ProfScope ps_(BILU_PROF_KRYLOV, s); k_state_reset<<<1, 1, 0, s>>>(st, maxit); }
  for (;;) {
    // (re)start from the residual of the current x
    if (ops.spmv(x, t, nullptr, awork)) { status = BILU_ERR_CUDA; break; }
    { ProfScope ps_(BILU_PROF_KRYLOV, s); k_init<<<vb, vt, 0, s>>>(m, rhs, t, r, rh, pv, v, partials); }
    { ProfScope ps_(BILU_PROF_KRYLOV, s); k_fin<<<1, vt, 0, s>>>(st, partials, kFinInit, 2, tol); }
    bool done_loop = false;
    while (!done_loop) {
      for (int it = 0; it < batch; ++it) {
        { ProfScope ps_(BILU_PROF_KRYLOV, s); k_update_p<<<vb, vt, 0, s>>>(m, st, r, pv, v); }
        ops.apply(pv, ph, stop, awork);
        spmv_applied(ph, v, stop, awork);
        { ProfScope ps_(BILU_PROF_KRYLOV, s); k_dot<<<vb, vt, 0, s>>>(m, st, rh, v, partials); }
        { ProfScope ps_(BILU_PROF_KRYLOV, s); k_fin<<<1, vt, 0, s>>>(st, partials, kFinAlpha, 1, tol); }
        { ProfScope ps_(BILU_PROF_KRYLOV, s); k_s<<<vb, vt, 0, s>>>(m, st, r, v, ph, sv, x, partials); }
        { ProfScope ps_(BILU_PROF_KRYLOV, s); k_fin<<<1, vt, 0, s>>>(st, partials, kFinS, 1, tol); }
        ops.apply(sv, sh, stop, awork);
        spmv_applied(sh, t, stop, awork);
        { ProfScope ps_(BILU_PROF_KRYLOV, s); k_dot_ts<<<vb, vt, 0, s>>>(m, st, t, sv, partials); }
        { ProfScope ps_(BILU_PROF_KRYLOV, s); k_fin<<<1, vt, 0, s>>>(st, partials, kFinOmega, 2, tol); }
        { ProfScope ps_(BILU_PROF_KRYLOV, s); k_xr<<<vb, vt, 0, s>>>(m, st, sh, sv, t, rh, x, r, partials); }
        { ProfScope ps_(BILU_PROF_KRYLOV, s); k_fin<<<1, vt, 0, s>>>(st, partials, kFinR, 2, tol); }
      }
      if (cudaGetLastError() != cudaSuccess) { status = BILU_ERR_CUDA; done_loop = true; break; }
      int aerr = 0;
      if (cudaMemcpyAsync(&hs, st, sizeof(KState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaMemcpyAsync(&aerr, aheader + kErr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        status = BILU_ERR_CUDA;
        done_loop = true;
        break;
      }
      if (aerr) { status = aerr; done_loop = true; break; }
      if (hs.stop) done_loop = true;
    }
    if (status != BILU_OK) break;
    if (hs.bnorm2 == 0.0) {  // rhs = 0: x = 0 solves it exactly
      { ProfScope ps_(BILU_PROF_KRYLOV, s); k_zero<<<vb, vt, 0, s>>>(m, x); }
      hs.true2 = 0.0;
      status = BILU_OK;
      break;
    }
    if (!confirm) {
      hs.true2 = hs.last2;
      status = hs.reason == kConverged ? BILU_OK : hs.reason == kBreakdown ? BILU_ERR_BREAKDOWN
                                                                           : BILU_ERR_NOT_CONVERGED;
      break;
    }
    // true residual
    ops.spmv(x, t, nullptr, awork);
    { ProfScope ps_(BILU_PROF_KRYLOV, s); k_resid<<<vb, vt, 0, s>>>(m, rhs, t, partials); }
    { ProfScope ps_(BILU_PROF_KRYLOV, s); k_fin<<<1, vt, 0, s>>>(st, partials, kFinTrue, 1, tol); }
    if (cudaMemcpyAsync(&hs, st, sizeof(KState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      status = BILU_ERR_CUDA;
      break;
    }
    const double rel = std::sqrt(hs.true2) / std::sqrt(hs.bnorm2);
    if (rel <= tol) { status = BILU_OK; break; }
    if (hs.reason == kBreakdown) { status = BILU_ERR_BREAKDOWN; break; }
    if (hs.iters >= maxit) { status = BILU_ERR_NOT_CONVERGED; break; }
    // recurrence converged but the true residual did not: restart
  }
  if (iters_out) *iters_out = hs.iters;
  if (relres_out) *relres_out = hs.bnorm2 > 0.0 ? std::sqrt(hs.true2) / std::sqrt(hs.bnorm2) : 0.0;
  if (bnorm2_out) *bnorm2_out = hs.bnorm2;
  return status;
}

namespace {

struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  double stop_ms() {
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
  }
};

}  // namespace

// FP64 BiCGSTAB (FP64 SpMV, vectors, scalars and dot products) with the
// preconditioner stored and applied in double (f) or in float (f32).
int run_bicgstab(const bilu_pattern* p, const bilu_bsr* A, const double* f, const double* rhs,
                 double* x, double tol, int32_t maxit, void* work, void* stream,
                 bilu_solve_info* info, int batch, const float* f32) {
  const int32_t n = p->n, b = A->b;
  KOps ops;
  ops.spmv = [=](const double* xin, double* yout, int32_t* stop, void*) {
    return launch_spmv(n, b, A->row_ptr, A->col_idx, A->vals, xin, yout, stream, stop);
  };
  if (f32)
    ops.apply = [=](const double* rin, double* zout, int32_t* stop, void* aw) {
      return launch_apply_f32(p, b, f32, rin, zout, aw, stop, stream);
    };
  else
    ops.apply = [=](const double* rin, double* zout, int32_t* stop, void* aw) {
      return launch_apply(p, b, f, rin, zout, aw, stop, stream);
    };
  Timer timer((cudaStream_t)stream);
  int32_t iters = 0;
  double relres = 0.0;
  const int status = bicgstab_core(ops, (long long)n * b, rhs, x, tol, maxit, true, work, stream, batch, &iters,
                                   &relres, nullptr);
  const double ms = timer.stop_ms();
  if (info) {
    info->status = status;
    info->iters = iters;
    info->true_relres = relres;
    info->ms = ms;
  }
  return status;
}

// Mixed precision: the outer loop keeps x, the residual and its norm in FP64
// (r = rhs - A x with the FP64 matrix); each correction d solves A d = r with
// BiCGSTAB whose SpMV uses the FP32 copy of A and whose preconditioner is the
// FP32-stored factorization (FP64 Krylov vectors, scalars and dot products),
// to the relative tolerance inner_tol; then x += d.
int run_bicgstab_mixed(const bilu_pattern* p, const bilu_bsr* A, const float* vals32, const float* f32,
                       const double* rhs, double* x, double tol, int32_t maxit, double inner_tol,
                       int32_t inner_maxit, void* work, void* stream, bilu_solve_info* info, int batch) {
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t n = p->n, b = A->b;
  const long long m = (long long)n * b;
  const size_t vec = align256((size_t)m * sizeof(double));
  char* tail = reinterpret_cast<char*>(work) + krylov_workspace_bytes(n, b);
  double* rout = reinterpret_cast<double*>(tail);
  double* d = reinterpret_cast<double*>(tail + vec);
  double* norms = reinterpret_cast<double*>(tail + 2 * vec);  // [(r, r), (rhs, rhs)]
  double* partials = reinterpret_cast<double*>(reinterpret_cast<char*>(work) + align256(sizeof(KState)));
  // A's block count picks the FP32 SpMV kernel (rows of at most about seven
  // blocks are staged in shared memory)
  // (a failed read leaves nnzb = 0, and the solve's own CUDA checks report it)
  int32_t nnzb = 0;
  if (cudaMemcpyAsync(&nnzb, A->row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    nnzb = 0;
  const bool staged = spmv_f32_staging_fits(n, nnzb);
  KOps ops;
  ops.spmv = [=](const double* xin, double* yout, int32_t* stop, void*) {
    return launch_spmv_f32(n, b, A->row_ptr, A->col_idx, vals32, xin, yout, stream, stop, staged);
  };
  // p_hat and s_hat come from the FP32 apply: its FP32 result is x rounded to
  // FP32 exactly, so the SpMV reads that (the same products and sums)
  ops.spmv_applied = [=](const double*, double* yout, int32_t* stop, void* aw) {
    return launch_spmv_f32x(n, b, A->row_ptr, A->col_idx, vals32, apply_f32_result(aw, n, b), yout, stream,
                            stop, staged);
  };
  ops.apply = [=](const double* rin, double* zout, int32_t* stop, void* aw) {
    return launch_apply_f32(p, b, f32, rin, zout, aw, stop, stream);
  };
  const int vb = kRedBlocks, vt = kRedThreads;
  Timer timer(s);
  int status = BILU_ERR_NOT_CONVERGED;
  int32_t iters = 0;
  double relres = 0.0;
  for (int outer = 0;; ++outer) {
    if (launch_spmv(n, b, A->row_ptr, A->col_idx, A->vals, x, rout, stream, nullptr)) { status = BILU_ERR_CUDA; break; }
    { ProfScope ps_(BILU_PROF_KRYLOV, s); k_resid2<<<vb, vt, 0, s>>>(m, rhs, rout, partials); }
    { ProfScope ps_(BILU_PROF_KRYLOV, s); k_sum2<<<1, vt, 0, s>>>(partials, norms); }
    double hn[2] = {0.0, 0.0};
    if (cudaMemcpyAsync(hn, norms, sizeof(hn), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      status = BILU_ERR_CUDA;
      break;
    }
    if (hn[1] == 0.0) {
      { ProfScope ps_(BILU_PROF_KRYLOV, s); k_zero<<<vb, vt, 0, s>>>(m, x); }
      relres = 0.0;
      status = BILU_OK;
      break;
    }
    relres = std::sqrt(hn[0]) / std::sqrt(hn[1]);
    if (relres <= tol) { status = BILU_OK; break; }
    if (!std::isfinite(relres)) { status = BILU_ERR_BREAKDOWN; break; }
    if (iters >= maxit) { status = BILU_ERR_NOT_CONVERGED; break; }
    cudaMemsetAsync(d, 0, (size_t)m * sizeof(double), s);
    int32_t it = 0;
    const int32_t budget = std::min(inner_maxit, maxit - iters);
    if (budget <= 0) { status = BILU_ERR_NOT_CONVERGED; break; }
    const int st = bicgstab_core(ops, m, rout, d, inner_tol, budget, false, work, stream, batch, &it, nullptr,
                                 nullptr);
    if (st == BILU_ERR_CUDA || st == BILU_ERR_TIMEOUT) { status = st; break; }
    { ProfScope ps_(BILU_PROF_KRYLOV, s); k_axpy1<<<vb, vt, 0, s>>>(m, x, d); }
    iters += it;
    if (st == BILU_ERR_BREAKDOWN && it == 0) { status = BILU_ERR_BREAKDOWN; break; }
  }
  const double ms = timer.stop_ms();
  if (info) {
    info->status = status;
    info->iters = iters;
    info->true_relres = relres;
    info->ms = ms;
  }
  return status;
}

}  // namespace bilu
