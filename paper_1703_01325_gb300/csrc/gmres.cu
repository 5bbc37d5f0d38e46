// gmres.cu -- restarted GMRES(m), preconditioned on the right with M = L D U'
// (Eq. 5-6): the solver of the paper's experiments (Section 4 restarts it
// every 20 iterations).
//
// One cycle:  r0 = rhs - A x, beta = ||r0||, v_1 = r0 / beta;  Arnoldi step j:
// w = A M^{-1} v_j, modified Gram-Schmidt h_ij = (w, v_i), w -= h_ij v_i for
// i = 1..j in order, h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j};  Givens
// rotations keep H upper triangular and |g_{j+1}| is the least-squares
// residual.  The cycle ends at |g_{j+1}| <= tol ||rhs||, h_{j+1,j} = 0, m
// steps or the iteration budget; then y = R^{-1} g, x += M^{-1} (V y), and the
// true residual decides between stopping and the next cycle.
//
// On the device: every vector pass is one kernel over the vector (the MGS
// update of step i is fused with the dot product of step i + 1, so each
// Gram-Schmidt step reads w once and v_i once), every dot product reduces in
// two deterministic stages (fixed per-block partials, then one block), and
// the Hessenberg matrix, rotations and scalars live in device memory, updated
// by one-block kernels.  Kernels inside a cycle return at once when the
// cycle's stop word is set, so the host enqueues several Arnoldi steps
// between looks at the state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "device_common.cuh"

namespace bilu {
namespace {

constexpr int kGRedBlocks = 608;
constexpr int kGRedThreads = 256;
constexpr int kMaxRestart = 64;

enum GReason : int { gRunning = 0, gConverged = 1, gBreakdown = 2, gMaxit = 3, gCycle = 4 };

struct GState {
  double H[(kMaxRestart + 1) * kMaxRestart];  // column j at H[j * (m + 1)]
  double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1], y[kMaxRestart];
  double hnext;  // h_{j+1,j} of the last step, before its rotation
  double bnorm2, beta, true2;
  int m, cols, stop, reason, iters, maxit;
};

__device__ __forceinline__ bool gstopped(const GState* st) { return ld_volatile_s32(&st->stop) != 0; }

template <int NV>
__device__ __forceinline__ void reduce_store(double (&v)[NV], double* partials) {
  __shared__ double red[NV][kGRedThreads / 32];
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
    for (int k = 0; k < kGRedThreads / 32; ++k) s += red[threadIdx.x][k];
    partials[threadIdx.x * kGRedBlocks + blockIdx.x] = s;
  }
}

// sum of the partials of value q (fixed order), valid in thread 0
__device__ double sum_partials(const double* partials, int q) {
  __shared__ double tot[kGRedThreads / 32];
  double v = 0.0;
  for (int k = threadIdx.x; k < kGRedBlocks; k += blockDim.x) v += partials[q * kGRedBlocks + k];
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_down_sync(kFull, v, d);
  if ((threadIdx.x & 31) == 0) tot[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kGRedThreads / 32; ++k) s += tot[k];
  __syncthreads();
  return s;
}

#define GRID_STRIDE(q, len) \
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < (len); q += (long long)gridDim.x * blockDim.x)

// v0 = rhs - t; partials (v0, v0), (rhs, rhs)
__global__ void g_init(long long len, const double* rhs, const double* t, double* v0, double* partials) {
  double acc[2] = {0.0, 0.0};
  GRID_STRIDE(q, len) {
    const double b = rhs[q], r = b - t[q];
    v0[q] = r;
    acc[0] = fma(r, r, acc[0]);
    acc[1] = fma(b, b, acc[1]);
  }
  reduce_store<2>(acc, partials);
}

__global__ void g_fin_init(GState* st, const double* partials, double tol) {
  const double rr = sum_partials(partials, 0);
  const double bb = sum_partials(partials, 1);
  if (threadIdx.x != 0) return;
  st->bnorm2 = bb;
  st->beta = sqrt(rr);
  for (int q = 0; q <= st->m; ++q) st->g[q] = 0.0;
  st->g[0] = st->beta;
  st->cols = 0;
  st->stop = 0;
  st->reason = gRunning;
  if (bb == 0.0 || sqrt(rr) <= tol * sqrt(bb)) { st->reason = gConverged; st->stop = 1; }
  else if (st->iters >= st->maxit) { st->reason = gMaxit; st->stop = 1; }
}

// v *= 1 / beta
__global__ void g_scale0(long long len, const GState* st, double* v) {
  if (gstopped(st)) return;
  const double inv = 1.0 / st->beta;
  GRID_STRIDE(q, len) v[q] *= inv;
}

// i == 0: partial (w, v_0).  i > 0: w -= h_{i-1,j} v_{i-1}, then partial (w, v_i).
__global__ void g_mgs(long long len, const GState* st, int i, int j, double* w, const double* vprev,
                      const double* vi, double* partials) {
  if (gstopped(st)) return;
  const double h = i > 0 ? st->H[j * (st->m + 1) + i - 1] : 0.0;
  double acc[1] = {0.0};
  GRID_STRIDE(q, len) {
    double wq = w[q];
    if (i > 0) {
      wq = fma(-h, vprev[q], wq);
      w[q] = wq;
    }
    acc[0] = fma(wq, vi[q], acc[0]);
  }
  reduce_store<1>(acc, partials);
}

__global__ void g_fin_h(GState* st, const double* partials, int i, int j) {
  const double s = sum_partials(partials, 0);
  if (threadIdx.x == 0 && !st->stop) st->H[j * (st->m + 1) + i] = s;
}

// w -= h_{j,j} v_j; partial (w, w)
__global__ void g_mgs_last(long long len, const GState* st, int j, double* w, const double* vj, double* partials) {
  if (gstopped(st)) return;
  const double h = st->H[j * (st->m + 1) + j];
  double acc[1] = {0.0};
  GRID_STRIDE(q, len) {
    const double wq = fma(-h, vj[q], w[q]);
    w[q] = wq;
    acc[0] = fma(wq, wq, acc[0]);
  }
  reduce_store<1>(acc, partials);
}

// h_{j+1,j} = ||w||; rotations; residual estimate; cycle bookkeeping
__global__ void g_fin_step(GState* st, const double* partials, int j, double tol) {
  const double ww = sum_partials(partials, 0);
  if (threadIdx.x != 0 || st->stop) return;
  const int ld = st->m + 1;
  double* h = st->H + j * ld;
  const double hn = sqrt(ww);
  h[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = h[i], c = h[i + 1];
    h[i] = st->cs[i] * a + st->sn[i] * c;
    h[i + 1] = -st->sn[i] * a + st->cs[i] * c;
  }
  const double a = h[j], c = h[j + 1];
  const double rho = sqrt(a * a + c * c);
  st->iters += 1;
  // rho = 0: w and v_j both vanish, the step adds nothing.  A non-finite
  // column (an overflowing operator) is dropped the same way: the cycle ends
  // with the columns before it, so x never takes a non-finite update.
  if (rho == 0.0 || !isfinite(rho)) {
    st->cols = j;
    st->reason = j == 0 ? gBreakdown : gCycle;
    st->stop = 1;
    return;
  }
  st->cs[j] = a / rho;
  st->sn[j] = c / rho;
  h[j] = rho;
  h[j + 1] = 0.0;
  st->g[j + 1] = -st->sn[j] * st->g[j];
  st->g[j] = st->cs[j] * st->g[j];
  st->cols = j + 1;
  st->hnext = hn;
  if (fabs(st->g[j + 1]) <= tol * sqrt(st->bnorm2)) { st->reason = gConverged; st->stop = 1; }
  else if (hn == 0.0) { st->reason = gConverged; st->stop = 1; }  // invariant Krylov space: exact
  else if (j + 1 == st->m) { st->reason = gCycle; st->stop = 1; }
  else if (st->iters >= st->maxit) { st->reason = gMaxit; st->stop = 1; }
}

// v_{j+1} = w / h_{j+1,j}
__global__ void g_vnext(long long len, const GState* st, const double* w, double* vn) {
  if (gstopped(st)) return;
  const double inv = 1.0 / st->hnext;
  GRID_STRIDE(q, len) vn[q] = w[q] * inv;
}

// y = R^{-1} g (back substitution over the cycle's columns)
__global__ void g_backsolve(GState* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = st->cols, ld = st->m + 1;
  for (int i = k - 1; i >= 0; --i) {
    double s = st->g[i];
    for (int l = i + 1; l < k; ++l) s -= st->H[l * ld + i] * st->y[l];
    st->y[i] = s / st->H[i * ld + i];
  }
}

// u = sum_{i < cols} y_i v_i (basis vectors spaced `stride` doubles apart)
__global__ void g_combine(long long len, const GState* st, const double* V, long long stride, double* u) {
  const int k = st->cols;
  GRID_STRIDE(q, len) {
    double s = 0.0;
    for (int i = 0; i < k; ++i) s = fma(st->y[i], V[i * stride + q], s);
    u[q] = s;
  }
}

// x += z (when the cycle produced columns)
__global__ void g_update_x(long long len, const GState* st, double* x, const double* z) {
  if (st->cols == 0) return;
  GRID_STRIDE(q, len) x[q] += z[q];
}

// t = rhs - t; partial (t, t)
__global__ void g_resid(long long len, const double* rhs, double* t, double* partials) {
  double acc[1] = {0.0};
  GRID_STRIDE(q, len) {
    const double d = rhs[q] - t[q];
    t[q] = d;
    acc[0] = fma(d, d, acc[0]);
  }
  reduce_store<1>(acc, partials);
}

__global__ void g_fin_true(GState* st, const double* partials) {
  const double s = sum_partials(partials, 0);
  if (threadIdx.x == 0) st->true2 = s;
}

__global__ void g_reset(GState* st, int m, int maxit) {
  st->m = m;
  st->iters = 0;
  st->maxit = maxit;
  st->stop = 0;
  st->reason = gRunning;
  st->cols = 0;
}

__global__ void g_zero(long long len, double* x) {
  GRID_STRIDE(q, len) x[q] = 0.0;
}

#undef GRID_STRIDE

}  // namespace

size_t gmres_workspace_bytes_impl(int32_t n, int32_t b, int32_t m) {
  const size_t vec = align256((size_t)n * b * sizeof(double));
  return align256(sizeof(GState)) + align256(2 * kGRedBlocks * sizeof(double)) + ((size_t)m + 4) * vec +
         apply_workspace_bytes(n, b);
}

int gmres_max_restart() { return kMaxRestart; }

int run_gmres(const bilu_pattern* p, const bilu_bsr* A, const double* f, const double* rhs, double* x, double tol,
              int32_t maxit, int32_t m, void* work, void* stream, bilu_solve_info* info, int batch) {
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t n = p->n, b = A->b;
  const long long len = (long long)n * b;
  const size_t vec = align256((size_t)len * sizeof(double));
  char* base = reinterpret_cast<char*>(work);
  GState* st = reinterpret_cast<GState*>(base);
  base += align256(sizeof(GState));
  double* partials = reinterpret_cast<double*>(base);
  base += align256(2 * kGRedBlocks * sizeof(double));
  double* V = reinterpret_cast<double*>(base);  // m + 1 basis vectors
  const long long stride = (long long)(vec / sizeof(double));
  double* w = reinterpret_cast<double*>(base + (size_t)(m + 1) * vec);
  double* z = reinterpret_cast<double*>(base + (size_t)(m + 2) * vec);
  double* t = reinterpret_cast<double*>(base + (size_t)(m + 3) * vec);
  void* awork = base + (size_t)(m + 4) * vec;
  int32_t* aheader = reinterpret_cast<int32_t*>(awork);
  int32_t* stop = &st->stop;
  const int vb = kGRedBlocks, vt = kGRedThreads;
  auto spmv = [&](const double* xin, double* yout, int32_t* sw) {
    return launch_spmv(n, b, A->row_ptr, A->col_idx, A->vals, xin, yout, stream, sw);
  };
  auto apply = [&](const double* rin, double* zout, int32_t* sw) {
    return launch_apply(p, b, f, rin, zout, awork, sw, stream);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  cudaMemsetAsync(aheader, 0, kHeaderBytes, s);
  { ProfScope ps_(BILU_PROF_KRYLOV, s); g_reset<<<1, 1, 0, s>>>(st, m, maxit); }
  struct Host {
    double bnorm2, beta, true2;
    int m, cols, stop, reason, iters, maxit;
  } hs{};
  auto read_state = [&]() -> int {
    int aerr = 0;
    if (cudaMemcpyAsync(&hs, &st->bnorm2, sizeof(Host), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&aerr, aheader + kErr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return BILU_ERR_CUDA;
    return aerr ? aerr : BILU_OK;
  };
  int status = BILU_OK;
  double relres = 0.0;
  for (;;) {
    if (spmv(x, t, nullptr)) { status = BILU_ERR_CUDA; break; }
    { ProfScope ps_(BILU_PROF_KRYLOV, s); g_init<<<vb, vt, 0, s>>>(len, rhs, t, V, partials); }
    { ProfScope ps_(BILU_PROF_KRYLOV, s); g_fin_init<<<1, vt, 0, s>>>(st, partials, tol); }
    { ProfScope ps_(BILU_PROF_KRYLOV, s); g_scale0<<<vb, vt, 0, s>>>(len, st, V); }
    for (int j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * stride;
      apply(vj, z, stop);
      spmv(z, w, stop);
      for (int i = 0; i <= j; ++i) {
        { ProfScope ps_(BILU_PROF_KRYLOV, s);
          g_mgs<<<vb, vt, 0, s>>>(len, st, i, j, w, i > 0 ? V + (size_t)(i - 1) * stride : nullptr,
                                  V + (size_t)i * stride, partials); }
        { ProfScope ps_(BILU_PROF_KRYLOV, s); g_fin_h<<<1, vt, 0, s>>>(st, partials, i, j); }
      }
      { ProfScope ps_(BILU_PROF_KRYLOV, s); g_mgs_last<<<vb, vt, 0, s>>>(len, st, j, w, vj, partials); }
      { ProfScope ps_(BILU_PROF_KRYLOV, s); g_fin_step<<<1, vt, 0, s>>>(st, partials, j, tol); }
      { ProfScope ps_(BILU_PROF_KRYLOV, s); g_vnext<<<vb, vt, 0, s>>>(len, st, w, V + (size_t)(j + 1) * stride); }
      if ((j + 1) % batch == 0 || j + 1 == m) {
        if (cudaGetLastError() != cudaSuccess) { status = BILU_ERR_CUDA; break; }
        status = read_state();
        if (status != BILU_OK || hs.stop) break;
      }
    }
    if (status != BILU_OK) break;
    if (hs.bnorm2 == 0.0) {  // rhs = 0: x = 0 solves it exactly
      { ProfScope ps_(BILU_PROF_KRYLOV, s); g_zero<<<vb, vt, 0, s>>>(len, x); }
      relres = 0.0;
      break;
    }
    if (hs.cols > 0) {
      { ProfScope ps_(BILU_PROF_KRYLOV, s); g_backsolve<<<1, 32, 0, s>>>(st); }
      { ProfScope ps_(BILU_PROF_KRYLOV, s); g_combine<<<vb, vt, 0, s>>>(len, st, V, stride, w); }
      apply(w, z, nullptr);
      { ProfScope ps_(BILU_PROF_KRYLOV, s); g_update_x<<<vb, vt, 0, s>>>(len, st, x, z); }
    }
    spmv(x, t, nullptr);
    { ProfScope ps_(BILU_PROF_KRYLOV, s); g_resid<<<vb, vt, 0, s>>>(len, rhs, t, partials); }
    { ProfScope ps_(BILU_PROF_KRYLOV, s); g_fin_true<<<1, vt, 0, s>>>(st, partials); }
    status = read_state();
    if (status != BILU_OK) break;
    relres = std::sqrt(hs.true2) / std::sqrt(hs.bnorm2);
    if (relres <= tol) break;
    if (hs.reason == gBreakdown && hs.cols == 0) { status = BILU_ERR_BREAKDOWN; break; }
    if (hs.iters >= maxit) { status = BILU_ERR_NOT_CONVERGED; break; }
    // next cycle from the true residual
  }
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    info->status = status;
    info->iters = hs.iters;
    info->true_relres = relres;
    info->ms = ms;
  }
  return status;
}

}  // namespace bilu
