// adjoint.cu -- the pieces of the adjoint solve A^T lambda = g.
//
// With A ~ M = L D U' (Eq. 5-6), M^T = U'^T D^T L^T, so M^{-T} r is: solve
// U'^T z = r (unit lower), then w = D^{-T} z, then solve L^T y = w (unit
// upper) -- exactly the apply of Eq. 6 / Algorithm 7 on the transposed
// pattern P'^T (lower part U'^T, upper part L^T) with the blocks transposed.
// bilu_factor_transpose builds that factor buffer from the forward one by a
// gather (each slot of P'^T reads the slot of P' it transposes), so the
// adjoint reuses the sync-free solves and the BSR SpMV unchanged (A^T is
// gathered the same way).  The gradient of a loss through x = A^{-1} b is
// dL/db = lambda and dL/dA_IJ = -lambda_I x_J^T on A's block pattern.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"

namespace bilu {
namespace {

// dst block s = (src block idx[s])^T; blocks are b x b, column-major.
template <int B>
__global__ void gather_transpose_kernel(long long nblocks, const int32_t* __restrict__ idx,
                                        const double* __restrict__ src, double* __restrict__ dst) {
  constexpr int BB = B * B;
  const long long total = nblocks * BB;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const long long s = q / BB;
    const int e = (int)(q - s * BB);
    const int r = e % B, c = e / B;  // dst element (r, c) = src element (c, r)
    dst[q] = __ldg(src + (size_t)__ldg(idx + s) * BB + r * B + c);
  }
}

// grad block t of row I (column J = ci[t]) = -lambda_I x_J^T, one warp per
// block row, lanes over the row's (block, element) pairs.
template <int B>
__global__ void __launch_bounds__(256) outer_grad_kernel(int32_t n, const int32_t* __restrict__ rp,
                                                         const int32_t* __restrict__ ci,
                                                         const double* __restrict__ lam,
                                                         const double* __restrict__ x, double* __restrict__ grad) {
  constexpr int BB = B * B;
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
    const int beg = rp[i], cnt = (rp[i + 1] - beg) * BB;
    for (int q = lane; q < cnt; q += 32) {
      const int t = beg + q / BB, e = q % BB;
      const int r = e % B, c = e / B;
      grad[(size_t)t * BB + e] = -__ldg(lam + (size_t)i * B + r) * __ldg(x + (size_t)__ldg(ci + t) * B + c);
    }
  }
}

int grid_for(long long work, int threads) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (int)std::max<long long>(1, std::min<long long>((work + threads - 1) / threads, (long long)sms * 16));
}

}  // namespace

int launch_gather_transpose(long long nblocks, int32_t b, const int32_t* idx, const double* src, double* dst,
                            void* stream) {
  if (nblocks == 0) return 0;
  const int grid = grid_for(nblocks * b * b, 256);
  BILU_DISPATCH_B(b, {
    ProfScope ps(BILU_PROF_ADJOINT, stream);
    gather_transpose_kernel<B><<<grid, 256, 0, (cudaStream_t)stream>>>(nblocks, idx, src, dst);
  });
  return (int)cudaGetLastError();
}

int launch_outer_grad(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci, const double* lam,
                      const double* x, double* grad, void* stream) {
  if (n == 0) return 0;
  const int grid = grid_for((long long)n * 32, 256);
  BILU_DISPATCH_B(b, {
    ProfScope ps(BILU_PROF_ADJOINT, stream);
    outer_grad_kernel<B><<<grid, 256, 0, (cudaStream_t)stream>>>(n, rp, ci, lam, x, grad);
  });
  return (int)cudaGetLastError();
}

}  // namespace bilu
