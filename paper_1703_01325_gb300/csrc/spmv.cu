// spmv.cu -- block CSR SpMV y = A x (the SpMV of Section 2.4 / Algorithm 7).
//
// One lane per output component: a warp owns R = floor(32 / b) consecutive
// block rows and lane (row, r) accumulates y[row][r] = sum_t sum_c
// A_t[r][c] x_{col(t)}[c] over the row's blocks in column order.  Each lane
// does exactly b FMAs per block, so the FP64 pipe (the scarce unit on this part)
// does no reduction work; the b lanes of a row read b consecutive doubles of
// each block column, and the R rows of a warp are consecutive in memory, so
// every byte of the warp's contiguous value range is used.  Values are
// streamed with cache-streaming loads; x stays in L2 for the gathers.
// In FP64 the kernel is bound by the FP64 pipe; in FP32 it is bound by load
// latency, so the FP32 kernel issues the loads of four blocks (column
// indices, then values and x) before their FMAs, which run in the same order
// as one block at a time (identical sums).  The FP32 kernel takes x in FP64
// and rounds it to nearest on the integer pipes, one component per lane.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"

namespace bilu {
namespace {

// Streaming load (cache-streaming: evict-first in L1 and L2).
template <typename TV>
__device__ __forceinline__ TV ld_stream(const TV* p) { return __ldcs(p); }

// FP32 values with FP64 x: each lane of a row converts one component of x_j
// (on the integer pipes, d2f_rn) and the row's b lanes share the components
// by shuffles, instead of every lane converting all b.
template <typename TV, typename XT>
constexpr bool kShareX = sizeof(TV) == 4 && sizeof(XT) == 8;

// TV: the type the matrix is stored in and the products are accumulated in
// (double, or float for the FP32 copy of A); y stays double.  XT: the type of
// x (double).  A hardware double -> float conversion runs at the FP64 rate and
// would bound the FP32 kernel like the FP64 one, hence d2f_rn and the sharing.
template <int B, typename TV, typename XT>
__global__ void __launch_bounds__(256) spmv_kernel(int32_t n, const int32_t* __restrict__ rp,
                                                   const int32_t* __restrict__ ci,
                                                   const TV* __restrict__ vals,
                                                   const XT* __restrict__ x,
                                                   double* __restrict__ y,
                                                   const int32_t* stop) {
  constexpr int R = 32 / B;
  if (stop && ld_volatile_s32(stop)) return;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int q = lane / B;
  const int r = lane - q * B;
  const long long row = warp * R + q;
  if (q >= R || row >= n) return;
  const int32_t beg = rp[row], end = rp[row + 1];
  TV acc = TV(0);
  // The b lanes of this row: they run the same trip counts, so they meet at every shuffle.
  const unsigned am = (B == 32 ? 0xFFFFFFFFu : ((1u << B) - 1u)) << (q * B);
  (void)am;
  constexpr int U = sizeof(TV) == 4 ? 4 : 1;  // blocks whose loads are in flight together
  int32_t t = beg;
  if (U > 1) {
    for (; t + U <= end; t += U) {
      int32_t j[U];
#pragma unroll
      for (int u = 0; u < U; ++u) j[u] = __ldg(ci + t + u);
      TV av[U][B];
      XT xv[U][B];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const TV* a = vals + (size_t)(t + u) * (B * B) + r;
#pragma unroll
        for (int c = 0; c < B; ++c) av[u][c] = ld_stream(a + c * B);
      }
      if constexpr (kShareX<TV, XT>) {
        TV xs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) xs[u] = d2f_rn(__ldg(x + (size_t)j[u] * B + r));
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int c = 0; c < B; ++c) acc = fma(av[u][c], __shfl_sync(am, xs[u], lane - r + c), acc);
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int c = 0; c < B; ++c) xv[u][c] = __ldg(x + (size_t)j[u] * B + c);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int c = 0; c < B; ++c) acc = fma(av[u][c], (TV)xv[u][c], acc);
      }
    }
  }
  for (; t < end; ++t) {
    const int32_t j = __ldg(ci + t);
    const TV* a = vals + (size_t)t * (B * B) + r;
    const XT* xj = x + (size_t)j * B;
    TV av[B];
#pragma unroll
    for (int c = 0; c < B; ++c) av[c] = ld_stream(a + c * B);
    if constexpr (kShareX<TV, XT>) {
      const TV xs = d2f_rn(__ldg(xj + r));
#pragma unroll
      for (int c = 0; c < B; ++c) acc = fma(av[c], __shfl_sync(am, xs, lane - r + c), acc);
    } else {
#pragma unroll
      for (int c = 0; c < B; ++c) acc = fma(av[c], (TV)__ldg(xj + c), acc);
    }
  }
  y[row * B + r] = (double)acc;
}

__global__ void convert_kernel(const double* __restrict__ src, float* __restrict__ dst, long long count,
                               const int32_t* stop) {
  if (stop && ld_volatile_s32(stop)) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride)
    dst[q] = d2f_rn(src[q]);
}

template <typename TV, typename XT>
int launch_spmv_t(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci, const TV* vals, const XT* x,
                  double* y, void* stream, const int32_t* stop) {
  if (n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  BILU_DISPATCH_B(b, {
    constexpr int R = 32 / B;
    const long long warps = ((long long)n + R - 1) / R;
    const int tpb = 256;
    const long long blocks = (warps * 32 + tpb - 1) / tpb;
    ProfScope ps(BILU_PROF_SPMV, stream);
    spmv_kernel<B, TV, XT><<<(unsigned)blocks, tpb, 0, s>>>(n, rp, ci, vals, x, y, stop);
  });
  return (int)cudaGetLastError();
}

}  // namespace

int launch_spmv(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci, const double* vals,
                const double* x, double* y, void* stream, const int32_t* stop) {
  return launch_spmv_t<double, double>(n, b, rp, ci, vals, x, y, stream, stop);
}

int launch_spmv_f32(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci, const float* vals,
                    const double* x, double* y, void* stream, const int32_t* stop) {
  return launch_spmv_t<float, double>(n, b, rp, ci, vals, x, y, stream, stop);
}

int launch_convert_f32(const double* src, float* dst, long long count, void* stream, const int32_t* stop) {
  if (count <= 0) return 0;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long blocks = std::min<long long>((count + 255) / 256, (long long)sms * 16);
  convert_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(src, dst, count, stop);
  return (int)cudaGetLastError();
}

}  // namespace bilu
