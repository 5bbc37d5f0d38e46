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
// latency, so the FP32 kernels issue the loads of four blocks (column
// indices, then values and x) before their FMAs, which run in the same order
// as one block at a time (identical sums).  For b <= 5 the FP32 path first
// stages each warp's whole value range in shared memory (one batch of
// 16-byte asynchronous copies, spmv_f32_staged_kernel below).  x is either
// FP64, rounded to nearest on the integer pipes one component per lane, or
// FP32 already (the FP32 preconditioner's own result).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device_common.cuh"

namespace bilu {
namespace {

// Streaming load (cache-streaming: evict-first in L1 and L2).
template <typename TV>
__device__ __forceinline__ TV ld_stream(const TV* p) { return __ldcs(p); }

// FP32 values: each lane of a row loads one component of x_j (an FP64 x is
// rounded to FP32 on the integer pipes, d2f_rn) and the row's b lanes share
// the components by shuffles, instead of every lane loading (and rounding)
// all b.
template <typename TV, typename XT>
constexpr bool kShareX = sizeof(TV) == 4;
__device__ __forceinline__ float x_f32(double v) { return d2f_rn(v); }
__device__ __forceinline__ float x_f32(float v) { return v; }

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
        for (int u = 0; u < U; ++u) xs[u] = x_f32(__ldg(x + (size_t)j[u] * B + r));
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
      const TV xs = x_f32(__ldg(xj + r));
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

// ---------------------------------------------------------------------------
// FP32 SpMV with each warp's matrix range staged in shared memory (b <= 5).
//
// As in spmv_kernel, a warp owns R = 32 / b consecutive block rows.  Their
// blocks are one contiguous range, so the warp first copies the column
// indices and values of the range into its own shared memory with 16-byte
// asynchronous copies (one batch for the whole group, rounded out to whole
// 4-block units so every copy is 16-byte aligned), then sums each row from
// shared memory, gathering only x.  A warp thus waits for three round trips
// (row pointers, the copy, x) instead of one per batch of blocks.  Blocks
// past the last multiple of 4 of the matrix, and every block of a group
// larger than the buffer, are read from global memory.  Sums run in the
// order of spmv_kernel (identical results).
template <int B>
struct StageGeom {
  static constexpr int R = 32 / B;
  static constexpr int CAP = (R * 7 + 8 + 3) / 4 * 4;  // blocks a warp stages: a 7-point group + slack
  static constexpr int BYTES = CAP * 4 * (1 + B * B);  // column indices, then values
  static constexpr int WARPS = 8;
  static constexpr int SMEM = WARPS * BYTES;
  static_assert(BYTES % 16 == 0 && SMEM <= 48 * 1024, "16-byte aligned per-warp buffers");
};

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// One row's FP32 sum over its blocks [beg, end) in spmv_kernel's order
// (batches of 4 blocks, then single blocks): col(t) is block t's column,
// val(t) lane r's element of block t in column 0 (column c at [c * B]).
template <int B, typename XT, typename Col, typename Val>
__device__ __forceinline__ float row_sum_f32(int32_t beg, int32_t end, Col col, Val val, const XT* __restrict__ x,
                                             int r, int lane, unsigned am) {
  constexpr int U = 4;
  float acc = 0.f;
  int32_t t = beg;
  for (; t + U <= end; t += U) {
    int32_t j[U];
#pragma unroll
    for (int u = 0; u < U; ++u) j[u] = col(t + u);
    float av[U][B];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int c = 0; c < B; ++c) av[u][c] = val(t + u, c);
    float xs[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xs[u] = x_f32(__ldg(x + (size_t)j[u] * B + r));
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int c = 0; c < B; ++c) acc = fmaf(av[u][c], __shfl_sync(am, xs[u], lane - r + c), acc);
  }
  for (; t < end; ++t) {
    const int32_t j = col(t);
    float av[B];
#pragma unroll
    for (int c = 0; c < B; ++c) av[c] = val(t, c);
    const float xs = x_f32(__ldg(x + (size_t)j * B + r));
#pragma unroll
    for (int c = 0; c < B; ++c) acc = fmaf(av[c], __shfl_sync(am, xs, lane - r + c), acc);
  }
  return acc;
}

template <int B, typename XT>
__global__ void __launch_bounds__(256) spmv_f32_staged_kernel(int32_t n, const int32_t* __restrict__ rp,
                                                              const int32_t* __restrict__ ci,
                                                              const float* __restrict__ vals,
                                                              const XT* __restrict__ x,
                                                              double* __restrict__ y, const int32_t* stop) {
  using G = StageGeom<B>;
  constexpr int R = G::R, BB = B * B;
  extern __shared__ __align__(16) unsigned char smem[];
  if (stop && ld_volatile_s32(stop)) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long g0 = ((long long)blockIdx.x * G::WARPS + wib) * R;
  if (g0 >= n) return;  // warp-uniform
  const int nrows = (int)min((long long)R, (long long)n - g0);
  int32_t* sci = reinterpret_cast<int32_t*>(smem + (size_t)wib * G::BYTES);
  float* sv = reinterpret_cast<float*>(smem + (size_t)wib * G::BYTES + G::CAP * 4);
  // row pointers of the group (lane i holds rp[g0 + i]), its end, and nnz
  const int32_t rpv = lane < nrows ? __ldg(rp + g0 + lane) : 0;
  const int32_t ge = __ldg(rp + g0 + nrows), nnz = __ldg(rp + n);
  const int q = lane / B, r = lane - q * B;
  const int32_t beg = __shfl_sync(0xFFFFFFFFu, rpv, q);
  const int32_t nxt = __shfl_sync(0xFFFFFFFFu, rpv, q + 1 < 32 ? q + 1 : 31);
  const int32_t end = q + 1 < nrows ? nxt : ge;
  const int32_t gb = __shfl_sync(0xFFFFFFFFu, rpv, 0);
  // the staged range [ka, kc): whole 4-block units inside the matrix
  const int32_t ka = gb & ~3;
  int32_t kc = (int32_t)min(((long long)ge + 3) & ~3LL, (long long)(nnz & ~3));
  if (kc < ka || kc - ka > G::CAP) kc = ka;  // nothing staged
  if (kc > ka) {
    const int nci = (kc - ka) / 4, nv = (kc - ka) * BB / 4;
    for (int i = lane; i < nci; i += 32) cp_async16(sci + 4 * i, ci + ka + 4 * i);
    for (int i = lane; i < nv; i += 32) cp_async16(sv + 4 * i, vals + (size_t)ka * BB + 4 * i);
    cp_async_wait_all();
  }
  __syncwarp();
  if (q >= nrows) return;
  const unsigned am = (B == 32 ? 0xFFFFFFFFu : ((1u << B) - 1u)) << (q * B);
  float acc;
  if (end <= kc) {  // the whole row is staged
    acc = row_sum_f32<B, XT>(
        beg, end, [&](int32_t t) { return sci[t - ka]; },
        [&](int32_t t, int c) { return sv[(size_t)(t - ka) * BB + r + c * B]; }, x, r, lane, am);
  } else {
    acc = row_sum_f32<B, XT>(
        beg, end, [&](int32_t t) { return __ldg(ci + t); },
        [&](int32_t t, int c) { return ld_stream(vals + (size_t)t * BB + r + c * B); }, x, r, lane, am);
  }
  y[(g0 + q) * B + r] = (double)acc;
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

template <int B, typename XT>
int launch_spmv_f32_staged(int32_t n, const int32_t* rp, const int32_t* ci, const float* vals, const XT* x,
                           double* y, void* stream, const int32_t* stop) {
  using G = StageGeom<B>;
  const long long warps = ((long long)n + G::R - 1) / G::R;
  const long long blocks = (warps + G::WARPS - 1) / G::WARPS;
  ProfScope ps(BILU_PROF_SPMV, stream);
  spmv_f32_staged_kernel<B, XT><<<(unsigned)blocks, G::WARPS * 32, G::SMEM, (cudaStream_t)stream>>>(
      n, rp, ci, vals, x, y, stop);
  return (int)cudaGetLastError();
}

// FP32 values, x of type XT: the staged kernel for b <= 5 with 16-byte aligned
// column indices and values (unless the caller knows the rows are too long
// for its buffers), else the direct kernel.
template <typename XT>
int launch_spmv_f32_any(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci, const float* vals,
                        const XT* x, double* y, void* stream, const int32_t* stop, bool allow_staged) {
  if (n == 0) return 0;
  if (allow_staged && b <= 5 && ((((uintptr_t)ci) | ((uintptr_t)vals)) & 15u) == 0) {
    switch (b) {
      case 1: return launch_spmv_f32_staged<1, XT>(n, rp, ci, vals, x, y, stream, stop);
      case 2: return launch_spmv_f32_staged<2, XT>(n, rp, ci, vals, x, y, stream, stop);
      case 3: return launch_spmv_f32_staged<3, XT>(n, rp, ci, vals, x, y, stream, stop);
      case 4: return launch_spmv_f32_staged<4, XT>(n, rp, ci, vals, x, y, stream, stop);
      default: return launch_spmv_f32_staged<5, XT>(n, rp, ci, vals, x, y, stream, stop);
    }
  }
  return launch_spmv_t<float, XT>(n, b, rp, ci, vals, x, y, stream, stop);
}

}  // namespace

int launch_spmv(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci, const double* vals,
                const double* x, double* y, void* stream, const int32_t* stop) {
  return launch_spmv_t<double, double>(n, b, rp, ci, vals, x, y, stream, stop);
}

int launch_spmv_f32(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci, const float* vals,
                    const double* x, double* y, void* stream, const int32_t* stop, bool allow_staged) {
  return launch_spmv_f32_any<double>(n, b, rp, ci, vals, x, y, stream, stop, allow_staged);
}

int launch_spmv_f32x(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci, const float* vals,
                     const float* x, double* y, void* stream, const int32_t* stop, bool allow_staged) {
  return launch_spmv_f32_any<float>(n, b, rp, ci, vals, x, y, stream, stop, allow_staged);
}

bool spmv_f32_staging_fits(int32_t n, long long nnzb) {
  // a stage buffer holds R rows of 7 blocks plus alignment slack: on average
  // at most 7.2 blocks per row (36 / 5), else most groups would read global
  // memory from a kernel whose shared memory still costs L1
  return nnzb * 5 <= (long long)n * 36;
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
