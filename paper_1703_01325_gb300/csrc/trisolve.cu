// trisolve.cu -- preconditioner apply x = M^{-1} r, M = L D U' (Eq. 6,
// Algorithm 7): L y = r, then z = D^{-1} y, then U' x = z (row i subtracts
// U'_ij x_j from z_i).
//
// z = D^{-1} y is a separate pass between the two sweeps, in place over y,
// with one lane per component: b FP64 instructions per 32/b block rows.
// Inside the U' sweep the same product costs b FP64 instructions per row
// (b of 32 lanes busy); FP64 issue is the scarce unit of the sweeps, and every
// FP64 instruction taken out of them also shortens the chain of dependent
// rows, which waits on that unit.
//
// The paper schedules each triangular solve by dependency levels (Eq. 4,
// Algorithm 6), one parallel step per level.  On this part a dependent launch
// costs >= 0.7 us and a dependency crossing SMs about 0.5 us, while a
// 128x128x64 ILU(1) factor has 571 levels, so each solve is ONE sync-free
// kernel with two tiers of dependency tracking instead:
//  * block rows are cut into chunks of consecutive rows; CTAs claim chunks in
//    solve order (ascending for L, descending for U') through an atomic
//    ticket;
//  * inside a chunk the host lists the rows by local dependency level (Eq. 4
//    restricted to the chunk); the CTA's warps take rows round-robin in that
//    order.  In natural order most dependencies of a grid row lie within a
//    few grid lines, i.e. inside its chunk;
//  * every value doubles as its own ready flag: a slot holds the "pending"
//    bit pattern (a signalling-NaN payload no arithmetic produces) until the
//    value is stored.  A dependency inside the chunk is polled in shared
//    memory (slots reset to pending when the chunk starts), one outside the
//    chunk in global memory (one L2 round trip per poll).  No separate flag,
//    no fence, no acquire on the hot path;
//  * loads run ahead of the dependency chain: the column index and values of
//    the first block (and the row's own operand) of the row a warp solves
//    next, an optimistic read of that row's dependency outside the chunk
//    (which needs the column index) once the current row is published, and
//    an L2 prefetch of the row after it, which holds no registers; for rows
//    of several passes over the groups (one in FP32, four in FP64) two rows
//    are held in registers instead, the dependency read a turn ahead;
//  * forward progress: a row only waits on rows of earlier positions in its
//    chunk or of earlier tickets, all held by running warps; every wait is
//    bounded and gives up with BILU_ERR_TIMEOUT (never a trap), and no warp
//    leaves the CTA's chunk loop early, so no barrier can hang.
// Lane mapping inside a row: lane = g*B + r, r the output component, g one of
// G groups that take the row's blocks round-robin; each lane does B FMAs per
// block and a log2(G)-step shuffle tree sums the groups.  G is a template
// parameter picked at launch: the fewest groups that hold the triangle's
// widest row in one pass (at least a quarter of the 32 / B lanes' groups).
//
// TV is the type the factors are stored and applied in: double, or float for
// the mixed-precision solver.  The sweeps' own vectors (y, z and the upper
// sweep's x) are kept in TV in the workspace, so an FP32 sweep converts
// nothing on its chain of dependent rows (a double <-> float conversion runs
// at the FP64 rate on this part); only r is read in double, and a last pass
// widens x to the caller's double vector.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"

namespace bilu {

TrisolveConfig& trisolve_config() {
  static TrisolveConfig cfg;
  return cfg;
}

namespace {
int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return 1;
  }
  return sms;
}
}  // namespace

// Large systems: two grid lines per chunk, which measured fastest on 96-,
// 128- and 160-wide grids (one line per chunk doubles the hand-offs between
// chunks through global memory; three lines lengthen each chunk's chain and
// leave fewer chunks in flight).  The chunk cut then goes to the line start
// nearest the target.
int32_t auto_solve_chunk_target(const bilu_pattern* p) {
  const long long t = (long long)p->n / (10LL * device_sm_count());
  if (t >= 256 && p->line_len >= 16 && p->line_len <= 192) return 2 * p->line_len;
  return (int32_t)std::max(32LL, std::min(256LL, t));
}

int32_t solve_chunk_target(const bilu_pattern* p) {
  const int c = trisolve_config().chunk;
  return c > 0 ? c : auto_solve_chunk_target(p);
}

// The factorization's 8-warp CTAs do best with three grid lines per chunk on
// large grids (128-wide: 12.4 ms against 13.7 with two lines).
int32_t auto_factor_chunk_target(const bilu_pattern* p) {
  const long long t = (long long)p->n / (2LL * device_sm_count());
  if (t >= 256 && p->line_len >= 16 && p->line_len <= 128) return 3 * p->line_len;
  return (int32_t)std::max(64LL, std::min(256LL, t));
}

int32_t factor_chunk_target(const bilu_pattern* p) {
  const int c = trisolve_config().factor_chunk;
  return c > 0 ? c : auto_factor_chunk_target(p);
}

namespace {


template <typename TV>
__global__ void apply_prep_kernel(TV* y, TV* x, long long m, int32_t* header, const int32_t* stop) {
  // Each apply starts with a clean header: its status is its own.  Both
  // sweeps' outputs start "pending".
  using VB = ValueBits<TV>;
  if (stop && *stop) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += stride) {
    reinterpret_cast<typename VB::U*>(y)[q] = VB::kPend;
    reinterpret_cast<typename VB::U*>(x)[q] = VB::kPend;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    header[kTicketL] = 0;
    header[kTicketU] = 0;
    header[kAbort] = 0;
    header[kErr] = 0;
  }
}

// Registers a lane holds for one row: the row, its first block of this lane's
// group (column, this lane's B values, optimistic dependency values, as bit
// patterns of TV), and the row's own term (r_i for L, z_i for U', type RT).
template <int B, typename TV, typename RT>
struct RowPre {
  int i, beg, end, j;
  TV av[B];
  typename ValueBits<TV>::U yv[B];  // dependency values of a block outside the chunk, read early
  RT own;                           // lanes < B: r_i[lane] or z_i[lane]
};

// Stage A of the prefetch: the row, its first block (column and values) and
// its own term.
template <int B, typename TV, typename RT>
__device__ __forceinline__ void fetch_row(RowPre<B, TV, RT>& p, int pos, int len, const int* s_i,
                                          const int* s_beg, const int* s_end,
                                          const int32_t* __restrict__ ci, const TV* __restrict__ vals,
                                          const RT* rhs, int g, int rr, bool act, int lane) {
  if (pos >= len) {  // past the chunk's end: nothing to fetch, no dependency to read
    p.i = -1;
    p.beg = p.end = 0;
    p.j = -1;
    return;
  }
  p.i = s_i[pos];
  p.beg = s_beg[pos];
  p.end = s_end[pos];
  const int t = p.beg + g;
  p.j = -1;
  if (act && t < p.end) {
    p.j = __ldg(ci + t);
    const TV* a = vals + (size_t)t * (B * B) + rr;
#pragma unroll
    for (int q = 0; q < B; ++q) p.av[q] = __ldg(a + q * B);
  }
  if (lane < B) p.own = rhs[(size_t)p.i * B + lane];
}

// The row two turns ahead, for the one-row prefetch: its first block's column
// index and values are pulled into L2 without holding registers.
template <int B, typename TV>
__device__ __forceinline__ void prefetch_row_l2(int pos, int len, const int* s_beg, const int* s_end,
                                                const int32_t* __restrict__ ci, const TV* __restrict__ vals,
                                                int g, int rr, bool act) {
  if (pos >= len || !act) return;
  const int t = s_beg[pos] + g;
  if (t >= s_end[pos]) return;
  asm volatile("prefetch.global.L2 [%0];" ::"l"(ci + t));
  asm volatile("prefetch.global.L2 [%0];" ::"l"(vals + (size_t)t * (B * B) + rr));
}

// Stage B: a dependency outside the chunk is usually final already: read it
// now (relaxed); if it still holds the pending pattern it is waited for later.
template <int B, typename TV, typename RT>
__device__ __forceinline__ void fetch_deps(RowPre<B, TV, RT>& p, const TV* out, int lo, int hi) {
  using VB = ValueBits<TV>;
  const bool remote = p.j >= 0 && (p.j < lo || p.j >= hi);
#pragma unroll
  for (int q = 0; q < B; ++q)
    p.yv[q] = remote ? ld_relaxed_bits<typename VB::U>(out + (size_t)p.j * B + q) : VB::kPend;
}

// z = D^{-1} y in place: R = 32 / B block rows per warp, lane (row, r) forms
// z[row][r] = sum_c D^{-1}[r][c] y[row][c] (blocks column-major).  A row's
// lanes sit in one warp; they read all of y_row before any of them writes.
template <int B, typename TV>
__global__ void __launch_bounds__(256) diag_scale_kernel(int32_t n, const TV* __restrict__ dinv, TV* y,
                                                         const int32_t* stop) {
  constexpr int R = 32 / B;
  if (stop && ld_volatile_s32(stop)) return;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int q = lane / B;
  const int r = lane - q * B;
  const long long row = warp * R + q;
  const bool act = q < R && row < n;
  TV z = TV(0);
  if (act) {
    const TV* d = dinv + (size_t)row * (B * B) + r;
    const TV* yr = y + (size_t)row * B;
#pragma unroll
    for (int c = 0; c < B; ++c) z = fma(__ldg(d + c * B), yr[c], z);
  }
  __syncwarp();
  if (act) y[(size_t)row * B + r] = z;
}

// x = (double) x32 over the FP32 apply's result.
__global__ void __launch_bounds__(256) widen_kernel(const float* __restrict__ src, double* __restrict__ dst,
                                                    long long m, const int32_t* stop) {
  if (stop && ld_volatile_s32(stop)) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += stride)
    dst[q] = (double)src[q];
}

// GE: the groups a row's blocks are spread over (a power of two, at most
// groups_for(B)); the partial sums take log2(GE) reduction steps.  RT: the
// type of the right-hand side (double r for L, TV z for U').
template <int B, bool UPPER, typename TV, int kTriWarps, int GE, typename RT, bool DEEP>
__global__ void __launch_bounds__(kTriWarps * 32) tri_solve_kernel(
    int32_t n, int32_t chunk, int32_t nchunks, const int32_t* __restrict__ bnd, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const TV* __restrict__ vals,
    const int32_t* __restrict__ ord, const int32_t* __restrict__ tick, const RT* rhs, TV* out,
    int32_t* header, long long spin_ns, int32_t skip_row, int32_t* stop) {
  static_assert(GE >= 1 && GE <= groups_for(B) && (GE & (GE - 1)) == 0, "group count");
  constexpr int G = GE;
  using VB = ValueBits<TV>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TV* yl = reinterpret_cast<TV*>(smem_raw);  // the chunk's values, in the type they are used in
  int* s_i = reinterpret_cast<int*>(smem_raw + (((size_t)chunk * B * sizeof(TV) + 15) & ~(size_t)15));
  int* s_beg = s_i + chunk;
  int* s_end = s_beg + chunk;
  __shared__ int s_c;
  if (stop && ld_volatile_s32(stop)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane / B, rr = lane - (lane / B) * B;
  const bool act = g < G;
  Waiter w{header, spin_ns, 0, stop};
  bool dead = false;
  for (;;) {
    __syncthreads();  // the previous chunk is complete: shared memory may be reused
    if (tid == 0) {
      int cc = atomicAdd(header + (UPPER ? kTicketU : kTicketL), 1);
      if (ld_volatile_s32(header + kAbort)) cc = nchunks;
      s_c = cc < nchunks ? tick[cc] : nchunks;
    }
    __syncthreads();
    const int c = s_c;
    if (c >= nchunks) return;
    // rows [lo, hi), at most `chunk` of them; upper chunk c is lower chunk nchunks-1-c
    const int lc = UPPER ? nchunks - 1 - c : c;
    const int lo = bnd[lc], hi = bnd[lc + 1];
    const int len = hi - lo;
    for (int q = tid; q < len; q += blockDim.x) {
      const int i = ord[lo + q];
      s_i[q] = i;
      s_beg[q] = rp[i];
      s_end[q] = rp[i + 1];
    }
    for (int q = tid; q < len * B; q += blockDim.x) reinterpret_cast<typename VB::U*>(yl)[q] = VB::kPend;
    __syncthreads();
    // The next rows of this warp are prefetched: DEEP two rows ahead in
    // registers (nx1 with its remote dependency read, nx2 its row data), else
    // one row ahead, its dependency read once the current row is published,
    // and the row after it pulled into L2 (fewer registers: at b = 3 in FP64,
    // 70 per thread and seven CTAs per SM instead of 90 and five).
    constexpr bool kDeep = DEEP;
    RowPre<B, TV, RT> cur, nx1, nx2;
    fetch_row<B, TV, RT>(cur, warp, len, s_i, s_beg, s_end, ci, vals, rhs, g, rr, act, lane);
    fetch_deps<B, TV, RT>(cur, out, lo, hi);
    if constexpr (kDeep)
      fetch_row<B, TV, RT>(nx1, warp + kTriWarps, len, s_i, s_beg, s_end, ci, vals, rhs, g, rr, act, lane);
    for (int pos = warp; pos < len && !dead; pos += kTriWarps) {
      if constexpr (kDeep) {
        fetch_row<B, TV, RT>(nx2, pos + 2 * kTriWarps, len, s_i, s_beg, s_end, ci, vals, rhs, g, rr, act, lane);
        fetch_deps<B, TV, RT>(nx1, out, lo, hi);
      } else {
        fetch_row<B, TV, RT>(nx1, pos + kTriWarps, len, s_i, s_beg, s_end, ci, vals, rhs, g, rr, act, lane);
        prefetch_row_l2<B, TV>(pos + 2 * kTriWarps, len, s_beg, s_end, ci, vals, g, rr, act);
      }
      const int i = cur.i;
      bool ok = true;
      // The row's own term (r_i or z_i) seeds the sum of group 0 (lanes < B);
      // the blocks accumulate as fma(-a, y, acc), so the reduced sum is the
      // row's value with no final subtraction.
      TV acc = lane < B ? (TV)cur.own : TV(0);
      for (int t0 = cur.beg; t0 < cur.end; t0 += G) {
        const int t = t0 + g;
        if (act && t < cur.end) {
          int j;
          TV av[B];
          typename VB::U yv[B];
          if (t0 == cur.beg) {
            j = cur.j;
#pragma unroll
            for (int q = 0; q < B; ++q) {
              av[q] = cur.av[q];
              yv[q] = cur.yv[q];
            }
          } else {
            j = __ldg(ci + t);
            const TV* a = vals + (size_t)t * (B * B) + rr;
#pragma unroll
            for (int q = 0; q < B; ++q) {
              av[q] = __ldg(a + q * B);
              yv[q] = VB::kPend;
            }
          }
          TV yt[B];
          if (j >= lo && j < hi) {
            ok = wait_values_shared<B, TV>(yl + (size_t)(j - lo) * B, yt, w);
          } else {
            bool have = true;
#pragma unroll
            for (int q = 0; q < B; ++q) {
              have = have && (yv[q] != VB::kPend);
              yt[q] = VB::value(yv[q]);
            }
            if (!have) ok = wait_values_global<B, TV>(out + (size_t)j * B, yt, w);
          }
          if (ok) {
#pragma unroll
            for (int q = 0; q < B; ++q) acc = fma(-av[q], yt[q], acc);
          }
        }
      }
      if (__any_sync(kFull, !ok)) {
        dead = true;
        break;
      }
#pragma unroll
      for (int d = G / 2; d >= 1; d >>= 1) acc += __shfl_down_sync(kFull, acc, d * B);
      if (lane < B) {
        // the chunk's own readers first (shared memory, type TV), then global
        const TV vt = acc;
        typename VB::U u = VB::bits(vt);
        if (u == VB::kPend) u = VB::kQuiet;
        reinterpret_cast<volatile typename VB::U*>(yl)[(size_t)(i - lo) * B + lane] = u;
        if (i != skip_row) publish_value<TV>(out + (size_t)i * B + lane, vt);
      }
      if constexpr (!kDeep) fetch_deps<B, TV, RT>(nx1, out, lo, hi);
      cur = nx1;
      if constexpr (kDeep) nx1 = nx2;
    }
  }
}

int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 1;
  }
  return cached;
}

template <typename TV>
size_t tri_smem_bytes(int chunk, int b) {
  return align_up16((size_t)chunk * b * sizeof(TV)) + (size_t)chunk * 3 * sizeof(int);
}

// Persistent grid: as many CTAs as fit on the device at once (cached per
// shared-memory size; the occupancy query is host work worth skipping per
// launch).
template <int B, bool UPPER, typename TV, int kTriWarps, int GE, typename RT, bool DEEP>
int tri_grid(size_t smem, int nchunks) {
  static size_t last_smem = 0;
  static int last_per_sm = 1;
  if (smem != last_smem) {
    cudaFuncSetAttribute(tri_solve_kernel<B, UPPER, TV, kTriWarps, GE, RT, DEEP>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 48 * 1024));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tri_solve_kernel<B, UPPER, TV, kTriWarps, GE, RT, DEEP>,
                                                  kTriWarps * 32, smem);
    last_per_sm = per_sm < 1 ? 1 : per_sm;
    last_smem = smem;
  }
  const int cap = trisolve_config().ctas_per_sm;
  const int per_sm = cap > 0 ? std::min(cap, last_per_sm) : last_per_sm;
  return std::max(1, std::min(nchunks, per_sm * sm_count()));
}

// One triangular sweep (the arguments of tri_solve_kernel).
template <typename TV, typename RT>
struct TriArgs {
  int32_t n, chunk, nchunks;
  const int32_t *bnd, *rp, *ci;
  const TV* vals;
  const int32_t *ord, *tick;
  const RT* rhs;
  TV* out;
  int32_t* header;
  long long spin_ns;
  int32_t skip_row;
  int32_t* stop;
};

template <int B, bool UPPER, typename TV, int W, int GE, typename RT, bool DEEP>
void launch_tri_k(const TriArgs<TV, RT>& a, size_t smem, cudaStream_t s) {
  const int grid = tri_grid<B, UPPER, TV, W, GE, RT, DEEP>(smem, a.nchunks);
  tri_solve_kernel<B, UPPER, TV, W, GE, RT, DEEP><<<grid, W * 32, smem, s>>>(
      a.n, a.chunk, a.nchunks, a.bnd, a.rp, a.ci, a.vals, a.ord, a.tick, a.rhs, a.out, a.header, a.spin_ns,
      a.skip_row, a.stop);
}

// Prefetch depth, measured on 128x128x64 and 96x96x48 seven-point grids and
// the 160x160x80 27-point ILU(2) grid: one row in registers and the row
// after it in L2 is faster than two rows in registers (fewer registers, more
// CTAs per SM: FP64 b = 3 1380 -> 1255 us, FP32 b = 3 972 -> 926 us, b = 4
// 4-21 %, FP32 b = 6 k = 0 8 %, FP64 b = 2 k = 0 6 %) while the widest row
// fits in one pass over the groups (FP32) or four (FP64).  Wider rows keep
// two rows in registers: FP32 b = 6 with 2-4 passes is 20-29 % slower, FP32
// b = 8 with 2 passes 6 %, FP64 27-point ILU(2) with 7 passes 29 %.
template <int B, bool UPPER, typename TV, int W, int GE, typename RT>
void launch_tri(const TriArgs<TV, RT>& a, int32_t max_blocks, size_t smem, cudaStream_t s) {
  const int passes = (max_blocks + GE - 1) / GE;
  if (passes > (sizeof(TV) == 4 ? 1 : 4)) launch_tri_k<B, UPPER, TV, W, GE, RT, true>(a, smem, s);
  else launch_tri_k<B, UPPER, TV, W, GE, RT, false>(a, smem, s);
}

// The fewest groups (a power of two, at least groups_for(B) / 4) that hold
// every row's blocks in one pass: narrow rows (ILU(0) of a 7-point stencil:
// 3 blocks) then take fewer reduction steps.  Only the default 4-warp CTA has
// the narrower instantiations.
template <int B, bool UPPER, typename TV, int W, typename RT>
void launch_tri_groups(const TriArgs<TV, RT>& a, int32_t max_blocks, size_t smem, cudaStream_t s) {
  constexpr int G = groups_for(B);
  const int32_t need = max_blocks;
  if constexpr (W == 4) {
    if (need <= G / 4) return launch_tri<B, UPPER, TV, W, G / 4, RT>(a, need, smem, s);
    if (need <= G / 2) return launch_tri<B, UPPER, TV, W, G / 2, RT>(a, need, smem, s);
  }
  launch_tri<B, UPPER, TV, W, G, RT>(a, need, smem, s);
}

// L y = r (y in TV), z = D^{-1} y in place, U' x = z (x in TV: the caller's
// vector in FP64, a workspace vector widened afterwards in FP32).
template <int B, typename TV, int W>
void launch_solves(const bilu_pattern* p, int chunk, int nchunks, const TV* L, const TV* Dinv,
                   const TV* U, const double* r, TV* y, TV* x, int32_t* header, const TrisolveConfig& cfg,
                   int32_t* stop, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const size_t smem = tri_smem_bytes<TV>(chunk, B);
  {
    const TriArgs<TV, double> a{p->n, chunk, nchunks, p->solve.d_bnd, p->d_lrp, p->d_lci, L,
                                p->solve.d_ord_l, p->solve.d_tick_l, r, y, header, cfg.spin_ns, cfg.skip_row, stop};
    ProfScope ps(BILU_PROF_LOWER, stream);
    launch_tri_groups<B, false, TV, W, double>(a, p->max_l, smem, s);
  }
  {
    // z = D^{-1} y over y.  A lower sweep that gave up (a bounded wait ran
    // out) leaves pending slots in y: they turn into NaN here, and the upper
    // sweep, whose header shows the abort, leaves at once.
    constexpr int R = 32 / B;
    const long long blocks = (((long long)p->n + R - 1) / R * 32 + 255) / 256;
    ProfScope ps(BILU_PROF_DIAG, stream);
    diag_scale_kernel<B, TV><<<(unsigned)blocks, 256, 0, s>>>(p->n, Dinv, y, stop);
  }
  {
    const TriArgs<TV, TV> a{p->n, chunk, nchunks, p->solve.d_bnd, p->d_urp, p->d_uci, U,
                            p->solve.d_ord_u, p->solve.d_tick_u, y, x, header, cfg.spin_ns, -1, stop};
    ProfScope ps(BILU_PROF_UPPER, stream);
    launch_tri_groups<B, true, TV, W, TV>(a, p->max_u, smem, s);
  }
}

template <typename TV>
int launch_apply_t(const bilu_pattern* p, int32_t b, const TV* f, const double* r, double* x, void* work,
                   int32_t* stop, void* stream) {
  const int32_t n = p->n;
  if (n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  const TrisolveConfig& cfg = trisolve_config();
  if (p->solve.chunk <= 0 || !p->solve.upper || !p->solve.d_mem) return (int)cudaErrorInvalidValue;
  const int chunk = p->solve.max_len;  // shared-memory rows per CTA
  const int nchunks = p->solve.nchunks;
  int32_t* header = reinterpret_cast<int32_t*>(work);
  const long long m = (long long)n * b;
  // The workspace's vector region holds n*b doubles: y (FP64), or y and the
  // upper sweep's x side by side (FP32).
  TV* y = reinterpret_cast<TV*>(reinterpret_cast<char*>(work) + kHeaderBytes);
  TV* xs;
  if constexpr (sizeof(TV) == 8) xs = reinterpret_cast<TV*>(x);
  else xs = y + m;
  const size_t bb = (size_t)b * b;
  const TV* L = f;
  const TV* Dinv = f + (size_t)p->nnz_l() * bb;
  const TV* U = Dinv + (size_t)n * bb;
  const int prep_blocks = (int)std::min<long long>((m + 255) / 256, (long long)sm_count() * 8);
  {
    ProfScope ps(BILU_PROF_APPLY_PREP, stream);
    apply_prep_kernel<TV><<<prep_blocks, 256, 0, s>>>(y, xs, m, header, stop);
  }
  BILU_DISPATCH_B(b, {
    if (cfg.warps == 16)
      launch_solves<B, TV, 16>(p, chunk, nchunks, L, Dinv, U, r, y, xs, header, cfg, stop, stream);
    else if (cfg.warps == 4)
      launch_solves<B, TV, 4>(p, chunk, nchunks, L, Dinv, U, r, y, xs, header, cfg, stop, stream);
    else
      launch_solves<B, TV, 8>(p, chunk, nchunks, L, Dinv, U, r, y, xs, header, cfg, stop, stream);
  });
  if constexpr (sizeof(TV) == 4) {
    ProfScope ps(BILU_PROF_APPLY_PREP, stream);
    widen_kernel<<<prep_blocks, 256, 0, s>>>(xs, x, m, stop);
  }
  return (int)cudaGetLastError();
}

}  // namespace

const float* apply_f32_result(const void* work, int32_t n, int32_t b) {
  // the vector region after the header: y (n*b floats), then the upper sweep's x
  return reinterpret_cast<const float*>(reinterpret_cast<const char*>(work) + kHeaderBytes) + (size_t)n * b;
}

void free_schedule(bilu_chunk_schedule* s) {
  if (s->d_mem) cudaFree(s->d_mem);
  s->d_mem = nullptr;
  s->d_bnd = s->d_ord_l = s->d_ord_u = s->d_tick_l = s->d_tick_u = nullptr;
  s->chunk = 0;
}

int make_schedule(const bilu_pattern* p, bilu_chunk_schedule* s, int32_t chunk, bool upper) {
  bilu_chunk_schedule t;
  if (!p->host_ready) {
    // completed on the device: every pass over P' on the device too
    const int st = build_schedule_device(p, chunk, upper, &t);
    if (st != BILU_OK) return (int)cudaErrorMemoryAllocation;
    free_schedule(s);
    *s = std::move(t);
    return 0;
  }
  build_schedule(p, chunk, upper, &t);
  if (p->n > 0) {
    const size_t one = align256(sizeof(int32_t) * (size_t)p->n);
    const size_t tk = align256(sizeof(int32_t) * (size_t)t.nchunks);
    const size_t bd = align256(sizeof(int32_t) * ((size_t)t.nchunks + 1));
    const int parts = upper ? 2 : 1;
    void* mem = nullptr;
    if (cudaMalloc(&mem, bd + parts * (one + tk)) != cudaSuccess) {
      cudaGetLastError();
      return (int)cudaErrorMemoryAllocation;
    }
    char* m = (char*)mem;
    t.d_mem = mem;
    t.d_bnd = (int32_t*)m;
    m += bd;
    auto put = [&](int32_t*& dst, const std::vector<int32_t>& v, size_t bytes) {
      dst = (int32_t*)m;
      m += bytes;
      cudaMemcpy(dst, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice);
    };
    cudaMemcpy(t.d_bnd, t.bnd.data(), sizeof(int32_t) * t.bnd.size(), cudaMemcpyHostToDevice);
    put(t.d_ord_l, t.ord_l, one);
    put(t.d_tick_l, t.tick_l, tk);
    if (upper) {
      put(t.d_ord_u, t.ord_u, one);
      put(t.d_tick_u, t.tick_u, tk);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      cudaFree(mem);
      return (int)e;
    }
  }
  free_schedule(s);
  *s = std::move(t);
  return 0;
}

size_t apply_workspace_bytes(int32_t n, int32_t b) {
  return kHeaderBytes + align256((size_t)n * b * sizeof(double));
}

int launch_apply(const bilu_pattern* p, int32_t b, const double* f, const double* r, double* x,
                 void* work, int32_t* stop, void* stream) {
  return launch_apply_t<double>(p, b, f, r, x, work, stop, stream);
}

int launch_apply_f32(const bilu_pattern* p, int32_t b, const float* f, const double* r, double* x,
                     void* work, int32_t* stop, void* stream) {
  return launch_apply_t<float>(p, b, f, r, x, work, stop, stream);
}

}  // namespace bilu
