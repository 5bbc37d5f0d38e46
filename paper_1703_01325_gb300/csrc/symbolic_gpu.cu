// symbolic_gpu.cu -- the symbolic phase (Section 2.2, Algorithm 3 with Eq. 1
// and Eq. 2) on the device, bit-identical to the host phase in symbolic.cpp.
//
// Row i of P' is the same pivot-driven merge as on the host: start from A's
// row (Eq. 1: level 0), take the pivots p < i of level <= k in ascending
// column order (a pivot's level is final when it is reached, since only
// smaller pivots lower it), and for each merge row p's final upper part into
// the row with the sum rule lev_ij = min(lev_ij, lev_ip + lev_pj + 1) (Eq. 2),
// discarding candidates above k at once (a level only decreases).  Integer
// arithmetic, same pivot order: the same P' and levels.
//
// One warp per row; rows are claimed in ascending order through an atomic
// ticket and row i waits (bounded, acquire) for each pivot row p < i to be
// published, so the earliest unfinished row never waits on an unfinished row.
// The row is held in shared memory as a sorted (column, level) list of at
// most `cap` entries; a merge step takes 32 candidates of row p at a time:
// each lane binary-searches its column, found columns take the smaller level,
// new columns are inserted by one pass that shifts the list (the rank of each
// new column among the batch and the number of new columns before each old
// entry give every destination).  A row that outgrows `cap` stops the run with
// BILU_ERR_OOM (the caller retries with a larger capacity or the host phase).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <new>
#include <vector>

#include "device_common.cuh"

namespace bilu {
namespace {

constexpr int kSymWarps = 4;

// First index in a[0, len) whose value is >= key (a row of this warp, in
// shared memory).
__device__ __forceinline__ int lower_bound_i32(const int* a, int len, int key) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// First index in a[0, len) whose value is >= key (a row another warp
// published: L2 loads, never a line this SM cached before the publication).
__device__ __forceinline__ int lower_bound_pub(const int* a, int len, int key) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldcg(a + mid) < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Number of entries of the sorted a[0, len) that are <= key.
__device__ __forceinline__ int count_le(const int* a, int len, int key) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kSymWarps * 32) symbolic_kernel(
    int32_t n, int32_t k, int32_t cap, const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
    int32_t* ocol, int32_t* olev, int32_t* olen, int32_t* done, int32_t* header, long long spin_ns) {
  extern __shared__ int sym_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* C = sym_smem + (size_t)warp * (4 * (size_t)cap + 32);  // columns of the row (sorted)
  int* Lv = C + cap;                                           // their levels
  int* Cn = Lv + cap;                                          // merge destination
  int* Ln = Cn + cap;
  int* newpos = Ln + cap;  // insertion points of the new columns of a batch (32)
  Waiter w{header, spin_ns, 0, nullptr};
  for (;;) {
    int i = 0;
    if (lane == 0) {
      i = atomicAdd(header + kTicketF, 1);
      if (ld_volatile_s32(header + kAbort)) i = n;
    }
    i = __shfl_sync(kFull, i, 0);
    if (i >= n) return;
    const int ab = arp[i], na = arp[i + 1] - ab;
    int err = na > cap ? (int)BILU_ERR_OOM : 0;
    int len = err ? 0 : na;
    for (int t = lane; t < len; t += 32) {  // Eq. 1
      C[t] = aci[ab + t];
      Lv[t] = 0;
    }
    __syncwarp();
    int pos = 0;  // the next pivot is searched from here
    while (!err) {
      // next pivot: first entry at or after pos with column < i and level <= k
      int q = -1;
      for (int base = pos; base < len; base += 32) {
        const int idx = base + lane;
        const bool inr = idx < len;
        const int col = inr ? C[idx] : INT_MAX;
        const unsigned past = __ballot_sync(kFull, inr && col >= i);
        unsigned hit = __ballot_sync(kFull, inr && col < i && Lv[idx] <= k);
        if (past) hit &= (past & (0u - past)) - 1u;  // only entries before the first column >= i
        if (hit) {
          q = base + __ffs(hit) - 1;
          break;
        }
        if (past) break;
      }
      if (q < 0) break;
      const int p = C[q], lp = Lv[q];
      pos = q + 1;  // new columns are > p: entries up to q never move
      int ok = 1;
      if (lane == 0) ok = wait_flag(done + p, w) ? 1 : 0;
      ok = __shfl_sync(kFull, ok, 0);
      __syncwarp();  // lane 0's acquire orders the whole warp's reads of row p
      if (!ok) {
        err = BILU_ERR_TIMEOUT;
        break;
      }
      // row p's final upper part: its entries after the diagonal
      const int* pc = ocol + (size_t)p * cap;
      const int* pl = olev + (size_t)p * cap;
      const int plen = __ldcg(olen + p);
      const int dp = lower_bound_pub(pc, plen, p);
      for (int u0 = dp + 1; u0 < plen && !err; u0 += 32) {
        const int u = u0 + lane;
        int jb = 0;
        long long lb = LLONG_MAX;
        if (u < plen) {
          jb = __ldcg(pc + u);
          lb = (long long)lp + __ldcg(pl + u) + 1;  // Eq. 2
        }
        const bool valid = u < plen && lb <= k;
        int pb = 0;
        bool found = false;
        if (valid) {
          pb = lower_bound_i32(C, len, jb);
          found = pb < len && C[pb] == jb;
          if (found && lb < Lv[pb]) Lv[pb] = (int)lb;
        }
        const bool isnew = valid && !found;
        const unsigned nm = __ballot_sync(kFull, isnew);
        const int nnew = __popc(nm);
        __syncwarp();
        if (nnew == 0) continue;
        if (len + nnew > cap) {
          err = BILU_ERR_OOM;
          break;
        }
        const int rank = __popc(nm & ((1u << lane) - 1u));
        if (isnew) newpos[rank] = pb;
        __syncwarp();
        for (int e = lane; e < len; e += 32) {
          const int sh = count_le(newpos, nnew, e);  // new columns inserted before entry e
          Cn[e + sh] = C[e];
          Ln[e + sh] = Lv[e];
        }
        if (isnew) {
          Cn[pb + rank] = jb;
          Ln[pb + rank] = (int)lb;
        }
        __syncwarp();
        int* tc = C; C = Cn; Cn = tc;
        int* tl = Lv; Lv = Ln; Ln = tl;
        len += nnew;
      }
    }
    if (err) {  // publish an empty row so that no waiter hangs, and stop the run
      if (lane == 0) {
        atomicCAS(header + kErr, 0, err);
        atomicMin(header + kBadRow, i);
        atomicExch(header + kAbort, 1);
      }
      len = 0;
    }
    for (int t = lane; t < len; t += 32) {
      ocol[(size_t)i * cap + t] = C[t];
      olev[(size_t)i * cap + t] = Lv[t];
    }
    if (lane == 0) olen[i] = len;
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release_s32(done + i, 1);
  }
}

// ---- completion of the pattern on the device (Eq. 4, L / U' split,
// backfill map), so that no host pass over P' is needed ----

// Statistics words (device scratch).
enum StatWord : int { kMaxL = 0, kMaxU = 1, kNlevL = 2, kNlevU = 3, kStatWords = 8 };

// Per row of P' (capacity layout, columns sorted, the diagonal present): its
// length, the blocks left (nl) and right (nu) of the diagonal, and whether
// the row depends on its predecessor (its last lower column is i - 1: the
// rows that do not start grid lines in a natural ordering).
__global__ void row_info_kernel(int32_t n, int32_t cap, const int32_t* __restrict__ ocol,
                                const int32_t* __restrict__ olen, int32_t* __restrict__ nl,
                                int32_t* __restrict__ nu, int32_t* __restrict__ linestart, int32_t* stats) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int32_t* c = ocol + (size_t)i * cap;
    const int len = olen[i];
    int lo = 0, hi = len;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (c[mid] < (int)i) lo = mid + 1;
      else hi = mid;
    }
    const int dp = lo;  // position of the diagonal
    nl[i] = dp;
    nu[i] = len - dp - 1;
    linestart[i] = (dp > 0 && c[dp - 1] == (int)i - 1) ? 0 : 1;
    atomicMax(stats + kMaxL, dp);
    atomicMax(stats + kMaxU, len - dp - 1);
  }
}

// Exclusive scan of n int32 counts into out[0..n] (out[n] = total), in three
// launches: per-block scans of kScanTile values, a scan of the block sums (one
// block), and the offsets added back.  The total is also left, as 64 bits, in
// part[nparts] for the caller to check against the int32 range.
constexpr int kScanTile = 1024;

__device__ __forceinline__ long long block_exscan(long long v, long long* wsum, long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long y = __shfl_up_sync(kFull, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    long long z = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long y = __shfl_up_sync(kFull, z, d);
      if (lane >= d) z += y;
    }
    wsum[lane] = z - w;  // exclusive prefix of the warp sums
    if (lane == 31) *total = z;
  }
  __syncthreads();
  const long long r = wsum[warp] + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanTile) scan_tiles_kernel(const int32_t* __restrict__ in, long long n,
                                                               int32_t* __restrict__ out, long long* part) {
  __shared__ long long wsum[32];
  __shared__ long long total;
  const long long i = (long long)blockIdx.x * kScanTile + threadIdx.x;
  const long long v = i < n ? in[i] : 0;
  const long long e = block_exscan(v, wsum, &total);
  if (i < n) out[i] = (int32_t)e;  // within-tile prefix; offsets come later
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanTile) scan_parts_kernel(long long* part, long long nparts) {
  __shared__ long long wsum[32];
  __shared__ long long total;
  long long carry = 0;
  for (long long b0 = 0; b0 < nparts; b0 += kScanTile) {
    const long long q = b0 + threadIdx.x;
    const long long v = q < nparts ? part[q] : 0;
    const long long e = block_exscan(v, wsum, &total);
    if (q < nparts) part[q] = carry + e;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) part[nparts] = carry;
}

__global__ void scan_add_kernel(int32_t* out, long long n, const long long* part, long long nparts) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)((long long)out[i] + part[i / kScanTile]);
  if (i == 0) out[n] = (int32_t)part[nparts];
}

// P' compacted from the capacity layout (ci, lev) and split into its strictly
// lower (lci) and strictly upper (uci) parts; one warp per row.
__global__ void split_kernel(int32_t n, int32_t cap, const int32_t* __restrict__ ocol,
                             const int32_t* __restrict__ olev, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ lrp, const int32_t* __restrict__ urp,
                             int32_t* __restrict__ ci, int32_t* __restrict__ lev, int32_t* __restrict__ lci,
                             int32_t* __restrict__ uci) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
    const int beg = rp[i], len = rp[i + 1] - beg;
    const int dp = lrp[i + 1] - lrp[i];
    for (int t = lane; t < len; t += 32) {
      const int c = ocol[(size_t)i * cap + t];
      ci[beg + t] = c;
      lev[beg + t] = olev[(size_t)i * cap + t];
      if (t < dp) lci[lrp[i] + t] = c;
      else if (t > dp) uci[urp[i] + t - dp - 1] = c;
    }
  }
}

__device__ __forceinline__ int ld_relaxed_s32(const int32_t* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_s32(int32_t* p, int v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Eq. 4 on the device: l(i) = 1 + max l(j) over the dependencies j of row i
// (0 for a row without any), 0-based, for L (j < i, rows ascending) or for
// the reversed graph of U' (j > i, rows descending).  Sync-free: warps claim
// rows in solve order through a ticket, so a row only waits on rows whose
// tickets were handed out before, all held by running warps; done[j] holds
// l(j) + 1 once known (0 = pending) and is itself the flag.  The waits are
// warp-uniform (the whole warp re-reads until no lane sees a pending value)
// and bounded: one that runs out records BILU_ERR_TIMEOUT and every warp
// leaves.
template <bool UPPER>
__global__ void __launch_bounds__(256) eq4_level_kernel(int32_t n, const int32_t* __restrict__ rpv,
                                                        const int32_t* __restrict__ civ, int32_t* done,
                                                        int32_t* __restrict__ lvl, int32_t* header, int32_t* stats,
                                                        long long spin_ns) {
  const int lane = threadIdx.x & 31;
  Waiter w{header, spin_ns, 0, nullptr};
  for (;;) {
    int tk = 0;
    if (lane == 0) {
      tk = atomicAdd(header + (UPPER ? kTicketU : kTicketL), 1);
      if (ld_volatile_s32(header + kAbort)) tk = n;
    }
    tk = __shfl_sync(kFull, tk, 0);
    if (tk >= n) return;
    const int i = UPPER ? n - 1 - tk : tk;
    const int beg = rpv[i], end = rpv[i + 1];
    int m = 0;
    bool ok = true;
    for (int t0 = beg; t0 < end && ok; t0 += 32) {
      const int t = t0 + lane;
      const bool has = t < end;
      const int j = has ? civ[t] : i;
      int v = has ? ld_relaxed_s32(done + j) : 1;
      w.t0 = 0;
      for (unsigned it = 1;; ++it) {
        if (__all_sync(kFull, v != 0)) break;
        if ((it & 31u) == 0u && __any_sync(kFull, w.give_up(0u, 0u))) {
          ok = false;
          break;
        }
        const int v2 = ld_relaxed_s32(done + j);  // every lane re-reads (no per-lane branch)
        v = v != 0 ? v : v2;
      }
      m = max(m, has ? v : 0);
    }
    if (!ok) return;  // the abort word stops every other warp
    m = __reduce_max_sync(kFull, m);
    if (lane == 0) {
      lvl[i] = m;
      st_relaxed_s32(done + i, m + 1);
      atomicMax(stats + (UPPER ? kNlevU : kNlevL), m + 1);
    }
  }
}

// Backfill gather map (Algorithm 5 steps 3-4): the factor slot of every block
// t of A, found by a binary search of its column in row i of P' -- slot
// lrp[i] + pos in L, nnz_l + i for the diagonal, nnz_l + n + urp[i] + pos - nl
// - 1 in U' -- gets t; slots no block of A lands in keep -1 (fill).  One warp
// per row of A.
__global__ void slot_map_kernel(int32_t n, const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const int32_t* __restrict__ lrp, const int32_t* __restrict__ urp, long long nnz_l,
                                int32_t* __restrict__ slot_src) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
    const int pb = rp[i], plen = rp[i + 1] - pb;
    const int nli = lrp[i + 1] - lrp[i];
    for (int t = arp[i] + lane; t < arp[i + 1]; t += 32) {
      const int j = aci[t];
      int lo = 0, hi = plen;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ci[pb + mid] < j) lo = mid + 1;
        else hi = mid;
      }
      long long slot;
      if (lo < nli) slot = lrp[i] + lo;
      else if (lo == nli) slot = nnz_l + i;
      else slot = nnz_l + n + urp[i] + (lo - nli - 1);
      slot_src[slot] = t;
    }
  }
}

// Line length: the histogram of the distances (up to 4096) between
// consecutive rows that do not depend on their predecessor; `idx` is the
// exclusive scan of the line-start flags, so row i with a flag is the idx[i]-th
// such row and starts[] lists them in order.
__global__ void line_starts_kernel(int32_t n, const int32_t* __restrict__ flag, const int32_t* __restrict__ idx,
                                   int32_t* __restrict__ starts) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    if (flag[i]) starts[idx[i]] = (int32_t)i;
}

__global__ void line_hist_kernel(int32_t count, const int32_t* __restrict__ starts, int32_t* __restrict__ hist) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x + 1; q < count; q += stride) {
    const int d = starts[q] - starts[q - 1];
    if (d <= 4096) atomicAdd(hist + d, 1);
  }
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  bool alloc(size_t bytes) { return cudaMalloc(&p, std::max<size_t>(bytes, 4)) == cudaSuccess; }
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

}  // namespace
}  // namespace bilu

using namespace bilu;

extern "C" int bilu_symbolic_gpu(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t k,
                                 int32_t row_capacity, void* stream, bilu_pattern** out) {
  if (!out || k < 0 || row_capacity < 1 || row_capacity > 8192) return BILU_ERR_ARG;
  *out = nullptr;
  const int st0 = validate_pattern(n, row_ptr, col_idx);
  if (st0 != BILU_OK) return st0;
  if (n == 0) return bilu_symbolic(n, row_ptr, col_idx, k, out);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nnz_a = row_ptr[n];
  const int cap = row_capacity;
  DevBuf d_arp, d_aci, d_ocol, d_olev, d_olen, d_done, d_header;
  if (!d_arp.alloc(sizeof(int32_t) * ((size_t)n + 1)) || !d_aci.alloc(sizeof(int32_t) * (size_t)nnz_a) ||
      !d_ocol.alloc(sizeof(int32_t) * (size_t)n * cap) || !d_olev.alloc(sizeof(int32_t) * (size_t)n * cap) ||
      !d_olen.alloc(sizeof(int32_t) * (size_t)n) || !d_done.alloc(sizeof(int32_t) * (size_t)n) ||
      !d_header.alloc(kHeaderBytes)) {
    cudaGetLastError();
    return BILU_ERR_OOM;
  }
  int32_t hdr[kHeaderWords] = {};
  hdr[kBadRow] = INT_MAX;
  cudaMemcpyAsync(d_arp.p, row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_aci.p, col_idx, sizeof(int32_t) * (size_t)nnz_a, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_header.p, hdr, sizeof(hdr), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(d_done.p, 0, sizeof(int32_t) * (size_t)n, s);
  const size_t smem = (size_t)kSymWarps * (4 * (size_t)cap + 32) * sizeof(int);
  if (smem > 227 * 1024) return BILU_ERR_ARG;
  cudaFuncSetAttribute(symbolic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)std::max<size_t>(smem, 48 * 1024));
  int dev = 0, sms = 1, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, symbolic_kernel, kSymWarps * 32, smem);
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + kSymWarps - 1) / kSymWarps,
                                                                    (long long)std::max(per_sm, 1) * sms));
  {
    ProfScope ps(BILU_PROF_SYMBOLIC, stream);
    symbolic_kernel<<<grid, kSymWarps * 32, smem, s>>>(n, k, cap, d_arp.as<int32_t>(), d_aci.as<int32_t>(),
                                                       d_ocol.as<int32_t>(), d_olev.as<int32_t>(),
                                                       d_olen.as<int32_t>(), d_done.as<int32_t>(),
                                                       d_header.as<int32_t>(), trisolve_config().spin_ns);
  }
  if (cudaGetLastError() != cudaSuccess) return BILU_ERR_CUDA;
  if (cudaMemcpyAsync(hdr, d_header.p, sizeof(hdr), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BILU_ERR_CUDA;
  if (hdr[kErr]) return hdr[kErr];
  // ---- completion on the device: row pointers, L / U' split, Eq. 4 levels,
  // backfill map, line length -- into the handle's device copy ----
  const long long ntiles = ((long long)n + kScanTile - 1) / kScanTile;
  const int gsm = std::max(1, sms * 8);
  DevBuf d_nl, d_nu, d_flag, d_part, d_stats, d_rp0, d_lrp0, d_urp0, d_idx, d_starts, d_hist;
  if (!d_nl.alloc(sizeof(int32_t) * (size_t)n) || !d_nu.alloc(sizeof(int32_t) * (size_t)n) ||
      !d_flag.alloc(sizeof(int32_t) * (size_t)n) || !d_part.alloc(sizeof(long long) * (size_t)(ntiles + 1)) ||
      !d_stats.alloc(sizeof(int32_t) * kStatWords) || !d_rp0.alloc(sizeof(int32_t) * ((size_t)n + 1)) ||
      !d_lrp0.alloc(sizeof(int32_t) * ((size_t)n + 1)) || !d_urp0.alloc(sizeof(int32_t) * ((size_t)n + 1)) ||
      !d_idx.alloc(sizeof(int32_t) * ((size_t)n + 1)) || !d_starts.alloc(sizeof(int32_t) * (size_t)n) ||
      !d_hist.alloc(sizeof(int32_t) * 4097)) {
    cudaGetLastError();
    return BILU_ERR_OOM;
  }
  cudaMemsetAsync(d_stats.p, 0, sizeof(int32_t) * kStatWords, s);
  cudaMemsetAsync(d_hist.p, 0, sizeof(int32_t) * 4097, s);
  row_info_kernel<<<gsm, 256, 0, s>>>(n, cap, d_ocol.as<int32_t>(), d_olen.as<int32_t>(), d_nl.as<int32_t>(),
                                      d_nu.as<int32_t>(), d_flag.as<int32_t>(), d_stats.as<int32_t>());
  // exclusive scans; the totals are checked against the int32 range
  auto exscan = [&](const int32_t* in, int32_t* outp, long long* total) -> bool {
    scan_tiles_kernel<<<(unsigned)ntiles, kScanTile, 0, s>>>(in, n, outp, d_part.as<long long>());
    scan_parts_kernel<<<1, kScanTile, 0, s>>>(d_part.as<long long>(), ntiles);
    scan_add_kernel<<<(unsigned)(((long long)n + 256) / 256), 256, 0, s>>>(outp, n, d_part.as<long long>(), ntiles);
    return cudaMemcpyAsync(total, d_part.as<long long>() + ntiles, sizeof(long long), cudaMemcpyDeviceToHost, s) ==
               cudaSuccess &&
           cudaStreamSynchronize(s) == cudaSuccess;
  };
  long long nnz_p = 0, nnz_l = 0, nnz_u = 0, nstarts = 0;
  if (!exscan(d_olen.as<int32_t>(), d_rp0.as<int32_t>(), &nnz_p) ||
      !exscan(d_nl.as<int32_t>(), d_lrp0.as<int32_t>(), &nnz_l) ||
      !exscan(d_nu.as<int32_t>(), d_urp0.as<int32_t>(), &nnz_u) ||
      !exscan(d_flag.as<int32_t>(), d_idx.as<int32_t>(), &nstarts))
    return BILU_ERR_CUDA;
  if (nnz_p > (long long)INT32_MAX || nnz_l + n + nnz_u > (long long)INT32_MAX) return BILU_ERR_OOM;
  const long long nslots = nnz_l + n + nnz_u;
  // the handle's device copies: P' and its levels (d_sym), and the layout the
  // factorization and solves read (d_mem)
  const size_t s_rp = align256(sizeof(int32_t) * ((size_t)n + 1));
  const size_t s_ci = align256(sizeof(int32_t) * ((size_t)nnz_p + 1));
  const size_t s_lv = align256(sizeof(int32_t) * (size_t)n);
  const DeviceLayout lay = device_layout(n, nnz_l, nnz_u, nslots);
  void* sym = nullptr;
  void* mem = nullptr;
  if (cudaMalloc(&sym, s_rp + 2 * s_ci + 2 * s_lv) != cudaSuccess) {
    cudaGetLastError();
    return BILU_ERR_OOM;
  }
  if (cudaMalloc(&mem, lay.total) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(sym);
    return BILU_ERR_OOM;
  }
  char* cs = (char*)sym;
  int32_t* d_rp = (int32_t*)cs;
  int32_t* d_ci = (int32_t*)(cs + s_rp);
  int32_t* d_lev = (int32_t*)(cs + s_rp + s_ci);
  int32_t* d_lvl_l = (int32_t*)(cs + s_rp + 2 * s_ci);
  int32_t* d_lvl_u = (int32_t*)(cs + s_rp + 2 * s_ci + s_lv);
  char* cm = (char*)mem;
  int32_t* d_lrp = (int32_t*)cm;
  int32_t* d_lci = (int32_t*)(cm + lay.lrp);
  int32_t* d_urp = (int32_t*)(cm + lay.lrp + lay.lci);
  int32_t* d_uci = (int32_t*)(cm + lay.lrp + lay.lci + lay.urp);
  int32_t* d_slot = (int32_t*)(cm + lay.lrp + lay.lci + lay.urp + lay.uci);
  const size_t rpb = sizeof(int32_t) * ((size_t)n + 1);
  cudaMemcpyAsync(d_rp, d_rp0.p, rpb, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(d_lrp, d_lrp0.p, rpb, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(d_urp, d_urp0.p, rpb, cudaMemcpyDeviceToDevice, s);
  split_kernel<<<gsm, 256, 0, s>>>(n, cap, d_ocol.as<int32_t>(), d_olev.as<int32_t>(), d_rp, d_lrp, d_urp, d_ci,
                                   d_lev, d_lci, d_uci);
  cudaMemsetAsync(d_slot, 0xFF, sizeof(int32_t) * (size_t)nslots, s);
  slot_map_kernel<<<gsm, 256, 0, s>>>(n, d_arp.as<int32_t>(), d_aci.as<int32_t>(), d_rp, d_ci, d_lrp, d_urp, nnz_l,
                                      d_slot);
  // Eq. 4, lower then upper: persistent grids, one warp per claimed row
  int lv_per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lv_per_sm, eq4_level_kernel<false>, 256, 0);
  const int lgrid = std::max(1, std::min<int>((n + 7) / 8, std::max(lv_per_sm, 1) * sms));
  cudaMemsetAsync(d_done.p, 0, sizeof(int32_t) * (size_t)n, s);
  eq4_level_kernel<false><<<lgrid, 256, 0, s>>>(n, d_lrp, d_lci, d_done.as<int32_t>(), d_lvl_l,
                                                 d_header.as<int32_t>(), d_stats.as<int32_t>(),
                                                 trisolve_config().spin_ns);
  cudaMemsetAsync(d_done.p, 0, sizeof(int32_t) * (size_t)n, s);
  eq4_level_kernel<true><<<lgrid, 256, 0, s>>>(n, d_urp, d_uci, d_done.as<int32_t>(), d_lvl_u,
                                                d_header.as<int32_t>(), d_stats.as<int32_t>(),
                                                trisolve_config().spin_ns);
  // line length
  line_starts_kernel<<<gsm, 256, 0, s>>>(n, d_flag.as<int32_t>(), d_idx.as<int32_t>(), d_starts.as<int32_t>());
  line_hist_kernel<<<gsm, 256, 0, s>>>((int32_t)nstarts, d_starts.as<int32_t>(), d_hist.as<int32_t>());
  int32_t stats[kStatWords] = {};
  std::vector<int32_t> hist(4097, 0);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(stats, d_stats.p, sizeof(stats), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hist.data(), d_hist.p, sizeof(int32_t) * 4097, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hdr, d_header.p, sizeof(hdr), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaFree(sym);
    cudaFree(mem);
    return BILU_ERR_CUDA;
  }
  if (hdr[kErr]) {
    cudaFree(sym);
    cudaFree(mem);
    return hdr[kErr];
  }
  bilu_pattern* p = new (std::nothrow) bilu_pattern();
  if (!p) {
    cudaFree(sym);
    cudaFree(mem);
    return BILU_ERR_OOM;
  }
  p->n = n;
  p->k = k;
  p->nnz_a = nnz_a;
  p->cnt_p = nnz_p;
  p->cnt_l = nnz_l;
  p->cnt_u = nnz_u;
  p->max_l = stats[kMaxL];
  p->max_u = stats[kMaxU];
  p->nlev_l = stats[kNlevL];
  p->nlev_u = stats[kNlevU];
  int32_t best = 0;  // the rule of the host phase: the most common distance that recurs
  for (int32_t d = 2; d <= 4096; ++d)
    if (hist[(size_t)d] > hist[(size_t)best] && hist[(size_t)d] >= 2) best = d;
  p->line_len = best;
  p->host_ready = false;
  p->device = dev;
  p->d_sym = sym;
  p->d_rp = d_rp;
  p->d_ci = d_ci;
  p->d_lev = d_lev;
  p->d_lvl_l = d_lvl_l;
  p->d_lvl_u = d_lvl_u;
  p->d_mem = mem;
  p->d_lrp = d_lrp;
  p->d_lci = d_lci;
  p->d_urp = d_urp;
  p->d_uci = d_uci;
  p->d_slot_src = d_slot;
  *out = p;
  return BILU_OK;
}
