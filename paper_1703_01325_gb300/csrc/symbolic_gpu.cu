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

// ci[rp[i] + t] = ocol[i * cap + t] (and levels), one warp per row.
__global__ void compact_kernel(int32_t n, int32_t cap, const int32_t* __restrict__ rp,
                               const int32_t* __restrict__ ocol, const int32_t* __restrict__ olev,
                               int32_t* __restrict__ ci, int32_t* __restrict__ lev) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
    const int beg = rp[i], len = rp[i + 1] - beg;
    for (int t = lane; t < len; t += 32) {
      ci[beg + t] = ocol[(size_t)i * cap + t];
      lev[beg + t] = olev[(size_t)i * cap + t];
    }
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
  bilu_pattern* p = new (std::nothrow) bilu_pattern();
  if (!p) return BILU_ERR_OOM;
  try {
    std::vector<int32_t> len((size_t)n);
    if (cudaMemcpy(len.data(), d_olen.p, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess) {
      delete p;
      return BILU_ERR_CUDA;
    }
    p->n = n;
    p->k = k;
    p->nnz_a = nnz_a;
    p->rp.assign((size_t)n + 1, 0);
    int64_t tot = 0;
    for (int32_t i = 0; i < n; ++i) {
      tot += len[i];
      if (tot > (int64_t)INT32_MAX) {
        delete p;
        return BILU_ERR_OOM;
      }
      p->rp[(size_t)i + 1] = (int32_t)tot;
    }
    p->ci.resize((size_t)tot);
    p->lev.resize((size_t)tot);
    DevBuf d_rp, d_ci, d_lev;
    if (!d_rp.alloc(sizeof(int32_t) * ((size_t)n + 1)) || !d_ci.alloc(sizeof(int32_t) * (size_t)tot) ||
        !d_lev.alloc(sizeof(int32_t) * (size_t)tot)) {
      cudaGetLastError();
      delete p;
      return BILU_ERR_OOM;
    }
    cudaMemcpyAsync(d_rp.p, p->rp.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s);
    compact_kernel<<<std::max(1, std::min((n + 7) / 8, sms * 16)), 256, 0, s>>>(
        n, cap, d_rp.as<int32_t>(), d_ocol.as<int32_t>(), d_olev.as<int32_t>(), d_ci.as<int32_t>(),
        d_lev.as<int32_t>());
    if (cudaMemcpyAsync(p->ci.data(), d_ci.p, sizeof(int32_t) * (size_t)tot, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(p->lev.data(), d_lev.p, sizeof(int32_t) * (size_t)tot, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      delete p;
      return BILU_ERR_CUDA;
    }
    if (complete_pattern(p, row_ptr, col_idx) != BILU_OK) {
      delete p;
      return BILU_ERR_OOM;
    }
  } catch (const std::bad_alloc&) {
    delete p;
    return BILU_ERR_OOM;
  }
  *out = p;
  return BILU_OK;
}
