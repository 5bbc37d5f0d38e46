// schedule_gpu.cu -- the sync-free schedules (chunk cuts, the rows of each
// chunk by local Eq. 4 level, the chunk claim order) for a pattern completed
// on the device by bilu_symbolic_gpu, with every pass over P' run on the
// device.  The result is the schedule build_schedule (symbolic.cpp) builds on
// the host, bit for bit: the host keeps only the steps whose work grows with
// the number of rows or chunks -- the greedy chunk cuts over the per-row gaps
// and the list scheduling over the chunk graph -- and runs them through the
// same functions (schedule_cuts, ticket_order_lists).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cub/cub.cuh>
#include <new>
#include <vector>

#include "device_common.cuh"

namespace bilu {
namespace {

// Most rows of one chunk (schedule_cuts never makes a longer one).
constexpr int kMaxChunkRows = 1024;
constexpr int kOrderWarps = 4;

// gapl[r] = r - (last column of L(r)), gapu[r] = (first column of U'(r-1)) -
// (r-1); INT32_MAX where there is no such column.
__global__ void gap_kernel(int32_t n, const int32_t* __restrict__ lrp, const int32_t* __restrict__ lci,
                           const int32_t* __restrict__ urp, const int32_t* __restrict__ uci,
                           int32_t* __restrict__ gapl, int32_t* __restrict__ gapu) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    const int le = lrp[r + 1];
    gapl[r] = le > lrp[r] ? (int)r - lci[le - 1] : INT_MAX;
    gapu[r] = (r > 0 && urp[r] > urp[r - 1]) ? uci[urp[r - 1]] - (int)(r - 1) : INT_MAX;
  }
}

// The rows of every chunk listed by local level (Eq. 4 restricted to the
// chunk: 1 + the largest local level of the chunk's rows it depends on, 0 if
// none), ties by ascending row for L and by descending row for U'.  One warp
// per chunk: the levels in solve order (lanes share a row's dependencies, a
// warp maximum combines them), then a counting sort by level placed in tie
// order by one lane.
template <bool UPPER>
__global__ void __launch_bounds__(kOrderWarps * 32) chunk_order_kernel(int32_t nchunks,
                                                                        const int32_t* __restrict__ bnd,
                                                                        const int32_t* __restrict__ rpv,
                                                                        const int32_t* __restrict__ civ,
                                                                        int32_t* __restrict__ ord) {
  __shared__ int s_loc[kOrderWarps][kMaxChunkRows];
  __shared__ int s_cnt[kOrderWarps][kMaxChunkRows + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int* loc = s_loc[w];
  int* cnt = s_cnt[w];
  const long long nw = (long long)gridDim.x * kOrderWarps;
  for (long long c = (long long)blockIdx.x * kOrderWarps + w; c < nchunks; c += nw) {
    const int lo = bnd[c], hi = bnd[c + 1], len = hi - lo;
    for (int x = lane; x <= len; x += 32) cnt[x] = 0;
    for (int q = 0; q < len; ++q) {
      const int i = UPPER ? hi - 1 - q : lo + q;
      int l = 0;
      for (int t = rpv[i] + lane; t < rpv[i + 1]; t += 32) {
        const int j = civ[t];
        if (j >= lo && j < hi) l = max(l, loc[j - lo] + 1);
      }
      l = __reduce_max_sync(kFull, l);
      if (lane == 0) loc[i - lo] = l;
      __syncwarp();
    }
    for (int x = lane; x < len; x += 32) atomicAdd(&cnt[loc[x] + 1], 1);
    __syncwarp();
    if (lane == 0) {
      for (int x = 1; x <= len; ++x) cnt[x] += cnt[x - 1];  // cnt[l] = first position of level l
      for (int q = 0; q < len; ++q) {
        const int i = UPPER ? hi - 1 - q : lo + q;
        ord[lo + cnt[loc[i - lo]]++] = i;
      }
    }
    __syncwarp();
  }
}

// Chunk number c of a solve (lower: chunk c; upper: chunk nchunks-1-c) of row j.
__device__ __forceinline__ int chunk_of_row(const int32_t* bnd, int nchunks, int j) {
  int lo = 0, hi = nchunks;  // the last chunk whose first row is <= j
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (bnd[mid] <= j) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Per chunk (solve numbering): the smallest Eq. 4 level of its rows (the
// claim priority), and -- in pass 0 the count, in pass 1 the values -- the
// solve numbers of the chunks its rows depend on, one entry per run of equal
// chunks along a row's sorted columns (duplicates across rows are removed
// later).  One warp per chunk.
template <bool UPPER>
__global__ void chunk_edges_kernel(int32_t nchunks, const int32_t* __restrict__ bnd,
                                   const int32_t* __restrict__ rpv, const int32_t* __restrict__ civ,
                                   const int32_t* __restrict__ lvl, int pass, int32_t* __restrict__ prio,
                                   int64_t* __restrict__ count, const int64_t* __restrict__ off,
                                   int32_t* __restrict__ edges) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += nw) {
    const int lc = UPPER ? nchunks - 1 - (int)c : (int)c;
    const int lo = bnd[lc], hi = bnd[lc + 1];
    int pm = INT_MAX;
    long long k = 0;
    for (int i = lo; i < hi; ++i) {
      if (lane == 0) pm = min(pm, lvl[i]);
      int prev = -1;  // the chunk of the row's previous entry (-1: none, or inside the chunk)
      for (int t0 = rpv[i]; t0 < rpv[i + 1]; t0 += 32) {
        const int t = t0 + lane;
        int cj = -1;
        if (t < rpv[i + 1]) {
          const int j = civ[t];
          if (j < lo || j >= hi) {
            const int lj = chunk_of_row(bnd, nchunks, j);
            cj = UPPER ? nchunks - 1 - lj : lj;
          }
        }
        // skip an entry whose predecessor in the row falls in the same chunk
        int before = __shfl_up_sync(kFull, cj, 1);
        if (lane == 0) before = prev;
        const bool keep = cj >= 0 && cj != before;
        const unsigned m = __ballot_sync(kFull, keep);
        if (pass == 1 && keep) edges[off[c] + k + __popc(m & ((1u << lane) - 1u))] = cj;
        k += __popc(m);
        prev = __shfl_sync(kFull, cj, 31);
      }
    }
    pm = __reduce_min_sync(kFull, lane == 0 ? pm : INT_MAX);
    if (lane == 0) {
      if (pass == 0) {
        count[c] = k;
        prio[c] = pm;
      }
    }
  }
}

// Each chunk's sorted predecessor list with duplicates removed: ucount[c]
// distinct entries written from uniq[off[c]].  One warp per chunk.
__global__ void unique_kernel(int32_t nchunks, const int64_t* __restrict__ off, const int32_t* __restrict__ sorted,
                              int32_t* __restrict__ uniq, int64_t* __restrict__ ucount) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += nw) {
    const long long b = off[c], e = off[c + 1];
    long long k = 0;
    for (long long t0 = b; t0 < e; t0 += 32) {
      const long long t = t0 + lane;
      const bool keep = t < e && (t == b || sorted[t] != sorted[t - 1]);
      const unsigned m = __ballot_sync(kFull, keep);
      if (keep) uniq[b + k + __popc(m & ((1u << lane) - 1u))] = sorted[t];
      k += __popc(m);
    }
    if (lane == 0) ucount[c] = k;
  }
}

}  // namespace

namespace {

// Copies of each chunk's distinct predecessors packed back to back.
__global__ void pack_kernel(int32_t nchunks, const int64_t* __restrict__ off, const int64_t* __restrict__ ucount,
                            const int64_t* __restrict__ uoff, const int32_t* __restrict__ uniq,
                            int32_t* __restrict__ packed) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += nw)
    for (long long t = lane; t < ucount[c]; t += 32) packed[uoff[c] + t] = uniq[off[c] + t];
}

// Device scratch freed on every return path.
struct Scratch {
  std::vector<void*> bufs;
  ~Scratch() {
    for (void* b : bufs) cudaFree(b);
  }
  template <typename T>
  T* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 16)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    bufs.push_back(p);
    return reinterpret_cast<T*>(p);
  }
};

int device_sms() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, sms);
}

// Claim order of one triangle: priorities and distinct predecessor lists on
// the device, list scheduling on the host (work per chunk, not per entry).
template <bool UPPER>
int ticket_order_device(const bilu_pattern* p, const bilu_chunk_schedule* s, const int32_t* d_bnd,
                        std::vector<int32_t>& tick) {
  const int32_t nchunks = s->nchunks;
  const int32_t* rpv = UPPER ? p->d_urp : p->d_lrp;
  const int32_t* civ = UPPER ? p->d_uci : p->d_lci;
  const int32_t* lvl = UPPER ? p->d_lvl_u : p->d_lvl_l;
  const int grid = device_sms() * 8;
  Scratch sc;
  int32_t* d_prio = sc.get<int32_t>((size_t)nchunks);
  int64_t* d_count = sc.get<int64_t>((size_t)nchunks + 1);
  int64_t* d_off = sc.get<int64_t>((size_t)nchunks + 1);
  int64_t* d_ucount = sc.get<int64_t>((size_t)nchunks + 1);
  int64_t* d_uoff = sc.get<int64_t>((size_t)nchunks + 1);
  if (!d_prio || !d_count || !d_off || !d_ucount || !d_uoff) return BILU_ERR_OOM;
  cudaMemset(d_count, 0, sizeof(int64_t) * ((size_t)nchunks + 1));
  cudaMemset(d_ucount, 0, sizeof(int64_t) * ((size_t)nchunks + 1));
  chunk_edges_kernel<UPPER><<<grid, 256>>>(nchunks, d_bnd, rpv, civ, lvl, 0, d_prio, d_count, nullptr, nullptr);
  size_t tb = 0, tb2 = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tb, d_count, d_off, nchunks + 1);
  void* d_tmp = sc.get<unsigned char>(tb);
  if (!d_tmp) return BILU_ERR_OOM;
  cub::DeviceScan::ExclusiveSum(d_tmp, tb, d_count, d_off, nchunks + 1);
  int64_t total = 0;
  if (cudaMemcpy(&total, d_off + nchunks, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return BILU_ERR_CUDA;
  int32_t* d_edges = sc.get<int32_t>((size_t)total);
  int32_t* d_sorted = sc.get<int32_t>((size_t)total);
  int32_t* d_uniq = sc.get<int32_t>((size_t)total);
  if (!d_edges || !d_sorted || !d_uniq) return BILU_ERR_OOM;
  chunk_edges_kernel<UPPER><<<grid, 256>>>(nchunks, d_bnd, rpv, civ, lvl, 1, d_prio, d_count, d_off, d_edges);
  if (total > 0) {
    cub::DeviceSegmentedSort::SortKeys(nullptr, tb2, d_edges, d_sorted, total, nchunks, d_off, d_off + 1);
    void* d_tmp2 = sc.get<unsigned char>(tb2);
    if (!d_tmp2) return BILU_ERR_OOM;
    cub::DeviceSegmentedSort::SortKeys(d_tmp2, tb2, d_edges, d_sorted, total, nchunks, d_off, d_off + 1);
  }
  unique_kernel<<<grid, 256>>>(nchunks, d_off, d_sorted, d_uniq, d_ucount);
  cub::DeviceScan::ExclusiveSum(d_tmp, tb, d_ucount, d_uoff, nchunks + 1);
  int64_t utotal = 0;
  if (cudaMemcpy(&utotal, d_uoff + nchunks, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return BILU_ERR_CUDA;
  int32_t* d_packed = sc.get<int32_t>((size_t)utotal);
  if (!d_packed) return BILU_ERR_OOM;
  pack_kernel<<<grid, 256>>>(nchunks, d_off, d_ucount, d_uoff, d_uniq, d_packed);
  std::vector<int32_t> prio((size_t)nchunks), pred((size_t)utotal);
  std::vector<int64_t> pred_ptr((size_t)nchunks + 1);
  if (cudaMemcpy(prio.data(), d_prio, sizeof(int32_t) * (size_t)nchunks, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(pred_ptr.data(), d_uoff, sizeof(int64_t) * ((size_t)nchunks + 1), cudaMemcpyDeviceToHost) !=
          cudaSuccess ||
      (utotal > 0 &&
       cudaMemcpy(pred.data(), d_packed, sizeof(int32_t) * (size_t)utotal, cudaMemcpyDeviceToHost) != cudaSuccess))
    return BILU_ERR_CUDA;
  ticket_order_lists(nchunks, prio, pred_ptr, pred, tick);
  return BILU_OK;
}

}  // namespace

int build_schedule_device(const bilu_pattern* p, int32_t target, bool upper, bilu_chunk_schedule* s) {
  const int32_t n = p->n;
  s->chunk = target;
  s->upper = upper;
  if (n == 0) {
    s->bnd.assign(1, 0);
    s->nchunks = 0;
    s->max_len = 0;
    return BILU_OK;
  }
  try {
    std::vector<int32_t> gapl((size_t)n), gapu((size_t)n);
    {
      Scratch sc;
      int32_t* d_gl = sc.get<int32_t>((size_t)n);
      int32_t* d_gu = sc.get<int32_t>((size_t)n);
      if (!d_gl || !d_gu) return BILU_ERR_OOM;
      gap_kernel<<<device_sms() * 8, 256>>>(n, p->d_lrp, p->d_lci, p->d_urp, p->d_uci, d_gl, d_gu);
      if (cudaMemcpy(gapl.data(), d_gl, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(gapu.data(), d_gu, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return BILU_ERR_CUDA;
    }
    schedule_cuts(n, target, upper, gapl, gapu, s);
    if (s->max_len > kMaxChunkRows) return BILU_ERR_ARG;
    const int32_t nchunks = s->nchunks;
    const size_t one = align256(sizeof(int32_t) * (size_t)n);
    const size_t tk = align256(sizeof(int32_t) * (size_t)nchunks);
    const size_t bd = align256(sizeof(int32_t) * ((size_t)nchunks + 1));
    const int parts = upper ? 2 : 1;
    void* mem = nullptr;
    if (cudaMalloc(&mem, bd + parts * (one + tk)) != cudaSuccess) {
      cudaGetLastError();
      return BILU_ERR_OOM;
    }
    char* m = (char*)mem;
    s->d_mem = mem;
    s->d_bnd = (int32_t*)m;
    s->d_ord_l = (int32_t*)(m + bd);
    s->d_tick_l = (int32_t*)(m + bd + one);
    if (upper) {
      s->d_ord_u = (int32_t*)(m + bd + one + tk);
      s->d_tick_u = (int32_t*)(m + bd + 2 * one + tk);
    }
    cudaMemcpy(s->d_bnd, s->bnd.data(), sizeof(int32_t) * s->bnd.size(), cudaMemcpyHostToDevice);
    const int ogrid = std::max(1, std::min((nchunks + kOrderWarps - 1) / kOrderWarps, device_sms() * 8));
    chunk_order_kernel<false><<<ogrid, kOrderWarps * 32>>>(nchunks, s->d_bnd, p->d_lrp, p->d_lci, s->d_ord_l);
    if (upper)
      chunk_order_kernel<true><<<ogrid, kOrderWarps * 32>>>(nchunks, s->d_bnd, p->d_urp, p->d_uci, s->d_ord_u);
    int st = ticket_order_device<false>(p, s, s->d_bnd, s->tick_l);
    if (st == BILU_OK && upper) st = ticket_order_device<true>(p, s, s->d_bnd, s->tick_u);
    if (st == BILU_OK) {
      cudaMemcpy(s->d_tick_l, s->tick_l.data(), sizeof(int32_t) * (size_t)nchunks, cudaMemcpyHostToDevice);
      if (upper)
        cudaMemcpy(s->d_tick_u, s->tick_u.data(), sizeof(int32_t) * (size_t)nchunks, cudaMemcpyHostToDevice);
      if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) st = BILU_ERR_CUDA;
    }
    if (st != BILU_OK) {
      cudaFree(mem);
      s->d_mem = nullptr;
      return st;
    }
  } catch (const std::bad_alloc&) {
    return BILU_ERR_OOM;
  }
  return BILU_OK;
}

}  // namespace bilu
