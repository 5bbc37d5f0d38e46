// factor.cu -- numeric block factorization A' = L D U' on the pattern P'.
//
// 1. Backfill (Algorithm 5 steps 3-4): every slot of the factor buffer
//    [L | D | U] gathers its A block, or zero for a fill position.
// 2. Block ILU(0) on A' (Algorithm 4), one warp per block row, rows claimed in
//    ascending order through an atomic ticket.  Row i walks its pivots p < i
//    in ascending order; for each it waits (bounded, acquire) until row p is
//    finished, then
//        A_ip <- A_ip D_p^{-1}
//        A_ij <- A_ij - A_ip U_pj   for every j > p with (p,j) and (i,j) in P'
//    where U_pj is row p's final, still unscaled upper block.  The j updates of
//    one pivot are independent, so the warp spreads (block, element) pairs
//    over its lanes; each element is a b-term dot product.
//    Then D_i = A_ii is inverted in the warp (Gauss-Jordan with partial
//    pivoting inside the b x b block, one lane per column of [D_i | I]),
//    D_i^{-1} overwrites the D slot, and row i is released (fence + release
//    store of its ready flag).  Row i depends only on rows of smaller tickets,
//    which are held by running warps, so the schedule always progresses.
// 3. Eq. 5: U'_ij = D_i^{-1} U_ij for every upper block, once all rows are
//    done (later rows need the unscaled U_pj).
// A zero or non-finite pivot block records BILU_ERR_SINGULAR and the smallest
// such row; the row is still released so that no warp waits forever.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"

namespace bilu {
namespace {


template <typename TV>
__global__ void backfill_kernel(long long total, int bb, const int32_t* __restrict__ slot_src,
                                const double* __restrict__ a, TV* __restrict__ f) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const long long slot = q / bb;
    const int e = (int)(q - slot * bb);
    const int32_t src = __ldg(slot_src + slot);
    f[q] = src >= 0 ? (TV)__ldg(a + (size_t)src * bb + e) : TV(0);
  }
}

__global__ void factor_init_kernel(int32_t* header, int32_t* done, int32_t n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) done[q] = 0;
  if (blockIdx.x == 0 && threadIdx.x < kHeaderWords)
    header[threadIdx.x] = (threadIdx.x == kBadRow) ? 0x7fffffff : 0;
}

// Row storage of the factor kernel: up to RC blocks of a row are staged in
// shared memory (per warp); longer rows are worked on in place in global
// memory through the same slot interface.  8 warps per CTA: two CTAs fit on
// an SM for b <= 5 (registers), twice the chunks in flight of one 16-warp CTA
// for the same warps (measured 4-13 % faster with 256-row chunk targets).
template <int B>
struct FactorCap {
  static constexpr int W = 8;                          // warps per CTA
  static constexpr int RC = B <= 4 ? 64 : (B <= 6 ? 32 : 24);
  static constexpr int WDBL = RC * B * B + 4 * B * B;  // doubles per warp
  static constexpr int WINT = RC + 32;                 // ints per warp
};

template <int B, typename TV>
size_t factor_smem_bytes(int chunk) {
  return (size_t)FactorCap<B>::W * FactorCap<B>::WDBL * sizeof(TV) +
         ((size_t)2 * chunk + (size_t)FactorCap<B>::W * FactorCap<B>::WINT) * sizeof(int);
}

template <int B, typename TV>
__global__ void __launch_bounds__(FactorCap<B>::W * 32) factor_kernel(
    int32_t n, int32_t chunk, int32_t nchunks, const int32_t* __restrict__ bnd, const int32_t* __restrict__ ord,
    const int32_t* __restrict__ tick,
    const int32_t* __restrict__ lrp, const int32_t* __restrict__ lci,
    const int32_t* __restrict__ urp, const int32_t* __restrict__ uci, TV* f, long long nnz_l,
    int32_t* header, int32_t* done, long long spin_ns) {
  constexpr int BB = B * B;
  constexpr int H = (BB + 31) / 32;
  constexpr int RC = FactorCap<B>::RC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  TV* wd = reinterpret_cast<TV*>(smem_raw) + (size_t)warp * FactorCap<B>::WDBL;
  TV* rowv = wd;             // RC blocks of the row being factored
  TV* dp = rowv + RC * BB;   // D_p^{-1}
  TV* aip = dp + BB;         // scaled A_ip
  TV* aug = aip + BB;        // [D_i | I] for Gauss-Jordan
  int* ib = reinterpret_cast<int*>(reinterpret_cast<TV*>(smem_raw) + (size_t)FactorCap<B>::W * FactorCap<B>::WDBL);
  int* fl = ib;                  // chunk-local ready flags (value = chunk id)
  int* s_i = fl + chunk;         // rows of the chunk in local-level order
  int* cols = s_i + chunk + warp * FactorCap<B>::WINT;  // column of each staged slot
  int* dstv = cols + RC;         // destination slot per U_p entry of a batch
  __shared__ int s_c;
  TV* L = f;
  TV* D = f + (size_t)nnz_l * BB;
  TV* U = D + (size_t)n * BB;
  for (int q = tid; q < chunk; q += blockDim.x) fl[q] = -1;
  Waiter w{header, spin_ns, 0, nullptr};
  bool dead = false;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      int cc = atomicAdd(header + kTicketF, 1);
      if (ld_volatile_s32(header + kAbort)) cc = nchunks;
      s_c = cc < nchunks ? tick[cc] : nchunks;
    }
    __syncthreads();
    const int c = s_c;
    if (c >= nchunks) return;
    const int lo = bnd[c], hi = bnd[c + 1];  // at most `chunk` rows
    const int len = hi - lo;
    for (int q = tid; q < len; q += blockDim.x) s_i[q] = ord[lo + q];
    __syncthreads();
    for (int pos = warp; pos < len && !dead; pos += FactorCap<B>::W) {
      const int i = s_i[pos];
      const int lb = lrp[i], nl = lrp[i + 1] - lb;
      const int ub = urp[i], nu = urp[i + 1] - ub;
      const int nrow = nl + 1 + nu;
      const bool staged = nrow <= RC;
      // slot k of row i: L blocks (k < nl), the pivot block (k == nl), U blocks
      auto blk = [&](int k) -> TV* {
        if (staged) return rowv + k * BB;
        if (k < nl) return L + (size_t)(lb + k) * BB;
        if (k == nl) return D + (size_t)i * BB;
        return U + (size_t)(ub + k - nl - 1) * BB;
      };
      auto colk = [&](int k) -> int {
        if (staged) return cols[k];
        if (k < nl) return lci[lb + k];
        if (k == nl) return i;
        return uci[ub + k - nl - 1];
      };
      if (staged) {
        for (int k = lane; k < nrow; k += 32)
          cols[k] = k < nl ? lci[lb + k] : (k == nl ? i : uci[ub + k - nl - 1]);
        for (int q = lane; q < nl * BB; q += 32) rowv[q] = L[(size_t)lb * BB + q];
        for (int q = lane; q < BB; q += 32) rowv[nl * BB + q] = D[(size_t)i * BB + q];
        for (int q = lane; q < nu * BB; q += 32) rowv[(nl + 1) * BB + q] = U[(size_t)ub * BB + q];
      }
      __syncwarp();
      for (int k = 0; k < nl; ++k) {
        const int p = colk(k);
        const int pb = urp[p], pe = urp[p + 1];
        // destination slots of the first batch of row p's U entries (pattern
        // only: done before waiting for row p)
        auto find_dst = [&](int s0) {
          const int cnt = min(32, pe - s0);
          if (lane < cnt) {
            const int j = uci[s0 + lane];
            int a = k + 1, z = nrow, d = -1;
            while (a < z) {
              const int mid = (a + z) >> 1;
              const int v = colk(mid);
              if (v == j) { d = mid; break; }
              if (v < j) a = mid + 1; else z = mid;
            }
            dstv[lane] = d;
          }
        };
        find_dst(pb);
        const bool ok = (p >= lo && p < hi) ? wait_local_flag(fl + (p - lo), c, w) : wait_flag(done + p, w);
        if (__any_sync(kFull, !ok)) {
          dead = true;
          break;
        }
        // A_ip <- A_ip * D_p^{-1}; D_p^{-1} and this lane's first U_pj
        // operands are fetched together (one memory round trip per pivot)
        for (int e = lane; e < BB; e += 32) dp[e] = D[(size_t)p * BB + e];
        constexpr int NPRE = 4;
        TV upre[NPRE][B];
        {
          const int cnt0 = min(32, pe - pb);
#pragma unroll
          for (int h = 0; h < NPRE; ++h) {
            const int wk = lane + 32 * h;
            if (wk < cnt0 * BB) {
              const int sidx = wk / BB, e = wk - (wk / BB) * BB;
              const TV* upj = U + (size_t)(pb + sidx) * BB + (e / B) * B;
#pragma unroll
              for (int m = 0; m < B; ++m) upre[h][m] = upj[m];
            }
          }
        }
        __syncwarp();
        TV* a = blk(k);
        TV nv[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
          const int e = lane + 32 * h;
          if (e < BB) {
            const int r = e % B, cc = e / B;
            TV s = TV(0);
#pragma unroll
            for (int m = 0; m < B; ++m) s = fma(a[m * B + r], dp[cc * B + m], s);
            nv[h] = s;
          }
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < H; ++h) {
          const int e = lane + 32 * h;
          if (e < BB) {
            a[e] = nv[h];
            aip[e] = nv[h];
          }
        }
        __syncwarp();
        // A_ij <- A_ij - A_ip U_pj for j > p in both P'(p) and P'(i)
        for (int s0 = pb; s0 < pe; s0 += 32) {
          if (s0 != pb) {
            find_dst(s0);
            __syncwarp();
          }
          const int cnt = min(32, pe - s0);
          if (s0 == pb) {
#pragma unroll
            for (int h = 0; h < NPRE; ++h) {
              const int wk = lane + 32 * h;
              if (wk < cnt * BB) {
                const int sidx = wk / BB, e = wk - (wk / BB) * BB;
                const int d = dstv[sidx];
                if (d >= 0) {
                  const int r = e % B;
                  TV s = TV(0);
#pragma unroll
                  for (int m = 0; m < B; ++m) s = fma(aip[m * B + r], upre[h][m], s);
                  blk(d)[e] -= s;
                }
              }
            }
          }
          for (int wk = lane + (s0 == pb ? 32 * NPRE : 0); wk < cnt * BB; wk += 32) {
            const int sidx = wk / BB;
            const int e = wk - sidx * BB;
            const int d = dstv[sidx];
            if (d >= 0) {
              const int r = e % B, cc = e / B;
              const TV* upj = U + (size_t)(s0 + sidx) * BB + cc * B;
              TV s = TV(0);
#pragma unroll
              for (int m = 0; m < B; ++m) s = fma(aip[m * B + r], upj[m], s);
              blk(d)[e] -= s;
            }
          }
          __syncwarp();
        }
      }
      if (dead) break;
      // D_i^{-1} by Gauss-Jordan with partial pivoting on [D_i | I].
      {
        const TV* di = blk(nl);
        for (int e = lane; e < 2 * BB; e += 32) {
          const int q = e / B, r = e % B;
          aug[e] = q < B ? di[e] : (r == q - B ? TV(1) : TV(0));
        }
      }
      __syncwarp();
      bool bad = false;
      for (int e = lane; e < BB; e += 32) bad |= !isfinite(aug[e]);
      bad = __any_sync(kFull, bad);
      for (int cc = 0; cc < B && !bad; ++cc) {
        int pr = cc;
        TV best = fabs(aug[cc * B + cc]);
#pragma unroll
        for (int r = cc + 1; r < B; ++r) {
          const TV v = fabs(aug[cc * B + r]);
          if (v > best) { best = v; pr = r; }
        }
        if (!(best > TV(0))) { bad = true; break; }
        const TV piv = aug[cc * B + pr];
        __syncwarp();
        if (lane < 2 * B) {
          TV* col = aug + lane * B;
          if (pr != cc) { const TV tmp = col[cc]; col[cc] = col[pr]; col[pr] = tmp; }
          col[cc] = col[cc] / piv;
        }
        __syncwarp();
        TV fr[B];
#pragma unroll
        for (int r = 0; r < B; ++r) fr[r] = aug[cc * B + r];
        __syncwarp();
        if (lane < 2 * B) {
          TV* col = aug + lane * B;
          const TV pc = col[cc];
#pragma unroll
          for (int r = 0; r < B; ++r)
            if (r != cc && fr[r] != TV(0)) col[r] = fma(-fr[r], pc, col[r]);
        }
        __syncwarp();
      }
      if (!bad) {
        for (int e = lane; e < BB; e += 32) bad |= !isfinite(aug[BB + e]);
        bad = __any_sync(kFull, bad);
      }
      // write the finished row back: L blocks, D_i^{-1}, unscaled U blocks
      for (int e = lane; e < BB; e += 32) D[(size_t)i * BB + e] = aug[BB + e];
      if (staged) {
        for (int q = lane; q < nl * BB; q += 32) L[(size_t)lb * BB + q] = rowv[q];
        for (int q = lane; q < nu * BB; q += 32) U[(size_t)ub * BB + q] = rowv[(nl + 1) * BB + q];
      }
      if (bad && lane == 0) {
        atomicMin(header + kBadRow, i);
        atomicCAS(header + kErr, 0, (int)BILU_ERR_SINGULAR);
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) {
        st_release_cta_shared_s32(fl + (i - lo), c);
        st_release_s32(done + i, 1);
      }
    }
  }
}

// Eq. 5: U'_ij = D_i^{-1} U_ij, one warp per block row; lane q of the row's
// (block, column) pairs reads one column of U_ij, forms that column of
// D_i^{-1} U_ij (b x b FMAs) and writes it back in place.  Columns are
// independent, so no lane waits on another.
template <int B, typename TV>
__global__ void __launch_bounds__(256) scale_upper_kernel(int32_t n, const int32_t* __restrict__ urp,
                                                          const TV* __restrict__ dinv,
                                                          TV* __restrict__ u) {
  constexpr int BB = B * B;
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
    const int ub = urp[i], cnt = (urp[i + 1] - ub) * B;
    if (cnt == 0) continue;
    TV d[BB];  // D_i^{-1}, column-major
#pragma unroll
    for (int e = 0; e < BB; ++e) d[e] = __ldg(dinv + (size_t)i * BB + e);
    for (int q = lane; q < cnt; q += 32) {
      TV* col = u + ((size_t)ub + q / B) * BB + (q % B) * B;
      TV x[B];
#pragma unroll
      for (int m = 0; m < B; ++m) x[m] = col[m];
#pragma unroll
      for (int r = 0; r < B; ++r) {
        TV acc = TV(0);
#pragma unroll
        for (int m = 0; m < B; ++m) acc = fma(d[m * B + r], x[m], acc);
        col[r] = acc;
      }
    }
  }
}

int device_sms() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <typename TV>
int launch_backfill_t(const bilu_pattern* p, int32_t b, const double* a_vals, TV* f, void* stream) {
  const long long total = p->nslots() * (long long)b * b;
  if (total == 0) return 0;
  const int blocks = (int)std::min<long long>((total + 255) / 256, (long long)device_sms() * 16);
  ProfScope ps(BILU_PROF_BACKFILL, stream);
  backfill_kernel<TV><<<blocks, 256, 0, (cudaStream_t)stream>>>(total, b * b, p->d_slot_src, a_vals, f);
  return (int)cudaGetLastError();
}

template <typename TV>
int launch_factor_t(const bilu_pattern* p, int32_t b, TV* f, int32_t* header, int32_t* done,
                    void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t n = p->n;
  const int sms = device_sms();
  {
    ProfScope ps0(BILU_PROF_FACTOR_INIT, stream);
    factor_init_kernel<<<std::max(1, std::min((n + 255) / 256, sms * 4)), 256, 0, s>>>(header, done, n);
  }
  if (n == 0) return (int)cudaGetLastError();
  if (p->fact.chunk <= 0 || !p->fact.d_mem) return (int)cudaErrorInvalidValue;
  const int chunk = p->fact.max_len;  // shared-memory rows per CTA
  const int nchunks = p->fact.nchunks;
  const long long spin = trisolve_config().spin_ns;
  BILU_DISPATCH_B(b, {
    const size_t smem = factor_smem_bytes<B, TV>(chunk);
    static int last_chunk = -1, per_sm = 1;
    if (last_chunk != chunk) {
      cudaFuncSetAttribute(factor_kernel<B, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)std::max<size_t>(smem, 48 * 1024));
      int q = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, factor_kernel<B, TV>, FactorCap<B>::W * 32, smem);
      per_sm = q < 1 ? 1 : q;
      last_chunk = chunk;
    }
    const int grid = std::max(1, std::min(nchunks, per_sm * sms));
    ProfScope ps(BILU_PROF_FACTOR, stream);
    factor_kernel<B, TV><<<grid, FactorCap<B>::W * 32, smem, s>>>(n, chunk, nchunks, p->fact.d_bnd, p->fact.d_ord_l, p->fact.d_tick_l, p->d_lrp, p->d_lci,
                                                            p->d_urp, p->d_uci, f, p->nnz_l(), header, done,
                                                            spin);
  });
  return (int)cudaGetLastError();
}

template <typename TV>
int launch_scale_upper_t(const bilu_pattern* p, int32_t b, TV* f, void* stream) {
  const int32_t n = p->n;
  if (n == 0 || p->nnz_u() == 0) return 0;
  const size_t bb = (size_t)b * b;
  const TV* dinv = f + (size_t)p->nnz_l() * bb;
  TV* u = f + ((size_t)p->nnz_l() + n) * bb;
  const int grid = std::max(1, std::min((n + 7) / 8, device_sms() * 8));
  BILU_DISPATCH_B(b, {
    ProfScope ps(BILU_PROF_SCALE_UPPER, stream);
    scale_upper_kernel<B, TV><<<grid, 256, 0, (cudaStream_t)stream>>>(n, p->d_urp, dinv, u);
  });
  return (int)cudaGetLastError();
}

}  // namespace

int launch_backfill(const bilu_pattern* p, int32_t b, const double* a_vals, double* f, void* stream) {
  return launch_backfill_t<double>(p, b, a_vals, f, stream);
}
int launch_factor(const bilu_pattern* p, int32_t b, double* f, int32_t* header, int32_t* done, void* stream) {
  return launch_factor_t<double>(p, b, f, header, done, stream);
}
int launch_scale_upper(const bilu_pattern* p, int32_t b, double* f, void* stream) {
  return launch_scale_upper_t<double>(p, b, f, stream);
}
int launch_backfill_f32(const bilu_pattern* p, int32_t b, const double* a_vals, float* f, void* stream) {
  return launch_backfill_t<float>(p, b, a_vals, f, stream);
}
int launch_factor_f32(const bilu_pattern* p, int32_t b, float* f, int32_t* header, int32_t* done, void* stream) {
  return launch_factor_t<float>(p, b, f, header, done, stream);
}
int launch_scale_upper_f32(const bilu_pattern* p, int32_t b, float* f, void* stream) {
  return launch_scale_upper_t<float>(p, b, f, stream);
}

}  // namespace bilu
