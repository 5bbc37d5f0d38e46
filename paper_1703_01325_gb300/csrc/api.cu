// api.cu -- C ABI entry points of libbilu (declared in include/bilu.h and
// include/bilu_tuning.h): argument checks, the pattern's device copy, and the
// stream-ordered launches of the kernels in spmv.cu, factor.cu, trisolve.cu and
// krylov.cu.
#include <cuda_runtime.h>

#include <cstring>
#include <new>

#include "../../include/bilu_tuning.h"
#include "bilu_internal.h"

using namespace bilu;

namespace {

bool valid_b(int32_t b) { return b >= 1 && b <= 8; }

// The schedules the factorization and the solves run on exist once the
// pattern is uploaded; only bilu_pattern_upload and bilu_pattern_schedule
// (re)build them.  The compute calls never do.
int solve_schedule(const bilu_pattern* p) {
  return (p->n == 0 || (p->solve.d_mem && p->solve.upper)) ? BILU_OK : BILU_ERR_STATE;
}
int factor_schedule(const bilu_pattern* p) { return (p->n == 0 || p->fact.d_mem) ? BILU_OK : BILU_ERR_STATE; }

int build_schedules(bilu_pattern* p) {
  if (make_schedule(p, &p->solve, solve_chunk_target(p), true) != 0) return BILU_ERR_OOM;
  if (!p->is_transpose && make_schedule(p, &p->fact, factor_chunk_target(p), false) != 0) return BILU_ERR_OOM;
  return BILU_OK;
}

int ready(const bilu_pattern* p) {
  if (!p) return BILU_ERR_ARG;
  if (p->n > 0 && !p->d_mem) return BILU_ERR_STATE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return BILU_ERR_CUDA;
  if (p->n > 0 && dev != p->device) return BILU_ERR_STATE;
  return BILU_OK;
}

int cuda_status(int e) { return e == 0 ? BILU_OK : BILU_ERR_CUDA; }

}  // namespace

extern "C" const char* bilu_status_string(int status) {
  switch (status) {
    case BILU_OK: return "ok";
    case BILU_ERR_ARG: return "invalid argument";
    case BILU_ERR_PATTERN: return "malformed block pattern (unsorted, duplicate or out-of-range column, or missing diagonal block)";
    case BILU_ERR_SINGULAR: return "singular or non-finite pivot block";
    case BILU_ERR_BREAKDOWN: return "Krylov breakdown (a zero or non-finite scalar)";
    case BILU_ERR_NOT_CONVERGED: return "iteration limit reached before the tolerance";
    case BILU_ERR_TIMEOUT: return "a bounded dependency wait timed out";
    case BILU_ERR_CUDA: return "CUDA runtime error";
    case BILU_ERR_OOM: return "out of memory or size overflow";
    case BILU_ERR_STATE: return "pattern not uploaded to this device, or workspace too small";
    default: return "unknown status";
  }
}

namespace bilu {

DeviceLayout device_layout(int32_t n, int64_t nnz_l, int64_t nnz_u, int64_t nslots) {
  DeviceLayout d;
  d.lrp = align256(sizeof(int32_t) * ((size_t)n + 1));
  d.lci = align256(sizeof(int32_t) * ((size_t)nnz_l + 1));
  d.urp = d.lrp;
  d.uci = align256(sizeof(int32_t) * ((size_t)nnz_u + 1));
  d.map = align256(sizeof(int32_t) * ((size_t)nslots + 1));
  d.total = d.lrp + d.lci + d.urp + d.uci + d.map;
  return d;
}

int ensure_host(const bilu_pattern* cp) {
  if (cp->host_ready) return BILU_OK;
  bilu_pattern* p = const_cast<bilu_pattern*>(cp);  // fills the lazily kept host copy (set-up/host calls only)
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return BILU_ERR_CUDA;
  if (dev != p->device || !p->d_sym || !p->d_mem) return BILU_ERR_STATE;
  const size_t n = (size_t)p->n, np = (size_t)p->cnt_p, nl = (size_t)p->cnt_l, nu = (size_t)p->cnt_u;
  try {
    p->rp.resize(n + 1);
    p->ci.resize(np);
    p->lev.resize(np);
    p->lvl_l.resize(n);
    p->lvl_u.resize(n);
    p->lrp.resize(n + 1);
    p->urp.resize(n + 1);
    p->lci.resize(nl);
    p->uci.resize(nu);
    p->slot_src.resize((size_t)p->nslots());
  } catch (const std::bad_alloc&) {
    return BILU_ERR_OOM;
  }
  auto get = [](void* dst, const void* src, size_t count) {
    return count == 0 || cudaMemcpy(dst, src, count * sizeof(int32_t), cudaMemcpyDeviceToHost) == cudaSuccess;
  };
  if (!get(p->rp.data(), p->d_rp, n + 1) || !get(p->ci.data(), p->d_ci, np) || !get(p->lev.data(), p->d_lev, np) ||
      !get(p->lvl_l.data(), p->d_lvl_l, n) || !get(p->lvl_u.data(), p->d_lvl_u, n) ||
      !get(p->lrp.data(), p->d_lrp, n + 1) || !get(p->urp.data(), p->d_urp, n + 1) ||
      !get(p->lci.data(), p->d_lci, nl) || !get(p->uci.data(), p->d_uci, nu) ||
      !get(p->slot_src.data(), p->d_slot_src, (size_t)p->nslots()))
    return BILU_ERR_CUDA;
  p->host_ready = true;
  return BILU_OK;
}

}  // namespace bilu

extern "C" int bilu_pattern_upload(bilu_pattern* p, void* stream) {
  if (!p) return BILU_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BILU_ERR_CUDA;
  if (!p->host_ready && p->d_mem && dev == p->device) {
    // completed on this device by bilu_symbolic_gpu: the copy is in place
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return BILU_ERR_CUDA;
    return build_schedules(p);
  }
  if (!p->host_ready) {
    // completed on another device: bring the host copy back from there first
    if (cudaSetDevice(p->device) != cudaSuccess) return BILU_ERR_CUDA;
    const int st = ensure_host(p);
    cudaSetDevice(dev);
    if (st != BILU_OK) return st;
  }
  if (p->d_mem) {
    cudaFree(p->d_mem);
    p->d_mem = nullptr;
  }
  // the schedules live on the device of the previous upload: rebuild them here
  free_schedule(&p->solve);
  free_schedule(&p->fact);
  const int32_t n = p->n;
  if (n == 0) {
    p->device = dev;
    return BILU_OK;
  }
  const DeviceLayout L = device_layout(n, p->nnz_l(), p->nnz_u(), p->nslots());
  void* mem = nullptr;
  if (cudaMalloc(&mem, L.total) != cudaSuccess) {
    cudaGetLastError();
    return BILU_ERR_OOM;
  }
  char* c = (char*)mem;
  p->d_lrp = (int32_t*)c; c += L.lrp;
  p->d_lci = (int32_t*)c; c += L.lci;
  p->d_urp = (int32_t*)c; c += L.urp;
  p->d_uci = (int32_t*)c; c += L.uci;
  p->d_slot_src = (int32_t*)c;
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemcpyAsync(p->d_lrp, p->lrp.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s);
  if (!p->lci.empty())
    cudaMemcpyAsync(p->d_lci, p->lci.data(), sizeof(int32_t) * p->lci.size(), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(p->d_urp, p->urp.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s);
  if (!p->uci.empty())
    cudaMemcpyAsync(p->d_uci, p->uci.data(), sizeof(int32_t) * p->uci.size(), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(p->d_slot_src, p->slot_src.data(), sizeof(int32_t) * p->slot_src.size(),
                  cudaMemcpyHostToDevice, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaFree(mem);
    return BILU_ERR_CUDA;
  }
  p->d_mem = mem;
  p->device = dev;
  if (p->d_sym) {  // the device-built copy of P' on the old device is no longer needed
    cudaFree(p->d_sym);
    p->d_sym = nullptr;
    p->d_rp = p->d_ci = p->d_lev = p->d_lvl_l = p->d_lvl_u = nullptr;
  }
  return build_schedules(p);
}

extern "C" int bilu_pattern_schedule(bilu_pattern* p, void* stream) {
  if (!p) return BILU_ERR_ARG;
  int st = ready(p);
  if (st) return st;
  if (p->n == 0) return BILU_OK;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return BILU_ERR_CUDA;
  return build_schedules(p);
}

extern "C" int bilu_pattern_schedule_info(const bilu_pattern* p, int32_t* solve_rows, int32_t* factor_rows) {
  if (!p) return BILU_ERR_ARG;
  if (solve_rows) *solve_rows = p->solve.d_mem ? p->solve.chunk : 0;
  if (factor_rows) *factor_rows = p->fact.d_mem ? p->fact.chunk : 0;
  return BILU_OK;
}

extern "C" void bilu_destroy_pattern(bilu_pattern* p) {
  if (!p) return;
  if (p->d_mem) cudaFree(p->d_mem);
  if (p->d_sym) cudaFree(p->d_sym);
  free_schedule(&p->solve);
  free_schedule(&p->fact);
  delete p;
}

extern "C" size_t bilu_factor_bytes(const bilu_pattern* p, int32_t b) {
  if (!p || !valid_b(b)) return 0;
  return (size_t)p->nslots() * b * b * sizeof(double);
}

extern "C" size_t bilu_factor_workspace_bytes(const bilu_pattern* p, int32_t b) {
  if (!p || !valid_b(b)) return 0;
  return kHeaderBytes + align256(sizeof(int32_t) * ((size_t)p->n + 1));
}

namespace {

template <typename TV>
int factor_impl(const bilu_pattern* p, int32_t b, const double* d_a_vals, TV* d_factors, void* d_work,
                size_t work_bytes, void* stream, bilu_factor_info* info) {
  if (info) {
    info->status = BILU_ERR_ARG;
    info->bad_row = -1;
    info->ms = 0.0;
  }
  if (!p || !valid_b(b) || p->is_transpose) return BILU_ERR_ARG;
  int st = ready(p);
  if (st) return st;
  if (p->n > 0 && (!d_a_vals || !d_factors || !d_work)) return BILU_ERR_ARG;
  if (work_bytes < bilu_factor_workspace_bytes(p, b)) return BILU_ERR_STATE;
  if (factor_schedule(p) != BILU_OK) return BILU_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* header = (int32_t*)d_work;
  int32_t* done = (int32_t*)((char*)d_work + kHeaderBytes);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  int e = 0;
  if constexpr (sizeof(TV) == sizeof(double)) {
    if (p->n > 0) e = launch_backfill(p, b, d_a_vals, d_factors, s);
    if (!e) e = launch_factor(p, b, d_factors, header, done, s);
    if (!e) e = launch_scale_upper(p, b, d_factors, s);
  } else {
    if (p->n > 0) e = launch_backfill_f32(p, b, d_a_vals, d_factors, s);
    if (!e) e = launch_factor_f32(p, b, d_factors, header, done, s);
    if (!e) e = launch_scale_upper_f32(p, b, d_factors, s);
  }
  cudaEventRecord(e1, s);
  int32_t hdr[kHeaderWords] = {0};
  if (!e) e = (int)cudaMemcpyAsync(hdr, header, kHeaderBytes, cudaMemcpyDeviceToHost, s);
  if (!e) e = (int)cudaStreamSynchronize(s);
  float ms = 0.f;
  if (!e) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e) return BILU_ERR_CUDA;
  st = hdr[kErr];
  if (info) {
    info->status = st;
    info->bad_row = (st == BILU_ERR_SINGULAR) ? hdr[kBadRow] : -1;
    info->ms = ms;
  }
  return st;
}

}  // namespace

extern "C" int bilu_factor(const bilu_pattern* p, int32_t b, const double* d_a_vals, double* d_factors,
                           void* d_work, size_t work_bytes, void* stream, bilu_factor_info* info) {
  return factor_impl<double>(p, b, d_a_vals, d_factors, d_work, work_bytes, stream, info);
}

extern "C" int bilu_factor_f32(const bilu_pattern* p, int32_t b, const double* d_a_vals, float* d_factors32,
                               void* d_work, size_t work_bytes, void* stream, bilu_factor_info* info) {
  return factor_impl<float>(p, b, d_a_vals, d_factors32, d_work, work_bytes, stream, info);
}

extern "C" size_t bilu_apply_workspace_bytes(const bilu_pattern* p, int32_t b) {
  if (!p || !valid_b(b)) return 0;
  return apply_workspace_bytes(p->n, b);
}

extern "C" int bilu_apply(const bilu_pattern* p, int32_t b, const double* d_factors,
                          const double* d_r, double* d_x, void* d_work, size_t work_bytes,
                          void* stream) {
  if (!p || !valid_b(b)) return BILU_ERR_ARG;
  int st = ready(p);
  if (st) return st;
  if (p->n == 0) return BILU_OK;
  if (!d_factors || !d_r || !d_x || !d_work || (const void*)d_r == (const void*)d_x) return BILU_ERR_ARG;
  if (work_bytes < apply_workspace_bytes(p->n, b)) return BILU_ERR_STATE;
  if (solve_schedule(p) != BILU_OK) return BILU_ERR_STATE;
  return cuda_status(launch_apply(p, b, d_factors, d_r, d_x, d_work, nullptr, stream));
}

extern "C" int bilu_workspace_status(const void* d_work, void* stream) {
  if (!d_work) return BILU_ERR_ARG;
  int err = 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&err, (const int32_t*)d_work + kErr, sizeof(int), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BILU_ERR_CUDA;
  return err;
}

extern "C" int bsr_spmv(int32_t n, int32_t b, const int32_t* d_row_ptr, const int32_t* d_col_idx,
                        const double* d_vals, const double* d_x, double* d_y, void* stream) {
  if (n < 0 || !valid_b(b)) return BILU_ERR_ARG;
  if (n == 0) return BILU_OK;
  if (!d_row_ptr || !d_col_idx || !d_vals || !d_x || !d_y || (const void*)d_x == (const void*)d_y)
    return BILU_ERR_ARG;
  return cuda_status(launch_spmv(n, b, d_row_ptr, d_col_idx, d_vals, d_x, d_y, stream));
}

extern "C" size_t bicgstab_workspace_bytes(const bilu_pattern* p, int32_t b) {
  if (!p || !valid_b(b)) return 0;
  return krylov_workspace_bytes(p->n, b);
}

static int g_check_every = 4;

extern "C" int bicgstab_solve(const bilu_pattern* p, const bilu_bsr* A, const double* d_factors,
                              const double* d_rhs, double* d_x, double tol, int32_t maxit,
                              void* d_work, size_t work_bytes, void* stream, bilu_solve_info* info) {
  if (info) {
    info->status = BILU_ERR_ARG;
    info->iters = 0;
    info->true_relres = 0.0;
    info->ms = 0.0;
  }
  if (!p || !A || !valid_b(A->b) || A->n != p->n || !(tol > 0.0) || maxit < 0) return BILU_ERR_ARG;
  int st = ready(p);
  if (st) return st;
  if (p->n == 0) {
    if (info) info->status = BILU_OK;
    return BILU_OK;
  }
  if (!A->row_ptr || !A->col_idx || !A->vals || !d_factors || !d_rhs || !d_x || !d_work ||
      (const void*)d_rhs == (const void*)d_x)
    return BILU_ERR_ARG;
  if (work_bytes < krylov_workspace_bytes(p->n, A->b)) return BILU_ERR_STATE;
  if (solve_schedule(p) != BILU_OK) return BILU_ERR_STATE;
  return run_bicgstab(p, A, d_factors, d_rhs, d_x, tol, maxit, d_work, stream, info, g_check_every);
}

extern "C" int bicgstab_solve_f32prec(const bilu_pattern* p, const bilu_bsr* A, const float* d_factors32,
                                      const double* d_rhs, double* d_x, double tol, int32_t maxit, void* d_work,
                                      size_t work_bytes, void* stream, bilu_solve_info* info) {
  if (info) {
    info->status = BILU_ERR_ARG;
    info->iters = 0;
    info->true_relres = 0.0;
    info->ms = 0.0;
  }
  if (!p || !A || !valid_b(A->b) || A->n != p->n || !(tol > 0.0) || maxit < 0) return BILU_ERR_ARG;
  int st = ready(p);
  if (st) return st;
  if (p->n == 0) {
    if (info) info->status = BILU_OK;
    return BILU_OK;
  }
  if (!A->row_ptr || !A->col_idx || !A->vals || !d_factors32 || !d_rhs || !d_x || !d_work ||
      (const void*)d_rhs == (const void*)d_x)
    return BILU_ERR_ARG;
  if (work_bytes < krylov_workspace_bytes(p->n, A->b)) return BILU_ERR_STATE;
  if (solve_schedule(p) != BILU_OK) return BILU_ERR_STATE;
  return run_bicgstab(p, A, nullptr, d_rhs, d_x, tol, maxit, d_work, stream, info, g_check_every, d_factors32);
}

extern "C" size_t gmres_workspace_bytes(const bilu_pattern* p, int32_t b, int32_t restart) {
  if (!p || !valid_b(b) || restart < 1 || restart > gmres_max_restart()) return 0;
  return gmres_workspace_bytes_impl(p->n, b, restart);
}

extern "C" int gmres_solve(const bilu_pattern* p, const bilu_bsr* A, const double* d_factors, const double* d_rhs,
                           double* d_x, double tol, int32_t maxit, int32_t restart, void* d_work,
                           size_t work_bytes, void* stream, bilu_solve_info* info) {
  if (info) {
    info->status = BILU_ERR_ARG;
    info->iters = 0;
    info->true_relres = 0.0;
    info->ms = 0.0;
  }
  if (!p || !A || !valid_b(A->b) || A->n != p->n || !(tol > 0.0) || maxit < 0 || restart < 1 ||
      restart > gmres_max_restart())
    return BILU_ERR_ARG;
  int st = ready(p);
  if (st) return st;
  if (p->n == 0) {
    if (info) info->status = BILU_OK;
    return BILU_OK;
  }
  if (!A->row_ptr || !A->col_idx || !A->vals || !d_factors || !d_rhs || !d_x || !d_work ||
      (const void*)d_rhs == (const void*)d_x)
    return BILU_ERR_ARG;
  if (work_bytes < gmres_workspace_bytes_impl(p->n, A->b, restart)) return BILU_ERR_STATE;
  if (solve_schedule(p) != BILU_OK) return BILU_ERR_STATE;
  return run_gmres(p, A, d_factors, d_rhs, d_x, tol, maxit, restart, d_work, stream, info, g_check_every);
}

// ---- mixed precision ----

extern "C" size_t bilu_factor_bytes_f32(const bilu_pattern* p, int32_t b) {
  if (!p || !valid_b(b)) return 0;
  return (size_t)p->nslots() * b * b * sizeof(float);
}

extern "C" int bilu_convert_f32(const double* d_src, float* d_dst, int64_t count, void* stream) {
  if (count < 0 || (count > 0 && (!d_src || !d_dst))) return BILU_ERR_ARG;
  return cuda_status(launch_convert_f32(d_src, d_dst, count, stream));
}

extern "C" int bilu_apply_f32(const bilu_pattern* p, int32_t b, const float* d_factors32, const double* d_r,
                              double* d_x, void* d_work, size_t work_bytes, void* stream) {
  if (!p || !valid_b(b)) return BILU_ERR_ARG;
  int st = ready(p);
  if (st) return st;
  if (p->n == 0) return BILU_OK;
  if (!d_factors32 || !d_r || !d_x || !d_work || (const void*)d_r == (const void*)d_x) return BILU_ERR_ARG;
  if (work_bytes < apply_workspace_bytes(p->n, b)) return BILU_ERR_STATE;
  if (solve_schedule(p) != BILU_OK) return BILU_ERR_STATE;
  return cuda_status(launch_apply_f32(p, b, d_factors32, d_r, d_x, d_work, nullptr, stream));
}

extern "C" int bsr_spmv_f32(int32_t n, int32_t b, const int32_t* d_row_ptr, const int32_t* d_col_idx,
                            const float* d_vals32, const double* d_x, double* d_y, void* stream) {
  if (n < 0 || !valid_b(b)) return BILU_ERR_ARG;
  if (n == 0) return BILU_OK;
  if (!d_row_ptr || !d_col_idx || !d_vals32 || !d_x || !d_y || (const void*)d_x == (const void*)d_y)
    return BILU_ERR_ARG;
  return cuda_status(launch_spmv_f32(n, b, d_row_ptr, d_col_idx, d_vals32, d_x, d_y, stream));
}

extern "C" int bsr_spmv_f32x(int32_t n, int32_t b, const int32_t* d_row_ptr, const int32_t* d_col_idx,
                             const float* d_vals32, const float* d_x32, double* d_y, void* stream) {
  if (n < 0 || !valid_b(b)) return BILU_ERR_ARG;
  if (n == 0) return BILU_OK;
  if (!d_row_ptr || !d_col_idx || !d_vals32 || !d_x32 || !d_y || (const void*)d_x32 == (const void*)d_y)
    return BILU_ERR_ARG;
  return cuda_status(launch_spmv_f32x(n, b, d_row_ptr, d_col_idx, d_vals32, d_x32, d_y, stream));
}

extern "C" size_t bicgstab_mixed_workspace_bytes(const bilu_pattern* p, int32_t b) {
  if (!p || !valid_b(b)) return 0;
  return krylov_mixed_workspace_bytes(p->n, b);
}

extern "C" int bicgstab_solve_mixed(const bilu_pattern* p, const bilu_bsr* A, const float* d_vals32,
                                    const float* d_factors32, const double* d_rhs, double* d_x, double tol,
                                    int32_t maxit, double inner_tol, int32_t inner_maxit, void* d_work,
                                    size_t work_bytes, void* stream, bilu_solve_info* info) {
  if (info) {
    info->status = BILU_ERR_ARG;
    info->iters = 0;
    info->true_relres = 0.0;
    info->ms = 0.0;
  }
  if (!p || !A || !valid_b(A->b) || A->n != p->n || !(tol > 0.0 && tol < 1.0) ||
      !(inner_tol > 0.0 && inner_tol < 1.0) || maxit < 0 || inner_maxit < 1)
    return BILU_ERR_ARG;
  int st = ready(p);
  if (st) return st;
  if (p->n == 0) {
    if (info) info->status = BILU_OK;
    return BILU_OK;
  }
  if (!A->row_ptr || !A->col_idx || !A->vals || !d_vals32 || !d_factors32 || !d_rhs || !d_x || !d_work ||
      (const void*)d_rhs == (const void*)d_x)
    return BILU_ERR_ARG;
  if (work_bytes < krylov_mixed_workspace_bytes(p->n, A->b)) return BILU_ERR_STATE;
  if (solve_schedule(p) != BILU_OK) return BILU_ERR_STATE;
  return run_bicgstab_mixed(p, A, d_vals32, d_factors32, d_rhs, d_x, tol, maxit, inner_tol, inner_maxit,
                            d_work, stream, info, g_check_every);
}

// ---- tuning and test hooks (include/bilu_tuning.h) ----

extern "C" int bilu_set_trisolve_chunk(int32_t rows) {
  if (rows < 0 || rows > 1024) return BILU_ERR_ARG;
  trisolve_config().chunk = rows;
  return BILU_OK;
}

extern "C" int32_t bilu_get_trisolve_chunk(void) { return trisolve_config().chunk; }

extern "C" int bilu_set_factor_chunk(int32_t rows) {
  if (rows < 0 || rows > 1024) return BILU_ERR_ARG;
  trisolve_config().factor_chunk = rows;
  return BILU_OK;
}

extern "C" int32_t bilu_get_factor_chunk(void) { return trisolve_config().factor_chunk; }

extern "C" int32_t bilu_auto_trisolve_chunk(const bilu_pattern* p) {
  return p ? auto_solve_chunk_target(p) : -1;
}

extern "C" int32_t bilu_auto_factor_chunk(const bilu_pattern* p) {
  return p ? auto_factor_chunk_target(p) : -1;
}

extern "C" int bilu_set_trisolve_warps(int32_t warps) {
  if (warps != 4 && warps != 8 && warps != 16) return BILU_ERR_ARG;
  trisolve_config().warps = warps;
  return BILU_OK;
}

extern "C" int bilu_set_trisolve_ctas_per_sm(int32_t ctas) {
  if (ctas < 0 || ctas > 32) return BILU_ERR_ARG;
  trisolve_config().ctas_per_sm = ctas;
  return BILU_OK;
}

extern "C" int bilu_set_spin_limit_ns(int64_t ns) {
  if (ns < 1000) return BILU_ERR_ARG;
  trisolve_config().spin_ns = ns;
  return BILU_OK;
}

extern "C" int bilu_set_check_every(int32_t iters) {
  if (iters < 1 || iters > 1000) return BILU_ERR_ARG;
  g_check_every = iters;
  return BILU_OK;
}

extern "C" int bilu_test_withhold_row(int32_t row) {
  trisolve_config().skip_row = row;
  return BILU_OK;
}

extern "C" int bilu_schedule_export(const bilu_pattern* p, int32_t rows, int32_t* nchunks, int32_t* bounds,
                                    int32_t* ord_lower, int32_t* ord_upper, int32_t* tick_lower,
                                    int32_t* tick_upper) {
  if (!p || !nchunks || rows < 1 || rows > 1024) return BILU_ERR_ARG;
  bilu_chunk_schedule tmp;
  if (!p->host_ready) {
    // a pattern that lives on the device: the device builder, orders copied back
    const int st = build_schedule_device(p, rows, true, &tmp);
    if (st != BILU_OK) return st;
    const size_t n0 = (size_t)p->n;
    tmp.ord_l.resize(n0);
    tmp.ord_u.resize(n0);
    const bool okc = n0 == 0 ||
                     (cudaMemcpy(tmp.ord_l.data(), tmp.d_ord_l, sizeof(int32_t) * n0, cudaMemcpyDeviceToHost) ==
                          cudaSuccess &&
                      cudaMemcpy(tmp.ord_u.data(), tmp.d_ord_u, sizeof(int32_t) * n0, cudaMemcpyDeviceToHost) ==
                          cudaSuccess);
    free_schedule(&tmp);
    if (!okc) return BILU_ERR_CUDA;
  } else {
    build_schedule(p, rows, true, &tmp);
  }
  *nchunks = tmp.nchunks;
  const size_t n = (size_t)p->n;
  auto put = [](int32_t* dst, const std::vector<int32_t>& v) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), sizeof(int32_t) * v.size());
  };
  put(bounds, tmp.bnd);
  if (n > 0) {
    put(ord_lower, tmp.ord_l);
    put(ord_upper, tmp.ord_u);
    put(tick_lower, tmp.tick_l);
    put(tick_upper, tmp.tick_u);
  }
  return BILU_OK;
}

// ---- adjoint ----

extern "C" int bilu_factor_transpose(const bilu_pattern* pt, int32_t b, const double* d_factors,
                                     double* d_factors_t, void* stream) {
  if (!pt || !valid_b(b) || !pt->is_transpose) return BILU_ERR_ARG;
  int st = ready(pt);
  if (st) return st;
  if (pt->n == 0) return BILU_OK;
  if (!d_factors || !d_factors_t || (const void*)d_factors == (const void*)d_factors_t) return BILU_ERR_ARG;
  return cuda_status(launch_gather_transpose(pt->nslots(), b, pt->d_slot_src, d_factors, d_factors_t, stream));
}

extern "C" int bsr_gather_transpose(int64_t nblocks, int32_t b, const int32_t* d_perm, const double* d_src,
                                    double* d_dst, void* stream) {
  if (nblocks < 0 || !valid_b(b)) return BILU_ERR_ARG;
  if (nblocks == 0) return BILU_OK;
  if (!d_perm || !d_src || !d_dst || (const void*)d_src == (const void*)d_dst) return BILU_ERR_ARG;
  return cuda_status(launch_gather_transpose(nblocks, b, d_perm, d_src, d_dst, stream));
}

extern "C" int bsr_outer_grad(int32_t n, int32_t b, const int32_t* d_row_ptr, const int32_t* d_col_idx,
                              const double* d_lambda, const double* d_x, double* d_grad, void* stream) {
  if (n < 0 || !valid_b(b)) return BILU_ERR_ARG;
  if (n == 0) return BILU_OK;
  if (!d_row_ptr || !d_col_idx || !d_lambda || !d_x || !d_grad) return BILU_ERR_ARG;
  return cuda_status(launch_outer_grad(n, b, d_row_ptr, d_col_idx, d_lambda, d_x, d_grad, stream));
}
