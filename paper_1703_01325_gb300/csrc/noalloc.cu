// noalloc.cu -- bilu_apply_noalloc: the preconditioner apply with its scratch
// in a fixed device array instead of a caller-supplied workspace.
//
// Some callers may not allocate device memory themselves: a host program that
// owns all device memory and hands plugins none of it, or code that must not
// trigger the device-wide synchronisation a cudaMalloc or cudaFree can cause.
// For them this entry point takes its scratch (the apply header and the
// intermediate y = L^{-1} r) from g_apply_scratch below, which every GPU that
// loads the library holds until the process exits.  Nothing here allocates:
// no cudaMalloc, no cudaFree, no allocating library routine.
#include <cuda_runtime.h>

#include <mutex>

#include "bilu_internal.h"

namespace {

// 32 MiB: room for the 256-byte apply header plus n*b doubles of y, i.e.
// n*b <= 4,194,272 (the 128 x 128 x 64, b = 3 system needs 3,145,728).
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;

static __device__ __align__(256) unsigned char g_apply_scratch[kNoAllocScratchBytes];

// Device address of g_apply_scratch per device ordinal, looked up once with
// that device current.  In host code the array's name is only a stand-in for
// the symbol; it must never be passed to a kernel.
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BILU_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_apply_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return BILU_ERR_CUDA;
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return BILU_OK;
}

}  // namespace

extern "C" int bilu_apply_noalloc(const bilu_pattern* p, int32_t b, const double* d_factors,
                                  const double* d_r, double* d_x, void* stream) {
  if (!p || b < 1 || b > 8) return BILU_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return BILU_ERR_CUDA;
  if (p->n > 0 && (!p->d_mem || dev != p->device)) return BILU_ERR_STATE;
  if (p->n == 0) return BILU_OK;
  if (!d_factors || !d_r || !d_x || (const void*)d_r == (const void*)d_x) return BILU_ERR_ARG;
  // The solve order must already exist (bilu_pattern_upload builds it):
  // building it here would allocate.
  if (p->solve.chunk <= 0 || !p->solve.upper || !p->solve.d_mem) return BILU_ERR_STATE;
  if (bilu::apply_workspace_bytes(p->n, b) > kNoAllocScratchBytes) return BILU_ERR_STATE;
  void* scratch = nullptr;
  const int st = scratch_for_current_device(&scratch);
  if (st != BILU_OK) return st;
  // launch_apply's first kernel resets the scratch header (tickets, abort
  // and error words) and marks y pending, so what a previous call left behind
  // is never read.
  return bilu::launch_apply(p, b, d_factors, d_r, d_x, scratch, nullptr, stream) == 0 ? BILU_OK
                                                                                     : BILU_ERR_CUDA;
}

// Status of the last bilu_apply_noalloc on the current device: the error word
// of the fixed scratch's header, copied out (4 bytes) after the stream's work.
// Uses only the address bilu_apply_noalloc cached; allocates nothing.
extern "C" int bilu_apply_noalloc_status(void* stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BILU_ERR_CUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    base = g_scratch_addr[dev];
  }
  if (!base) return BILU_ERR_STATE;
  int32_t err = 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&err, reinterpret_cast<const int32_t*>(base) + bilu::kErr, sizeof(err),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BILU_ERR_CUDA;
  return err;
}
