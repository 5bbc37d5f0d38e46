// profile.cu -- optional per-kernel timing with CUDA events on the launching
// stream, and a count of every kernel the library launches.  When enabled,
// each instrumented launch is bracketed by two events; bilu_profile_read
// waits for them and accumulates the elapsed times.  Off by default.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "../../include/bilu_tuning.h"
#include "bilu_internal.h"

namespace bilu {
namespace {

struct Pending {
  cudaEvent_t a, b;
  int id;
};

struct Prof {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  double total_ms[BILU_PROF_NKERNELS] = {0};
  long long launches[BILU_PROF_NKERNELS] = {0};
  long long all_launches = 0;
};

Prof& prof() {
  static Prof p;
  return p;
}

cudaEvent_t take_event(Prof& p) {
  if (!p.pool.empty()) {
    cudaEvent_t e = p.pool.back();
    p.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void drain(Prof& p) {
  for (const Pending& q : p.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      p.total_ms[q.id] += ms;
      p.launches[q.id] += 1;
    }
    p.pool.push_back(q.a);
    p.pool.push_back(q.b);
  }
  p.pending.clear();
}

}  // namespace

void count_launches(int k) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.all_launches += k;
}

ProfScope::ProfScope(int id, void* stream) : id_(id), stream_(stream), a_(nullptr) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.all_launches += 1;
  if (!p.on) return;
  a_ = take_event(p);
  cudaEventRecord((cudaEvent_t)a_, (cudaStream_t)stream_);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  cudaEvent_t b = take_event(p);
  cudaEventRecord(b, (cudaStream_t)stream_);
  p.pending.push_back(Pending{(cudaEvent_t)a_, b, id_});
  if (p.pending.size() > 100000) drain(p);
}

}  // namespace bilu

extern "C" int bilu_profile_enable(int32_t on) {
  bilu::Prof& p = bilu::prof();
  std::lock_guard<std::mutex> g(p.mu);
  bilu::drain(p);
  p.on = on != 0;
  for (int q = 0; q < BILU_PROF_NKERNELS; ++q) {
    p.total_ms[q] = 0.0;
    p.launches[q] = 0;
  }
  return BILU_OK;
}

extern "C" int bilu_profile_read(int32_t kernel, int64_t* launches, double* total_ms) {
  if (kernel < 0 || kernel >= BILU_PROF_NKERNELS || !launches || !total_ms) return BILU_ERR_ARG;
  bilu::Prof& p = bilu::prof();
  std::lock_guard<std::mutex> g(p.mu);
  bilu::drain(p);
  *launches = p.launches[kernel];
  *total_ms = p.total_ms[kernel];
  return BILU_OK;
}

extern "C" int64_t bilu_launch_count(void) {
  bilu::Prof& p = bilu::prof();
  std::lock_guard<std::mutex> g(p.mu);
  return p.all_launches;
}
