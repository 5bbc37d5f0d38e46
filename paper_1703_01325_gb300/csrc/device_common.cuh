// device_common.cuh -- device helpers shared by the libbilu kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bilu_internal.h"

namespace bilu {

constexpr unsigned kFull = 0xffffffffu;

// "Not yet computed" marker of the sync-free triangular solves: a signalling
// NaN with a fixed payload.  IEEE arithmetic quiets every signalling NaN it
// touches, so no computed value carries this bit pattern; a stored value that
// would (a copied input) is replaced by a quiet NaN first.
constexpr unsigned long long kPending = 0x7FF4DEADBEEF0001ull;
constexpr unsigned long long kQuietNaN = 0x7FF8000000000000ull;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const void* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(void* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const void* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(void* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Relaxed load / store of a value's bit pattern (32 or 64 bits).
template <typename U>
__device__ __forceinline__ U ld_relaxed_bits(const void* p) {
  if constexpr (sizeof(U) == 8) return ld_relaxed_u64(p);
  else return ld_relaxed_u32(p);
}
template <typename U>
__device__ __forceinline__ void st_relaxed_bits(void* p, U v) {
  if constexpr (sizeof(U) == 8) st_relaxed_u64(p, v);
  else st_relaxed_u32(p, v);
}
__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_s32(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_s32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}
__device__ __forceinline__ long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}

// Bounded wait state: the first waiter that runs out of time records
// BILU_ERR_TIMEOUT and raises the abort word so that every other waiter
// leaves promptly.  No waiter ever traps.
struct Waiter {
  int* header;
  long long limit_ns;
  long long t0;
  int* stop_word;  // optional: raised too, so a caller's pipeline stops
  // Checks the abort word and the clock every (mask + 1) polls.
  __device__ __forceinline__ bool give_up(unsigned it, unsigned mask = 31u) {
    if ((it & mask) != 0u) return false;
    if (ld_volatile_s32(header + kAbort)) return true;
    if (t0 == 0) t0 = global_ns();
    if (global_ns() - t0 > limit_ns) {
      atomicCAS(header + kErr, 0, (int)BILU_ERR_TIMEOUT);
      atomicExch(header + kAbort, 1);
      if (stop_word) atomicExch(stop_word, 1);
      return true;
    }
    return false;
  }
};

// Bit patterns of a value type for the shared-memory value cache of the
// solves: "pending" is a signalling NaN with a fixed payload (no arithmetic
// produces one), "quiet" replaces a computed value that would collide.
template <typename TV>
struct ValueBits;
template <>
struct ValueBits<double> {
  using U = unsigned long long;
  static constexpr U kPend = kPending, kQuiet = kQuietNaN;
  __device__ static U bits(double v) { return (U)__double_as_longlong(v); }
  __device__ static double value(U u) { return __longlong_as_double((long long)u); }
};
template <>
struct ValueBits<float> {
  using U = unsigned int;
  static constexpr U kPend = 0x7FA5A5A5u, kQuiet = 0x7FC00000u;
  __device__ static U bits(float v) { return (U)__float_as_uint(v); }
  __device__ static float value(U u) { return __uint_as_float(u); }
};

// Publish one computed value of type TV for the sync-free solves: its bit
// pattern, relaxed (the value is its own ready flag); a value that would
// carry the pending pattern is stored as a quiet NaN.
template <typename TV>
__device__ __forceinline__ void publish_value(TV* p, TV v) {
  using VB = ValueBits<TV>;
  typename VB::U u = VB::bits(v);
  if (u == VB::kPend) u = VB::kQuiet;
  st_relaxed_bits<typename VB::U>(p, u);
}

// Wait until all N values of type TV in global memory at p hold computed
// values (relaxed loads, issued together each round: one L2 round trip per
// poll); false if the wait was abandoned.
template <int N, typename TV>
__device__ __forceinline__ bool wait_values_global(const TV* p, TV (&out)[N], Waiter& w) {
  using VB = ValueBits<TV>;
  using U = typename VB::U;
  w.t0 = 0;
  for (unsigned it = 1;; ++it) {
    U u[N];
#pragma unroll
    for (int q = 0; q < N; ++q) u[q] = ld_relaxed_bits<U>(p + q);
    bool all = true;
#pragma unroll
    for (int q = 0; q < N; ++q) all = all && (u[q] != VB::kPend);
    if (all) {
#pragma unroll
      for (int q = 0; q < N; ++q) out[q] = VB::value(u[q]);
      return true;
    }
    if (w.give_up(it)) return false;
  }
}

// Wait until all N values of type TV in this CTA's shared memory at p hold
// computed values (volatile loads: each value is its own ready flag, so no
// fence is needed); false if the wait was abandoned.  The abort word and the
// clock are consulted only every 1024 polls: a shared-memory poll is short.
template <int N, typename TV>
__device__ __forceinline__ bool wait_values_shared(const TV* p, TV (&out)[N], Waiter& w) {
  using VB = ValueBits<TV>;
  w.t0 = 0;
  const volatile typename VB::U* v = reinterpret_cast<const volatile typename VB::U*>(p);
  for (unsigned it = 1;; ++it) {
    typename VB::U u[N];
#pragma unroll
    for (int q = 0; q < N; ++q) u[q] = v[q];
    bool all = true;
#pragma unroll
    for (int q = 0; q < N; ++q) all = all && (u[q] != VB::kPend);
    if (all) {
#pragma unroll
      for (int q = 0; q < N; ++q) out[q] = VB::value(u[q]);
      return true;
    }
    if (w.give_up(it, 1023u)) return false;
  }
}

// Wait until *flag != 0 (acquire); false if the wait was abandoned.
__device__ __forceinline__ bool wait_flag(const int* flag, Waiter& w) {
  w.t0 = 0;
  for (unsigned it = 1;; ++it) {
    if (ld_acquire_s32(flag) != 0) return true;
    if (w.give_up(it)) return false;
  }
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ int ld_acquire_cta_shared_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_cta_shared_s32(int* p, int v) {
  asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}

// Wait until a shared-memory flag of this CTA equals `want` (acquire, CTA
// scope); false if the wait was abandoned.  The abort word (a global load)
// and the clock are consulted every 1024 polls only.
__device__ __forceinline__ bool wait_local_flag(const int* flag, int want, Waiter& w) {
  w.t0 = 0;
  for (unsigned it = 1;; ++it) {
    if (ld_acquire_cta_shared_s32(flag) == want) return true;
    if (w.give_up(it, 1023u)) return false;
  }
}

// double -> float, rounded to nearest even, on the integer pipes: rebias the
// exponent, keep 23 mantissa bits and round on the 29 dropped ones (round up
// when the dropped bits plus the kept last bit exceed half; a carry into the
// exponent is the correct rounding, up to infinity).  Zero keeps its sign.
// NaN, infinity and results outside the normal float range (subnormal,
// overflow) take the hardware conversion.  The two 32-bit halves are taken
// by an opaque move, so the compiler cannot turn the tests on them back into
// FP64 comparisons: the FP64 pipe (which also runs the hardware double ->
// float conversion) is the scarce unit on this part, and kernels that convert
// once per FMA use this function.  (On the triangular solves' chain of
// dependent rows its longer latency loses to the hardware conversion:
// measured 5-30 % slower there.)
__device__ __forceinline__ float d2f_rn(double d) {
  unsigned lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(d));
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned sign = hi & 0x80000000u;
  if (((hi << 1) | lo) == 0u) return __uint_as_float(sign);
  if (e - 897u > 253u) return (float)d;  // float exponent outside [1, 254]
  unsigned r = ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  r += (lo & 0x1FFFFFFFu) + (r & 1u) > 0x10000000u ? 1u : 0u;
  return __uint_as_float(sign | r);
}

// Lanes per output-component group for a b x b block in a 32-lane warp: the
// largest power of two G with G*b <= 32.
__host__ __device__ constexpr int groups_for(int b) {
  return b == 1 ? 32 : b == 2 ? 16 : b <= 4 ? 8 : 4;
}

}  // namespace bilu

#define BILU_DISPATCH_B(b, ...)                  \
  switch (b) {                                   \
    case 1: { constexpr int B = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int B = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int B = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int B = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int B = 5; __VA_ARGS__; } break; \
    case 6: { constexpr int B = 6; __VA_ARGS__; } break; \
    case 7: { constexpr int B = 7; __VA_ARGS__; } break; \
    case 8: { constexpr int B = 8; __VA_ARGS__; } break; \
    default: break;                              \
  }
