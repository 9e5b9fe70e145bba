// Device helpers: loading a tile element in any storage format, rounding a
// float64/float32 value into a format (round-to-nearest-even; E4M3 with
// saturation to +-448), and the per-tile power-of-two E4M3 scale.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "mp_internal.h"

namespace mp {

__device__ __forceinline__ double load_f64(const char* base, int dt, int64_t i) {
  switch (dt) {
    case F64: return reinterpret_cast<const double*>(base)[i];
    case F32: return (double)reinterpret_cast<const float*>(base)[i];
    case BF16: return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(base)[i]);
    case F16: return (double)__half2float(reinterpret_cast<const __half*>(base)[i]);
    default: {
      __nv_fp8_e4m3 v;
      v.__x = reinterpret_cast<const __nv_fp8_storage_t*>(base)[i];
      return (double)float(v);
    }
  }
}

// Exact for every format but F64 (which callers with FP32 arithmetic never use).
__device__ __forceinline__ float load_f32(const char* base, int dt, int64_t i) {
  switch (dt) {
    case F64: return (float)reinterpret_cast<const double*>(base)[i];
    case F32: return reinterpret_cast<const float*>(base)[i];
    case BF16: return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(base)[i]);
    case F16: return __half2float(reinterpret_cast<const __half*>(base)[i]);
    default: {
      __nv_fp8_e4m3 v;
      v.__x = reinterpret_cast<const __nv_fp8_storage_t*>(base)[i];
      return float(v);
    }
  }
}

// Rounds v (already divided by the E4M3 scale for E4M3) into format dt.
__device__ __forceinline__ void store_round(char* base, int dt, int64_t i, double v) {
  switch (dt) {
    case F64: reinterpret_cast<double*>(base)[i] = v; break;
    case F32: reinterpret_cast<float*>(base)[i] = __double2float_rn(v); break;
    case BF16: reinterpret_cast<__nv_bfloat16*>(base)[i] = __double2bfloat16(v); break;
    case F16: reinterpret_cast<__half*>(base)[i] = __double2half(v); break;
    default:
      reinterpret_cast<__nv_fp8_storage_t*>(base)[i] =
          __nv_cvt_double_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
  }
}

__device__ __forceinline__ void store_round_f32(char* base, int dt, int64_t i, float v) {
  switch (dt) {
    case F64: reinterpret_cast<double*>(base)[i] = (double)v; break;
    case F32: reinterpret_cast<float*>(base)[i] = v; break;
    case BF16: reinterpret_cast<__nv_bfloat16*>(base)[i] = __float2bfloat16_rn(v); break;
    case F16: reinterpret_cast<__half*>(base)[i] = __float2half_rn(v); break;
    default:
      reinterpret_cast<__nv_fp8_storage_t*>(base)[i] =
          __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
  }
}

// Smallest power of two s with amax / s <= 448 (s = 1 for amax = 0 or not
// finite).  All comparisons are exact: 448 * 2^e is a float64 number.
__device__ __forceinline__ double e4m3_scale(double amax) {
  if (!(amax > 0.0) || !isfinite(amax)) return 1.0;
  int e = ilogb(amax) - 8;
  while (amax > ldexp(448.0, e)) ++e;
  while (e > -1074 && amax <= ldexp(448.0, e - 1)) --e;
  return ldexp(1.0, e);
}

// atomicMax of a non-negative float64 through its bit pattern (the order of
// non-negative IEEE doubles equals the order of their bits).
__device__ __forceinline__ void atomic_max_pos(unsigned long long* slot, double v) {
  if (v > 0.0) atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ double amax_value(const unsigned long long* slot) {
  return __longlong_as_double((long long)*slot);
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Progress counters of the task-graph kernels: acquire loads, release
// stores, and a bounded wait that gives up when the error word is set.
constexpr uint32_t DAG_WAIT_LIMIT = 1u << 21;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// A release at gpu scope is cumulative: after a __syncthreads(), one
// thread's release store (or reduction) publishes the stores that every
// thread of the block made before the barrier, with no separate fence.
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Waits until *ver >= need; false on timeout or when another CTA gave up.
// Chain-trace stamp `point` (%globaltimer ns and clock64) into a block's
// TRACE_WORDS words; no-op when tr is NULL (tracing off).
__device__ __forceinline__ void chain_stamp(unsigned long long* tr, int point) {
  if (!tr) return;
  unsigned long long g;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g));
  tr[point] = g;
  tr[8 + point] = (unsigned long long)clock64();
}

__device__ __forceinline__ bool dag_wait(const int* ver, int need, const int* err, int polls) {
  const uint32_t limit = polls > 0 ? (uint32_t)polls : DAG_WAIT_LIMIT;
  for (uint32_t i = 0; i < limit; ++i) {
    if (ld_acquire(ver) >= need) return true;
    if ((i & 63) == 63 && ld_acquire(err) != 0) return false;
    __nanosleep(64);
  }
  return false;
}

}  // namespace mp
