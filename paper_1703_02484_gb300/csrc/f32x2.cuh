// FP32 helpers shared by the all-pairs sweeps: Blackwell's packed f32x2
// arithmetic (two FP32 values in one 64-bit register pair, one instruction),
// the MUFU reciprocal square root, TwoSum accumulation and the status poll.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bd_internal.h"

namespace bdf {

typedef unsigned long long u64;

__device__ __forceinline__ float rsqrt_apx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// hi + lo += t with the rounding error of the high part kept in lo
__device__ __forceinline__ void two_sum(float &hi, float &lo, float t) {
  float s = __fadd_rn(hi, t);
  float bp = __fsub_rn(s, hi);
  float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(t, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

__device__ __forceinline__ int ctl_failed(const BdCtl *ctl) { return *(volatile const int *)&ctl->status; }

__device__ __forceinline__ u64 pk2(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void up2(u64 r, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

}  // namespace bdf
