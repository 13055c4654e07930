// Two FP32 lanes (two neighbouring cells) handled by one thread with the
// packed FP32x2 arithmetic of sm_100-family GPUs (__ffma2_rn, __fadd2_rn,
// __fmul2_rn): one instruction does the same FP32 operation on both cells,
// with the per-lane rounding of the scalar instruction.
#pragma once
#include <cuda_runtime.h>

namespace lbm {

struct F2 {
  float2 v;
  __host__ __device__ F2() {}
  __host__ __device__ F2(float2 a) : v(a) {}
  __host__ __device__ F2(float a, float b) : v(make_float2(a, b)) {}
  __host__ __device__ explicit F2(double a) : v(make_float2((float)a, (float)a)) {}
  __host__ __device__ explicit F2(float a) : v(make_float2(a, a)) {}
  __host__ __device__ explicit F2(int a) : v(make_float2((float)a, (float)a)) {}
};

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return __fadd2_rn(a.v, b.v); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return __ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return __fmul2_rn(a.v, b.v); }
__device__ __forceinline__ F2 operator-(F2 a) { return __fmul2_rn(a.v, make_float2(-1.f, -1.f)); }
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(a.v.x / b.v.x, a.v.y / b.v.y); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }
__device__ __forceinline__ F2& operator*=(F2& a, F2 b) { return a = a * b; }

// a * b + c, fused: one FFMA for scalars (contracted), one packed FMA for F2
template <class R>
__device__ __forceinline__ R madd(R a, R b, R c) {
  return a * b + c;
}
template <>
__device__ __forceinline__ F2 madd<F2>(F2 a, F2 b, F2 c) {
  return __ffma2_rn(a.v, b.v, c.v);
}

}  // namespace lbm
