// Double-float arithmetic on the FP32 pipes: a value is the unevaluated sum h + l of two floats
// (float2: .x high part, .y low part, about 48 significant bits).  Products are split exactly by
// fma (Dekker's TwoProduct with a hardware fma), additions' rounding errors captured by Knuth's
// TwoSum; the _rn intrinsics keep the compiler from contracting the error-free steps into fma.
// Shared by the double-float Cholesky of the line path and the trailing updates of the
// streaming path's blocked Cholesky.
#pragma once
#include <cuda_runtime.h>

namespace edt {

__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 df_norm(float2 a) { return fast_two_sum(a.x, a.y); }
__device__ __forceinline__ float2 df_of(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - double(h)));
}
__device__ __forceinline__ double df_val(float2 a) { return double(a.x) + double(a.y); }
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float2 s = two_sum(a.x, b.x);
  return fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = fmaf(a.x, b.y, fmaf(a.y, b.x, fmaf(a.x, b.x, -p)));
  return fast_two_sum(p, e);
}
// accumulator s (high sum, low sum; not normalised) += a * b
__device__ __forceinline__ void df_acc(float2& s, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = fmaf(a.x, b.y, fmaf(a.y, b.x, fmaf(a.x, b.x, -p)));
  const float2 t = two_sum(s.x, p);
  s.x = t.x;
  s.y = __fadd_rn(s.y, __fadd_rn(t.y, e));
}
__device__ __forceinline__ float2 shfl_df(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// 1 / sqrt(a) for a double-float a > 0: the FP32 estimate y0 and one Newton step carried in
// double-float, y = y0 + y0 (1 - a y0^2) / 2 (the step doubles the ~23 correct bits).
__device__ __forceinline__ float2 df_rsqrt(float2 a) {
  const float y0 = rsqrtf(a.x);
  const float2 y2 = df_mul(make_float2(y0, 0.f), make_float2(y0, 0.f));
  const float2 r = df_add(make_float2(1.f, 0.f), df_neg(df_mul(a, y2)));   // 1 - a y0^2, small
  return fast_two_sum(y0, 0.5f * y0 * r.x);
}

}  // namespace edt
