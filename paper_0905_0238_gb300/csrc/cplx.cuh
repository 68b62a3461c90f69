// Small complex-arithmetic helpers on CUDA vector types (device and host).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace edt {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx_t = typename cplx_of<T>::type;

__host__ __device__ __forceinline__ double2 cmk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 cmk(float a, float b) { return make_float2(a, b); }

__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double2 a, double2 b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return cmk(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator*(float2 a, float2 b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return cmk(s * a.x, s * a.y); }

__host__ __device__ __forceinline__ double2 cconj(double2 a) { return cmk(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return cmk(a.x, -a.y); }

__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  // Smith's algorithm (scaled division, avoids overflow in |b|^2)
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, den = b.x + b.y * r;
    return cmk((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  } else {
    double r = b.x / b.y, den = b.x * r + b.y;
    return cmk((a.x * r + a.y) / den, (a.y * r - a.x) / den);
  }
}

__host__ __device__ __forceinline__ double2 cexp(double2 a) {
  double e = exp(a.x), s, c;
  sincos(a.y, &s, &c);
  return cmk(e * c, e * s);
}

// Principal square root, then the branch with non-negative imaginary part.
__host__ __device__ __forceinline__ double2 csqrt_upper(double2 w) {
  double r = hypot(w.x, w.y);
  double2 z;
  if (r == 0.0) return cmk(0.0, 0.0);
  if (w.x >= 0.0) {
    double t = sqrt(0.5 * (r + w.x));
    z = cmk(t, w.y / (2.0 * t));
  } else {
    double t = sqrt(0.5 * (r - w.x));
    z = cmk(fabs(w.y) / (2.0 * t), copysign(t, w.y));
  }
  if (z.y < 0.0) z = cmk(-z.x, -z.y);
  return z;
}

// e^{i kappa x} for kappa = (kx, ky) and x >= 0 given as FP32 (hi, lo) pairs, ~1e-7
// relative: the phase kx x is formed as an unevaluated sum p + q (exact product of the high
// parts by fma, plus the cross terms), reduced modulo 2 pi with a three-constant Cody-Waite
// split (2 pi = C1 + C2 + C3, C1 = 6.28125 so that k C1 is exact for |k| < 2^16), and
// evaluated with FP32 sincos; the decay e^{-ky x} uses the FP32 product.
__device__ __forceinline__ float2 expi_ff(float kxh, float kxl, float kyh, float xh, float xl) {
  const float C1 = 6.28125f, C2 = 0.0019353071693331003f, C3 = 1.0253131677018246e-11f;
  const float p = kxh * xh;
  const float q = fmaf(kxh, xh, -p) + fmaf(kxh, xl, kxl * xh);
  const float k = rintf(p * 0.15915493667125702f);
  float r = fmaf(-k, C1, p);
  r = fmaf(-k, C2, r);
  r = fmaf(-k, C3, r);
  r += q;
  float sn, cs;
  sincosf(r, &sn, &cs);
  const float mag = expf(-kyh * (xh + xl));
  return make_float2(mag * cs, mag * sn);
}

// 1 / b in FP32 complex arithmetic (|b| far from the FP32 range limits)
__device__ __forceinline__ float2 cinv32(float2 b) {
  const float r = 1.f / (b.x * b.x + b.y * b.y);
  return make_float2(b.x * r, -b.y * r);
}

// principal square root in FP32, then the branch with non-negative imaginary part
__device__ __forceinline__ float2 csqrt_upper32(float2 w) {
  const float r = hypotf(w.x, w.y);
  if (r == 0.f) return make_float2(0.f, 0.f);
  float2 z;
  if (w.x >= 0.f) {
    const float t = sqrtf(0.5f * (r + w.x));
    z = make_float2(t, w.y / (2.f * t));
  } else {
    const float t = sqrtf(0.5f * (r - w.x));
    z = make_float2(fabsf(w.y) / (2.f * t), copysignf(t, w.y));
  }
  if (z.y < 0.f) z = make_float2(-z.x, -z.y);
  return z;
}

__device__ __forceinline__ void split_ff(double v, float& hi, float& lo) {
  hi = float(v);
  lo = float(v - double(hi));
}

}  // namespace edt
