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

// ---- one 32 x 32 diagonal block of a blocked double-float Cholesky factorisation ----------
// Shared scratch of the diagonal-block factorisation.
struct DfDiagScratch {
  float2 L[32 * 33];                             // L_kk (lower, [i][l])
  float2 col[2][32], inv[32], xr[2][32];
  int fail;
};

// Diagonal block of step k0 of one subproblem (kb = min(32, n - k0) columns), factored and
// inverted in double-float by a 256-thread CTA: thread (warp, lane) holds
// elements (warp + 8 q, lane), q < 4; per column one pivot step, one scale step and one rank-1
// update step between barriers (the column double-buffered in shared memory); then X = L_kk^-1
// by the same right-looking sweep over the identity.  Writes L_kk (lower triangle) and its FP32
// copy (L32, may be null; X goes there too), X to the strict upper triangle (X_il at (l, i)),
// and the reciprocal pivots (dinv FP64; dinv32 FP32, may be null).  A non-positive or
// non-finite pivot sets EDT_ENOTPD.  Every thread of the CTA calls it; A's block must be final
// and visible to the CTA.
__device__ inline void df_diag_block(float2* A, float* L32, double* dinv, float* dinv32, int* status, int n,
                                     int k0, DfDiagScratch& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int kb = min(32, n - k0);
  float2 a[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = warp + 8 * q;
    a[q] = i < kb && lane <= i ? A[size_t(k0 + i) * n + k0 + lane] : make_float2(0.f, 0.f);
  }
  if (threadIdx.x == 0) sh.fail = 0;
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    float2* col = sh.col[j & 1];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (warp + 8 * q == j && lane == j) {
        const float2 djj = df_norm(a[q]);
        if (!(djj.x > 0.f) || !isfinite(djj.x)) {
          sh.fail = 1;
        } else {
          const float2 inv = df_rsqrt(djj);
          a[q] = df_mul(djj, inv);
          sh.inv[j] = inv;
          col[j] = a[q];
        }
      }
    }
    __syncthreads();
    if (sh.fail) break;                              // the same value in every thread
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = warp + 8 * q;
      if (lane == j && i > j && i < kb) { a[q] = df_mul(df_norm(a[q]), sh.inv[j]); col[i] = a[q]; }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = warp + 8 * q;
      if (lane > j && i >= lane && i < kb) df_acc(a[q], df_neg(col[i]), col[lane]);
    }
  }
  if (sh.fail) {
    if (threadIdx.x == 0) *status = EDT_ENOTPD;
    return;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = warp + 8 * q;
    if (i < kb && lane <= i) {
      a[q] = df_norm(a[q]);
      sh.L[i * 33 + lane] = a[q];
      A[size_t(k0 + i) * n + k0 + lane] = a[q];
      if (L32) L32[size_t(k0 + i) * n + k0 + lane] = a[q].x;
    }
  }
  if (threadIdx.x < kb) {
    dinv[k0 + threadIdx.x] = df_val(sh.inv[threadIdx.x]);
    if (dinv32) dinv32[k0 + threadIdx.x] = sh.inv[threadIdx.x].x;
  }
  __syncthreads();
  // X = L_kk^-1: right-looking forward substitution on the identity, row k final at step k
  float2 x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] = make_float2(warp + 8 * q == lane ? 1.f : 0.f, 0.f);
  for (int k = 0; k < kb; ++k) {
    float2* xr = sh.xr[k & 1];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (warp + 8 * q == k) {
        if (lane <= k) x[q] = df_mul(df_norm(x[q]), sh.inv[k]);
        xr[lane] = lane <= k ? x[q] : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = warp + 8 * q;
      if (i > k && i < kb && lane <= k) df_acc(x[q], df_neg(sh.L[i * 33 + k]), xr[lane]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = warp + 8 * q;
    if (i < kb && lane < i) {
      const float2 v = df_norm(x[q]);
      A[size_t(k0 + lane) * n + k0 + i] = v;
      if (L32) L32[size_t(k0 + lane) * n + k0 + i] = v.x;   // X in the FP32 copy too
    }
  }
}

}  // namespace edt
