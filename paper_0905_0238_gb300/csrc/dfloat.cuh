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

// 1 / sqrt(a) for a double-float a > 0: the FP32 estimate y0 and one Newton step,
// y = y0 - y0 e / 2 with e = a y0^2 - 1 formed by fused multiply-adds on the exact square
// y0^2 = ph + pl (each fma rounds a quantity of order 2^-22 once, so e carries ~2^-46 absolute
// error); the step doubles the ~23 correct bits of the estimate.  Nine dependent operations
// after the estimate, on the critical path of every pivot.
__device__ __forceinline__ float2 df_rsqrt(float2 a) {
  const float y0 = rsqrtf(a.x);
  const float ph = __fmul_rn(y0, y0);
  const float pl = fmaf(y0, y0, -ph);
  float e = fmaf(a.x, ph, -1.0f);
  e = fmaf(a.x, pl, e);
  e = fmaf(a.y, ph, e);
  return fast_two_sum(y0, __fmul_rn(__fmul_rn(-0.5f, y0), e));
}

// ---- one 32 x 32 diagonal block of a blocked double-float Cholesky factorisation ----------
// Shared scratch of the diagonal-block factorisation.
struct DfDiagScratch {
  float2 col[3][32];                              // columns of L (three in use at a time)
  float2 xr[2][32];                               // finished rows of X = L^-1
  float2 pd[32];                                  // diagonal entries, published a step ahead
  float2 inv[32];                                 // 1 / L_jj
  int fail;
};

// Diagonal block of step k0 of one subproblem (kb = min(32, n - k0) columns), factored and
// inverted in double-float by a 256-thread CTA; thread (warp, lane) holds elements
// (warp + 8 q, lane), q < 4, of both A and X.  Right-looking with a one-column look-ahead, one
// barrier per column: in the phase that subtracts column j from the trailing block, the
// threads of column j + 1 (whose entries that subtraction finishes) also form its pivot
// L_{j+1,j+1}^2 = a_{j+1,j+1} - L_{j+1,j}^2 from the diagonal entry published one phase earlier,
// each of them redundantly (the same operations on the same values, so the same bits), take
// its 1 / sqrt and scale their entries: column j + 1 is ready at the next barrier.  The inverse
// rides along in the same phases: row j of X is u_j / L_jj, where u_i = e_i - sum_{k < i}
// L_ik X_k is updated with the finished row j - 1.  Writes L_kk (lower triangle) and
// its FP32 copy (L32, may be null; X goes there too), X to the strict upper triangle (X_il at
// (l, i)), and the reciprocal pivots (dinv FP64; dinv32 FP32, may be null).  A non-positive or
// non-finite pivot sets EDT_ENOTPD and returns false (in every thread).  Every thread of the CTA
// calls it; A's block must be final and visible to the CTA.
__device__ inline bool df_diag_block(float2* A, float* L32, double* dinv, float* dinv32, int* status, int n,
                                     int k0, DfDiagScratch& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int kb = min(32, n - k0);
  const float2 zero = make_float2(0.f, 0.f);
  float2 a[4], u[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = warp + 8 * q;
    a[q] = i < kb && lane <= i ? A[size_t(k0 + i) * n + k0 + lane] : zero;
    u[q] = make_float2(i == lane ? 1.f : 0.f, 0.f);
    if (i == lane && i < kb) sh.pd[i] = a[q];
  }
  if (threadIdx.x == 0) sh.fail = 0;
  __syncthreads();
  {                                               // column 0, by every thread
    const float2 d = df_norm(sh.pd[0]);
    if (!(d.x > 0.f) || !isfinite(d.x)) {
      if (threadIdx.x == 0) sh.fail = 1;
    } else {
      const float2 iv = df_rsqrt(d);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = warp + 8 * q;
        if (lane == 0 && i < kb) {
          a[q] = i == 0 ? df_mul(d, iv) : df_mul(df_norm(a[q]), iv);
          sh.col[0][i] = a[q];
        }
      }
      if (threadIdx.x == 0) sh.inv[0] = iv;
    }
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (sh.fail) break;                           // the same value in every thread
    const float2* cj = sh.col[j % 3];             // column j
    const float2* cp = sh.col[(j + 2) % 3];       // column j - 1
    float2* cn = sh.col[(j + 1) % 3];             // column j + 1, formed here
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = warp + 8 * q;
      if (lane > j && i >= lane && i < kb) df_acc(a[q], df_neg(cj[i]), cj[lane]);     // A -= L_j L_j^T
      if (j > 0 && lane < j && i >= j && i < kb)                                       // u_i -= L_{i,j-1} X_{j-1}
        df_acc(u[q], df_neg(cp[i]), sh.xr[(j - 1) & 1][lane]);
      if (i == j && lane <= j) {                                                       // row j of X
        u[q] = df_mul(df_norm(u[q]), sh.inv[j]);
        sh.xr[j & 1][lane] = u[q];
      }
      if (i == j + 2 && lane == j + 2 && i < kb) sh.pd[j + 2] = a[q];                  // next step's pivot input
    }
    if (j + 1 < kb && lane == j + 1) {            // column j + 1 (its entries are final now)
      float2 d = sh.pd[j + 1];
      df_acc(d, df_neg(cj[j + 1]), cj[j + 1]);
      d = df_norm(d);
      if (!(d.x > 0.f) || !isfinite(d.x)) {
        sh.fail = 1;
      } else {
        const float2 iv = df_rsqrt(d);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = warp + 8 * q;
          if (i > j && i < kb) {
            a[q] = i == j + 1 ? df_mul(d, iv) : df_mul(df_norm(a[q]), iv);
            cn[i] = a[q];
          }
        }
        if (warp == 0) sh.inv[j + 1] = iv;
      }
    }
    __syncthreads();
  }
  if (sh.fail) {
    if (threadIdx.x == 0) *status = EDT_ENOTPD;
    return false;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = warp + 8 * q;
    if (i < kb && lane <= i) {
      A[size_t(k0 + i) * n + k0 + lane] = a[q];
      if (L32) L32[size_t(k0 + i) * n + k0 + lane] = a[q].x;
    }
    if (i < kb && lane < i) {                     // X_{i, lane} to the upper triangle
      A[size_t(k0 + lane) * n + k0 + i] = u[q];
      if (L32) L32[size_t(k0 + lane) * n + k0 + i] = u[q].x;
    }
  }
  if (threadIdx.x < kb) {
    dinv[k0 + threadIdx.x] = df_val(sh.inv[threadIdx.x]);
    if (dinv32) dinv32[k0 + threadIdx.x] = sh.inv[threadIdx.x].x;
  }
  return true;
}
}  // namespace edt
