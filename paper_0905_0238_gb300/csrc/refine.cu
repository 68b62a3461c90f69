// Residual of the damped normal equations for one step of iterative refinement:
//   r_+- = Ahat^T (dhat_+- - Ahat x_+-)          (the -lam x term is added by refine_update)
// accumulated over every row of every subproblem, matrix-free: each kernel row
// a(z) = |s_f| g(k_p, z) g(k_q, z) is rebuilt from the FP32 table sqrt|s_f| g (rounded from
// the FP64 depth march), the row's prediction sum_z a(z) x(z) and residual u = d~ - a.x are
// formed in FP32, and w Re(conj(a(z)) u) is accumulated per lane in FP32 over the warp's
// rows, then summed across the CTA's warps in FP32; each CTA stores its partial (FP64) and
// refine_sum adds the partials of a subproblem in FP64 in CTA order, so repeated calls give the
// same bits.  Table
// rows are read with 16-byte loads (two depths per load) when nz is even, two rows at a time
// per warp so that both rows' loads are in flight together.  Each warp walks its rows two at a time so that the table loads of
// both rows are in flight together; rows p and -p sit side by side in the row order and
// share a table row, so one of the two reads is an L1 hit.  This is the matrix-free form of Ahat^T (dhat - Ahat x): the normal
// matrix used by the factorisation (from the tensor-core Gram) is not involved, so the
// refinement corrects the Gram's rounding.
#include "edt_internal.h"
#include "cplx.cuh"

#include <algorithm>

namespace edt {

namespace {

// Z4: float4 loads per lane per table row, i.e. nz <= 64 * Z4 (two depths per float4).
// FA: window geometry, where row ri of the subproblem is row ri of the assembled kernel
// table and the second factor is the table's row of ones (all weights 1).
// RF_WARPS warps per CTA, RF_ROWS_PER_WARP rows per warp: the CTA shape (autotuned).
template <int Z4, bool FA, int RF_WARPS, int RF_ROWS_PER_WARP>
__global__ void __launch_bounds__(RF_WARPS * 32) refine_kernel(Dev d) {
  constexpr int ZL = 64 * Z4;
  __shared__ float xs[2][ZL];
  __shared__ float red[RF_WARPS][2][ZL];
  const int m = blockIdx.y;
  const long long r0 = d.row_off[m], nr = d.row_off[m + 1] - r0;
  const long long c0 = (long long)blockIdx.x * RF_WARPS * RF_ROWS_PER_WARP;
  if (c0 >= nr || d.status[m] != EDT_OK) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nz = d.nz, N = d.N, msk = N - 1;
  for (int i = threadIdx.x; i < ZL; i += blockDim.x) {
    xs[0][i] = i < nz ? float(d.x[(size_t(m) * nz + i) * 2 + 0]) : 0.f;
    xs[1][i] = i < nz ? float(d.x[(size_t(m) * nz + i) * 2 + 1]) : 0.f;
  }
  __syncthreads();
  float acc[Z4][2][2];                         // [load t][depth 0/1 of the float4][rhs]
#pragma unroll
  for (int t = 0; t < Z4; ++t) acc[t][0][0] = acc[t][0][1] = acc[t][1][0] = acc[t][1][1] = 0.f;
  const float2* rhs = reinterpret_cast<const float2*>(d.rhs);
  const long long wb = c0 + warp * RF_ROWS_PER_WARP;
  const long long we = min(nr, wb + RF_ROWS_PER_WARP);
  for (long long i = wb; i < we; i += 2) {
    const bool two = i + 1 < we;
    float4 a[2][Z4];
    float wv[2];
    long long ri[2] = {r0 + i, r0 + (two ? i + 1 : i)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      size_t rp, rq;
      float w1 = 1.f;
      if (FA) {
        rp = size_t(ri[h]);
        rq = size_t(d.ones_row);
      } else {
        const uint32_t row = d.rows[ri[h]];
        const int f = row_f(row), p = row_p(row), q = (p - m) & msk;
        const int np = p <= N / 2 ? p : N - p, nq = q <= N / 2 ? q : N - q;
        rp = size_t(f) * d.nk + np;
        rq = size_t(f) * d.nk + nq;
        w1 = row_w2(row) ? 2.f : 1.f;
      }
      const float4* gp = reinterpret_cast<const float4*>(d.rowtab32 + rp * d.nzs);
      const float4* gq = reinterpret_cast<const float4*>(d.rowtab32 + rq * d.nzs);
      wv[h] = (h == 1 && !two) ? 0.f : w1;
#pragma unroll
      for (int t = 0; t < Z4; ++t) {
        const int z = 2 * lane + 64 * t;
        const float4 u = z < nz ? __ldg(gp + (z >> 1)) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 v = z < nz ? __ldg(gq + (z >> 1)) : make_float4(0.f, 0.f, 0.f, 0.f);
        // (z + 1 may be the zero padding of an odd nz)
        a[h][t] = make_float4(u.x * v.x - u.y * v.y, u.x * v.y + u.y * v.x,
                              u.z * v.z - u.w * v.w, u.z * v.w + u.w * v.z);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 tp = make_float2(0.f, 0.f), tm = tp;
#pragma unroll
      for (int t = 0; t < Z4; ++t) {
        const int z = 2 * lane + 64 * t;
        const float x0 = xs[0][z], x1 = xs[0][z + 1], y0 = xs[1][z], y1 = xs[1][z + 1];
        tp.x = fmaf(a[h][t].x, x0, fmaf(a[h][t].z, x1, tp.x));
        tp.y = fmaf(a[h][t].y, x0, fmaf(a[h][t].w, x1, tp.y));
        tm.x = fmaf(a[h][t].x, y0, fmaf(a[h][t].z, y1, tm.x));
        tm.y = fmaf(a[h][t].y, y0, fmaf(a[h][t].w, y1, tm.y));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        tp.x += __shfl_xor_sync(0xffffffffu, tp.x, o); tp.y += __shfl_xor_sync(0xffffffffu, tp.y, o);
        tm.x += __shfl_xor_sync(0xffffffffu, tm.x, o); tm.y += __shfl_xor_sync(0xffffffffu, tm.y, o);
      }
      const float w = wv[h];
      const float2 zero2 = make_float2(0.f, 0.f);
      const float2 dp = d.refine_nodata ? zero2 : rhs[2 * ri[h]];
      const float2 dm = d.refine_nodata ? zero2 : rhs[2 * ri[h] + 1];
      const float2 up = make_float2(w * (dp.x - tp.x), w * (dp.y - tp.y));
      const float2 um = make_float2(w * (dm.x - tm.x), w * (dm.y - tm.y));
#pragma unroll
      for (int t = 0; t < Z4; ++t) {
        acc[t][0][0] = fmaf(a[h][t].x, up.x, fmaf(a[h][t].y, up.y, acc[t][0][0]));
        acc[t][0][1] = fmaf(a[h][t].x, um.x, fmaf(a[h][t].y, um.y, acc[t][0][1]));
        acc[t][1][0] = fmaf(a[h][t].z, up.x, fmaf(a[h][t].w, up.y, acc[t][1][0]));
        acc[t][1][1] = fmaf(a[h][t].z, um.x, fmaf(a[h][t].w, um.y, acc[t][1][1]));
      }
    }
  }
#pragma unroll
  for (int t = 0; t < Z4; ++t) {
    const int z = 2 * lane + 64 * t;
    red[warp][0][z] = acc[t][0][0]; red[warp][1][z] = acc[t][0][1];
    red[warp][0][z + 1] = acc[t][1][0]; red[warp][1][z + 1] = acc[t][1][1];
  }
  __syncthreads();
  // the warps' FP32 partials added in FP32, in warp order (a handful of terms, each already an
  // FP32 sum); the CTA partials go to FP64 and are added across CTAs by refine_sum.  Every FP64
  // operation runs on GB300's narrow FP64 unit, so the CTA keeps them to one per output.
  double* part = d.rpart + (size_t(m) * d.rf_stride + blockIdx.x) * nz * 2;
  for (int i = threadIdx.x; i < 2 * nz; i += blockDim.x) {
    const int z = i >> 1, k = i & 1;
    float sacc = 0.f;
#pragma unroll
    for (int w = 0; w < RF_WARPS; ++w) sacc += red[w][k][z];
    part[i] = double(sacc);
  }
}

// ---- double-float residual (line geometry) -------------------------------------------
// The refinement converges to the solution of the system its residual describes, so at weak
// damping the residual must carry FP64 accuracy: its rounding errors reach x amplified by
// up to 1 / lam.  The accumulation Ahat^T u is the sensitive half (the prediction Ahat x only
// perturbs u like data noise, damped by 1 / (2 sqrt lam)), so here:
//   * each kernel row comes from the double-float table, sqrt|s_f| g = hi + lo (~1e-14),
//     as a = a_h + a_l with a_h the FP32 value of the hi-part product and a_l the rest
//     (exact product errors of the hi parts, the TwoSum error of their sum, and the
//     hi x lo cross terms);
//   * the prediction and u = w (d - a_h . x) stay FP32;
//   * every product a_h u is split exactly into p + e (fma), the p are summed per lane by
//     TwoSum (Knuth's error-free addition: each addition's rounding error is captured
//     exactly, the cascaded summation of Ogita, Rump and Oishi), the rounding errors, the e
//     and the a_l u go to a low-order FP32 sum; the lane sums are combined in FP64 across
//     warps and blocks.
// The error-free steps use the _rn intrinsics so that no multiply-add is contracted.

// exact product of two hi parts split as (rounded product, its error)
__device__ __forceinline__ float two_prod_err(float a, float b, float p) { return fmaf(a, b, -p); }

// a_h + a_l = (ph + pl)(qh + ql) for one complex depth value, to ~2^-44 relative
__device__ __forceinline__ void cmul_df(float2 ph, float2 pl, float2 qh, float2 ql, float2& ah, float2& al) {
  const float p1 = __fmul_rn(ph.x, qh.x), p2 = __fmul_rn(ph.y, qh.y);
  const float e1 = two_prod_err(ph.x, qh.x, p1), e2 = two_prod_err(ph.y, qh.y, p2);
  const float sr = __fsub_rn(p1, p2);
  const float br = __fsub_rn(sr, p1);
  const float er = __fadd_rn(__fsub_rn(p1, __fsub_rn(sr, br)), __fsub_rn(-p2, br));
  const float cr = fmaf(ph.x, ql.x, fmaf(pl.x, qh.x, -fmaf(ph.y, ql.y, __fmul_rn(pl.y, qh.y))));
  const float p3 = __fmul_rn(ph.x, qh.y), p4 = __fmul_rn(ph.y, qh.x);
  const float e3 = two_prod_err(ph.x, qh.y, p3), e4 = two_prod_err(ph.y, qh.x, p4);
  const float si = __fadd_rn(p3, p4);
  const float bi = __fsub_rn(si, p3);
  const float ei = __fadd_rn(__fsub_rn(p3, __fsub_rn(si, bi)), __fsub_rn(p4, bi));
  const float ci = fmaf(ph.x, ql.y, fmaf(pl.x, qh.y, fmaf(ph.y, ql.x, __fmul_rn(pl.y, qh.x))));
  ah = make_float2(sr, si);
  al = make_float2(((e1 - e2) + er) + cr, ((e3 + e4) + ei) + ci);
}

// TwoSum step: s + (the returned rounding error) = s_old + x exactly
__device__ __forceinline__ float two_sum_acc(float& s, float x) {
  const float t = __fadd_rn(s, x);
  const float b = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, b)), __fsub_rn(x, b));
  s = t;
  return e;
}

// (s, lo) += Re(conj(a) u) with a = ah + al, u exact FP32
__device__ __forceinline__ void acc_df(float& s, float& lo, float2 ah, float2 al, float2 u) {
  const float p1 = __fmul_rn(ah.x, u.x), p2 = __fmul_rn(ah.y, u.y);
  const float e = two_prod_err(ah.x, u.x, p1) + two_prod_err(ah.y, u.y, p2);
  const float r1 = two_sum_acc(s, p1);
  const float r2 = two_sum_acc(s, p2);
  lo += fmaf(al.x, u.x, fmaf(al.y, u.y, (e + r1) + r2));
}

template <int Z4, int RF_WARPS, int RF_ROWS_PER_WARP>
__global__ void __launch_bounds__(RF_WARPS * 32) refine_df_kernel(Dev d) {
  constexpr int ZL = 64 * Z4;
  __shared__ float xs[2][ZL];
  __shared__ double red[RF_WARPS][2][ZL];
  const int m = blockIdx.y;
  const long long r0 = d.row_off[m], nr = d.row_off[m + 1] - r0;
  const long long c0 = (long long)blockIdx.x * RF_WARPS * RF_ROWS_PER_WARP;
  if (c0 >= nr || d.status[m] != EDT_OK) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nz = d.nz, N = d.N, msk = N - 1;
  for (int i = threadIdx.x; i < ZL; i += blockDim.x) {
    xs[0][i] = i < nz ? float(d.x[(size_t(m) * nz + i) * 2 + 0]) : 0.f;
    xs[1][i] = i < nz ? float(d.x[(size_t(m) * nz + i) * 2 + 1]) : 0.f;
  }
  __syncthreads();
  // [load t][depth 0/1 of the float4][rhs]: high-order sum, low-order sum
  float as[Z4][2][2], al_[Z4][2][2];
#pragma unroll
  for (int t = 0; t < Z4; ++t)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int k = 0; k < 2; ++k) as[t][j][k] = al_[t][j][k] = 0.f;
  const float2* rhs = reinterpret_cast<const float2*>(d.rhs);
  const long long wb = c0 + warp * RF_ROWS_PER_WARP;
  const long long we = min(nr, wb + RF_ROWS_PER_WARP);
  for (long long i = wb; i < we; ++i) {
    const long long ri = r0 + i;
    const uint32_t row = d.rows[ri];
    const int f = row_f(row), p = row_p(row), q = (p - m) & msk;
    const int np = p <= N / 2 ? p : N - p, nq = q <= N / 2 ? q : N - q;
    const size_t rp = (size_t(f) * d.nk + np) * d.nzs, rq = (size_t(f) * d.nk + nq) * d.nzs;
    const float w = row_w2(row) ? 2.f : 1.f;
    const float4* gph = reinterpret_cast<const float4*>(d.g32 + rp);
    const float4* gqh = reinterpret_cast<const float4*>(d.g32 + rq);
    const float4* gpl = reinterpret_cast<const float4*>(d.g32lo + rp);
    const float4* gql = reinterpret_cast<const float4*>(d.g32lo + rq);
    float2 ah[Z4][2], al[Z4][2];
#pragma unroll
    for (int t = 0; t < Z4; ++t) {
      const int z = 2 * lane + 64 * t;
      const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 u = z < nz ? __ldg(gph + (z >> 1)) : zero, v = z < nz ? __ldg(gqh + (z >> 1)) : zero;
      const float4 ul = z < nz ? __ldg(gpl + (z >> 1)) : zero, vl = z < nz ? __ldg(gql + (z >> 1)) : zero;
      cmul_df(make_float2(u.x, u.y), make_float2(ul.x, ul.y), make_float2(v.x, v.y), make_float2(vl.x, vl.y),
              ah[t][0], al[t][0]);
      cmul_df(make_float2(u.z, u.w), make_float2(ul.z, ul.w), make_float2(v.z, v.w), make_float2(vl.z, vl.w),
              ah[t][1], al[t][1]);
    }
    float2 tp = make_float2(0.f, 0.f), tm = tp;
#pragma unroll
    for (int t = 0; t < Z4; ++t) {
      const int z = 2 * lane + 64 * t;
      const float x0 = xs[0][z], x1 = xs[0][z + 1], y0 = xs[1][z], y1 = xs[1][z + 1];
      tp.x = fmaf(ah[t][0].x, x0, fmaf(ah[t][1].x, x1, tp.x));
      tp.y = fmaf(ah[t][0].y, x0, fmaf(ah[t][1].y, x1, tp.y));
      tm.x = fmaf(ah[t][0].x, y0, fmaf(ah[t][1].x, y1, tm.x));
      tm.y = fmaf(ah[t][0].y, y0, fmaf(ah[t][1].y, y1, tm.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tp.x += __shfl_xor_sync(0xffffffffu, tp.x, o); tp.y += __shfl_xor_sync(0xffffffffu, tp.y, o);
      tm.x += __shfl_xor_sync(0xffffffffu, tm.x, o); tm.y += __shfl_xor_sync(0xffffffffu, tm.y, o);
    }
    const float2 zero2 = make_float2(0.f, 0.f);
    const float2 dp = d.refine_nodata ? zero2 : rhs[2 * ri];
    const float2 dm = d.refine_nodata ? zero2 : rhs[2 * ri + 1];
    const float2 up = make_float2(w * (dp.x - tp.x), w * (dp.y - tp.y));
    const float2 um = make_float2(w * (dm.x - tm.x), w * (dm.y - tm.y));
#pragma unroll
    for (int t = 0; t < Z4; ++t)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        acc_df(as[t][j][0], al_[t][j][0], ah[t][j], al[t][j], up);
        acc_df(as[t][j][1], al_[t][j][1], ah[t][j], al[t][j], um);
      }
  }
#pragma unroll
  for (int t = 0; t < Z4; ++t) {
    const int z = 2 * lane + 64 * t;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int k = 0; k < 2; ++k)
        red[warp][k][z + j] = double(as[t][j][k]) + double(al_[t][j][k]);
  }
  __syncthreads();
  double* part = d.rpart + (size_t(m) * d.rf_stride + blockIdx.x) * nz * 2;
  for (int i = threadIdx.x; i < 2 * nz; i += blockDim.x) {
    const int z = i >> 1, k = i & 1;
    double sacc = 0.0;
#pragma unroll
    for (int w = 0; w < RF_WARPS; ++w) sacc += red[w][k][z];
    part[i] = sacc;
  }
}

// r(m) = the partials of subproblem m's CTAs in CTA order (zero for a failed subproblem,
// whose CTAs stored nothing)
__global__ void __launch_bounds__(256) refine_sum_kernel(Dev d, int rpc) {
  const int m = blockIdx.x, nz = d.nz;
  const long long nr = d.row_off[m + 1] - d.row_off[m];
  const int ncta = d.status[m] == EDT_OK ? int((nr + rpc - 1) / rpc) : 0;
  const double* part = d.rpart + size_t(m) * d.rf_stride * nz * 2;
  for (int i = threadIdx.x; i < 2 * nz; i += blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < ncta; ++c) t += part[size_t(c) * nz * 2 + i];
    d.r[size_t(m) * nz * 2 + i] = t;
  }
}

// rows per refinement CTA of the autotuned shape tune_rf (warps x rows per warp)
int refine_rows_per_cta(int tune_rf) {
  switch (tune_rf) {
    case 1: return 8 * 32;
    case 2: return 4 * 64;
    case 3: return 8 * 16;
    default: return 4 * 32;
  }
}

}  // namespace

int refine_stride(long long rows_max_sub) {
  int least = refine_rows_per_cta(0);
  for (int t = 1; t <= 3; ++t) least = std::min(least, refine_rows_per_cta(t));
  return int((std::max(rows_max_sub, 1LL) + least - 1) / least);
}

template <int W, int R>
void refine_df_shape(const Dev& d, cudaStream_t s) {
  const long long rows_per_cta = W * R;
  dim3 g(unsigned((std::max(d.rows_max_sub, 1LL) + rows_per_cta - 1) / rows_per_cta), d.nsub);
  if (d.nzs <= 64) refine_df_kernel<1, W, R><<<g, W * 32, 0, s>>>(d);
  else if (d.nzs <= 128) refine_df_kernel<2, W, R><<<g, W * 32, 0, s>>>(d);
  else refine_df_kernel<4, W, R><<<g, W * 32, 0, s>>>(d);
}

template <int W, int R>
void refine_shape(const Dev& d, cudaStream_t s) {
  const long long rows_per_cta = W * R;
  dim3 g(unsigned((std::max(d.rows_max_sub, 1LL) + rows_per_cta - 1) / rows_per_cta), d.nsub);
  const bool fa = d.geom == EDT_GEOM_WINDOW;
  const int nz_even = d.nzs;
  if (nz_even <= 64) fa ? refine_kernel<1, true, W, R><<<g, W * 32, 0, s>>>(d) : refine_kernel<1, false, W, R><<<g, W * 32, 0, s>>>(d);
  else if (nz_even <= 128) fa ? refine_kernel<2, true, W, R><<<g, W * 32, 0, s>>>(d) : refine_kernel<2, false, W, R><<<g, W * 32, 0, s>>>(d);
  else fa ? refine_kernel<4, true, W, R><<<g, W * 32, 0, s>>>(d) : refine_kernel<4, false, W, R><<<g, W * 32, 0, s>>>(d);
}

cudaError_t launch_refine(const Dev& d, cudaStream_t s) {
  // table rows have an even stride (nzs), so 16-byte loads are aligned; the padding
  // element of an odd nz is zero and meets x = 0
  if (d.resid_df) {
    switch (d.tune_rf) {
      case 1: refine_df_shape<8, 32>(d, s); break;
      case 2: refine_df_shape<4, 64>(d, s); break;
      case 3: refine_df_shape<8, 16>(d, s); break;
      default: refine_df_shape<4, 32>(d, s); break;
    }
  } else {
    switch (d.tune_rf) {
      case 1: refine_shape<8, 32>(d, s); break;
      case 2: refine_shape<4, 64>(d, s); break;
      case 3: refine_shape<8, 16>(d, s); break;
      default: refine_shape<4, 32>(d, s); break;
    }
  }
  refine_sum_kernel<<<d.nsub, 256, 0, s>>>(d, refine_rows_per_cta(d.tune_rf));
  return cudaGetLastError();
}

}  // namespace edt
