// Residual of the damped normal equations for one step of iterative refinement:
//   r_+- = Ahat^T (dhat_+- - Ahat x_+-)          (the -lam x term is added by refine_update)
// accumulated over every row of every subproblem, matrix-free: each kernel row
// a(z) = |s_f| g(k_p, z) g(k_q, z) is rebuilt from the FP32 table sqrt|s_f| g (rounded from
// the FP64 depth march), the row's prediction sum_z a(z) x(z) and residual u = d~ - a.x are
// formed in FP32, and w Re(conj(a(z)) u) is accumulated per lane in FP32 over 16 rows at a
// time, then in FP64.  Each warp walks its rows two at a time so that the table loads of
// both rows are in flight together; rows p and -p sit side by side in the row order and
// share a table row, so one of the two reads is an L1 hit.  This is the matrix-free form of Ahat^T (dhat - Ahat x): the normal
// matrix used by the factorisation (from the tensor-core Gram) is not involved, so the
// refinement corrects the Gram's rounding.
#include "edt_internal.h"
#include "cplx.cuh"

namespace edt {

namespace {

constexpr int RF_WARPS = 8, RF_ROWS_PER_WARP = 32;

template <int ZPL>   // depths per lane: nz <= 32 * ZPL
__global__ void __launch_bounds__(RF_WARPS * 32) refine_kernel(Dev d) {
  __shared__ float xs[2][32 * ZPL];
  __shared__ double red[RF_WARPS][2][32 * ZPL];
  const int m = blockIdx.y;
  const long long r0 = d.row_off[m], nr = d.row_off[m + 1] - r0;
  const long long c0 = (long long)blockIdx.x * RF_WARPS * RF_ROWS_PER_WARP;
  if (c0 >= nr || d.status[m] != EDT_OK) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nz = d.nz, N = d.N, msk = N - 1;
  for (int i = threadIdx.x; i < 32 * ZPL; i += blockDim.x) {
    xs[0][i] = i < nz ? float(d.x[(size_t(m) * nz + i) * 2 + 0]) : 0.f;
    xs[1][i] = i < nz ? float(d.x[(size_t(m) * nz + i) * 2 + 1]) : 0.f;
  }
  __syncthreads();
  double acc64[ZPL][2];
  float acc[ZPL][2];
#pragma unroll
  for (int t = 0; t < ZPL; ++t) { acc64[t][0] = acc64[t][1] = 0.0; acc[t][0] = acc[t][1] = 0.f; }
  const float2* rhs = reinterpret_cast<const float2*>(d.rhs);
  const long long wb = c0 + warp * RF_ROWS_PER_WARP;
  const long long we = min(nr, wb + RF_ROWS_PER_WARP);
  int since = 0;
  // two rows per iteration: the table loads of both are in flight together
  for (long long i = wb; i < we; i += 2) {
    const bool two = i + 1 < we;
    float2 a[2][ZPL];
    float wv[2];
    long long ri[2] = {r0 + i, r0 + (two ? i + 1 : i)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t row = d.rows[ri[h]];
      const int f = row_f(row), p = row_p(row), q = (p - m) & msk;
      const int np = p <= N / 2 ? p : N - p, nq = q <= N / 2 ? q : N - q;
      const float2* gp = d.g32 + (size_t(f) * d.nk + np) * nz;
      const float2* gq = d.g32 + (size_t(f) * d.nk + nq) * nz;
      wv[h] = (h == 1 && !two) ? 0.f : (row_w2(row) ? 2.f : 1.f);
#pragma unroll
      for (int t = 0; t < ZPL; ++t) {
        const int z = lane + 32 * t;
        a[h][t] = z < nz ? __ldg(gp + z) : make_float2(0.f, 0.f);
        const float2 b = z < nz ? __ldg(gq + z) : make_float2(0.f, 0.f);
        a[h][t] = a[h][t] * b;
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 tp = make_float2(0.f, 0.f), tm = tp;
#pragma unroll
      for (int t = 0; t < ZPL; ++t) {
        const int z = lane + 32 * t;
        tp.x = fmaf(a[h][t].x, xs[0][z], tp.x); tp.y = fmaf(a[h][t].y, xs[0][z], tp.y);
        tm.x = fmaf(a[h][t].x, xs[1][z], tm.x); tm.y = fmaf(a[h][t].y, xs[1][z], tm.y);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        tp.x += __shfl_xor_sync(0xffffffffu, tp.x, o); tp.y += __shfl_xor_sync(0xffffffffu, tp.y, o);
        tm.x += __shfl_xor_sync(0xffffffffu, tm.x, o); tm.y += __shfl_xor_sync(0xffffffffu, tm.y, o);
      }
      const float w = wv[h];
      const float2 dp = rhs[2 * ri[h]], dm = rhs[2 * ri[h] + 1];
      const float2 up = make_float2(w * (dp.x - tp.x), w * (dp.y - tp.y));
      const float2 um = make_float2(w * (dm.x - tm.x), w * (dm.y - tm.y));
#pragma unroll
      for (int t = 0; t < ZPL; ++t) {
        acc[t][0] = fmaf(a[h][t].x, up.x, fmaf(a[h][t].y, up.y, acc[t][0]));
        acc[t][1] = fmaf(a[h][t].x, um.x, fmaf(a[h][t].y, um.y, acc[t][1]));
      }
    }
    since += 2;
    if (since >= 16) {
#pragma unroll
      for (int t = 0; t < ZPL; ++t) {
        acc64[t][0] += acc[t][0]; acc64[t][1] += acc[t][1];
        acc[t][0] = acc[t][1] = 0.f;
      }
      since = 0;
    }
  }
#pragma unroll
  for (int t = 0; t < ZPL; ++t) {
    red[warp][0][lane + 32 * t] = acc64[t][0] + acc[t][0];
    red[warp][1][lane + 32 * t] = acc64[t][1] + acc[t][1];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * nz; i += blockDim.x) {
    const int z = i >> 1, k = i & 1;
    double s = 0.0;
    for (int w = 0; w < RF_WARPS; ++w) s += red[w][k][z];
    atomicAdd(&d.r[(size_t(m) * nz + z) * 2 + k], s);
  }
}

}  // namespace

cudaError_t launch_refine(const Dev& d, cudaStream_t s) {
  const long long rows_per_cta = RF_WARPS * RF_ROWS_PER_WARP;
  dim3 g(unsigned((d.nf * (long long)d.N + rows_per_cta - 1) / rows_per_cta), d.nsub);
  if (d.nz <= 64) refine_kernel<2><<<g, RF_WARPS * 32, 0, s>>>(d);
  else if (d.nz <= 128) refine_kernel<4><<<g, RF_WARPS * 32, 0, s>>>(d);
  else refine_kernel<8><<<g, RF_WARPS * 32, 0, s>>>(d);
  return cudaGetLastError();
}

}  // namespace edt
