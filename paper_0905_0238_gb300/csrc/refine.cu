// Residual of the damped normal equations for one step of iterative refinement:
//   r_+- = Ahat^T (dhat_+- - Ahat x_+-)          (the -lam x term is added by refine_update)
// accumulated over every row of every subproblem, matrix-free: each kernel row
// a(z) = |s_f| g(k_p, z) g(k_q, z) is rebuilt from the FP32 table sqrt|s_f| g (rounded from
// the FP64 depth march), the row's prediction sum_z a(z) x(z) and residual u = d~ - a.x are
// formed in FP32, and w Re(conj(a(z)) u) is accumulated per lane in FP32 over the warp's 32
// rows (partial sums of <= 32 terms), then summed across warps and blocks in FP64.  Table
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
      const float2 dp = rhs[2 * ri[h]], dm = rhs[2 * ri[h] + 1];
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
  for (int i = threadIdx.x; i < 2 * nz; i += blockDim.x) {
    const int z = i >> 1, k = i & 1;
    double sacc = 0.0;
#pragma unroll
    for (int w = 0; w < RF_WARPS; ++w) sacc += red[w][k][z];
    atomicAdd(&d.r[(size_t(m) * nz + z) * 2 + k], sacc);
  }
}

}  // namespace

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
  switch (d.tune_rf) {
    case 1: refine_shape<8, 32>(d, s); break;
    case 2: refine_shape<4, 64>(d, s); break;
    case 3: refine_shape<8, 16>(d, s); break;
    default: refine_shape<4, 32>(d, s); break;
  }
  return cudaGetLastError();
}

}  // namespace edt
