// Plain FP64 normal matrices of the split systems (the FP64 comparison path).
//
// For midpoint index m with rows r = (f, p), q = (p - m) mod N and weights w_r:
//   a_r(z) = |s_f| g(k_p, z) g(k_q, z)                           (kernel row of eq. M)
//   G(z, z') = sum_r w_r [Re a_r(z) Re a_r(z') + Im a_r(z) Im a_r(z')]   = Re(A^H W A)
//   b_+-(z)  = sum_r w_r Re(conj(a_r(z)) d~_+-,r)                       = Re(A^H W d~)
// i.e. Ahat^T Ahat and Ahat^T dhat of the real-stacked system [Re A; Im A].  The kernel
// row is regenerated from the FP64 Green's-function table for every tile; nothing of
// size rows x nz is stored.  One block per (m, 64x64 upper tile); diagonal tiles also
// accumulate b.
#include "edt_internal.h"
#include "cplx.cuh"

namespace edt {

namespace {

constexpr int T64 = 64, KC = 16;

__global__ void __launch_bounds__(256) gram_f64_kernel(Dev d) {
  __shared__ double Ar[KC][T64], Ai[KC][T64], Br[KC][T64], Bi[KC][T64];
  __shared__ double2 rh[KC][2];
  const int m = blockIdx.y;
  // decode the upper-triangular tile pair (ti <= tj)
  const int nt = (d.nz + T64 - 1) / T64;
  int pid = blockIdx.x, ti = 0;
  while (pid >= nt - ti) { pid -= nt - ti; ++ti; }
  const int tj = ti + pid;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const long long r0 = d.row_off[m], nr = d.row_off[m + 1] - r0;
  const int N = d.N, msk = N - 1;
  double acc[4][4] = {};
  double bacc[2] = {0.0, 0.0};
  for (long long c0 = 0; c0 < nr; c0 += KC) {
    for (int e = threadIdx.x; e < KC * T64; e += blockDim.x) {
      int k = e / T64, zz = e - k * T64;
      double2 va = make_double2(0.0, 0.0), vb = va;
      if (c0 + k < nr) {
        uint32_t row = d.rows[r0 + c0 + k];
        int f = row_f(row), p = row_p(row), q = (p - m) & msk;
        int np = p <= N / 2 ? p : N - p, nq = q <= N / 2 ? q : N - q;
        double sa = d.fc[f].s_abs, w = row_w2(row) ? 2.0 : 1.0;
        const double2* g = d.g64 + size_t(f) * d.nk * d.nz;
        int za = ti * T64 + zz, zb = tj * T64 + zz;
        if (za < d.nz) va = sa * (g[size_t(np) * d.nz + za] * g[size_t(nq) * d.nz + za]);
        if (zb < d.nz) vb = (w * sa) * (g[size_t(np) * d.nz + zb] * g[size_t(nq) * d.nz + zb]);
        if (zz < 2 && ti == tj) {
          const double2* rr = reinterpret_cast<const double2*>(d.rhs) + 2 * size_t(r0 + c0 + k);
          rh[k][zz] = rr[zz];
        }
      } else if (zz < 2) {
        rh[k][zz] = make_double2(0.0, 0.0);
      }
      Ar[k][zz] = va.x; Ai[k][zz] = va.y;
      Br[k][zz] = vb.x; Bi[k][zz] = vb.y;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < KC; ++k) {
      double ar[4], ai[4], br[4], bi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ar[u] = Ar[k][ty * 4 + u]; ai[u] = Ai[k][ty * 4 + u];
        br[u] = Br[k][tx * 4 + u]; bi[u] = Bi[k][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(ar[u], br[v], fma(ai[u], bi[v], acc[u][v]));
    }
    if (ti == tj && threadIdx.x < T64) {
      for (int k = 0; k < KC; ++k) {
        double2 dp = rh[k][0], dm = rh[k][1];
        double xr = Br[k][threadIdx.x], xi = Bi[k][threadIdx.x];
        bacc[0] = fma(xr, dp.x, fma(xi, dp.y, bacc[0]));
        bacc[1] = fma(xr, dm.x, fma(xi, dm.y, bacc[1]));
      }
    }
    __syncthreads();
  }
  double* G = d.G + size_t(m) * d.nz * d.nz;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int zi = ti * T64 + ty * 4 + u, zj = tj * T64 + tx * 4 + v;
      if (zi < d.nz && zj < d.nz) {
        G[size_t(zi) * d.nz + zj] = acc[u][v];
        G[size_t(zj) * d.nz + zi] = acc[u][v];
      }
    }
  if (ti == tj && threadIdx.x < T64) {
    int z = ti * T64 + threadIdx.x;
    if (z < d.nz) {
      d.b[(size_t(m) * d.nz + z) * 2 + 0] = bacc[0];
      d.b[(size_t(m) * d.nz + z) * 2 + 1] = bacc[1];
    }
  }
}

}  // namespace

cudaError_t launch_gram_f64(const Dev& d, cudaStream_t s) {
  int nt = (d.nz + T64 - 1) / T64;
  dim3 g(nt * (nt + 1) / 2, d.nsub);
  gram_f64_kernel<<<g, 256, 0, s>>>(d);
  return cudaGetLastError();
}

}  // namespace edt
