// Depth march for the reference Green's function g(k_n, z_j; omega~_f).
//
// g solves g'' + (omega~^2/c0(z)^2 - k^2) g = -delta(z) (the Green's-function equation of
// Section "Two dimensions" after a lateral Fourier transform; G~ = g / sqrt(2 pi)).  The
// paper does not say how to evaluate it in layers; this is the stable reflectivity
// recursion:
//   kappa_j = sqrt(omega~^2/c_j^2 - k^2), Im kappa_j >= 0,
//   upward:   r_{J-1} = 0, y = kappa_{j+1}(1 - r_{j+1})/(1 + r_{j+1}),
//             rho_j = (kappa_j - y)/(kappa_j + y), r_j = rho_j exp(2 i kappa_j h_j),
//   downward: A_0 = i/(2 kappa_0), A_{j+1} = A_j exp(i kappa_j h_j)(1 + rho_j)/(1 + r_{j+1}),
//   field:    g(z) = A_j [exp(i kappa_j (z - t_j)) + rho_j exp(i kappa_j (2 h_j - (z - t_j)))]
// in which no exponential grows.  Within a layer the two exponentials advance from one
// depth sample to the next by multiplication with exp(+-i kappa_j dz) (error ~ n ulp),
// re-anchored by a direct evaluation at every layer entry and chunk start.
//
// Kernels: green_coef (one thread per (f, n): the two recursions, all in FP64) and
// green_eval (a CTA per (f, block of 32 n); each warp marches a chunk of depths and
// stages its tile in shared memory so that the table rows are written coalesced).
#include "edt_internal.h"
#include "cplx.cuh"

namespace edt {

namespace {

constexpr int NCOEF = 5;   // kappa, rho, amp, exp(i kappa dz), exp(-i kappa dz)

__global__ void green_coef_kernel(Dev d) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  int f = blockIdx.y;
  if (n >= d.nk) return;
  const FreqConst fc = d.fc[f];
  const double L = double(d.N) * d.dx;
  const double k = 2.0 * M_PI * double(n) / L;
  const double2 om = cmk(fc.om_re, fc.om_im);
  const double2 om2 = om * om;
  const int J = d.nlayer;
  double2* c = d.coef + (size_t(f) * d.nk + n) * size_t(J) * NCOEF;
  for (int j = 0; j < J; ++j) {
    double inv_c2 = 1.0 / (d.layer_vel[j] * d.layer_vel[j]);
    double2 kap = csqrt_upper(cmk(om2.x * inv_c2 - k * k, om2.y * inv_c2));
    c[j * NCOEF + 0] = kap;
    c[j * NCOEF + 3] = cexp(cmk(-kap.y * d.dz, kap.x * d.dz));    // exp(i kap dz)
    c[j * NCOEF + 4] = cexp(cmk(kap.y * d.dz, -kap.x * d.dz));    // exp(-i kap dz)
  }
  // upward recursion; r_j is parked in the amplitude slot until the downward pass
  double2 r_next = cmk(0.0, 0.0);
  c[(J - 1) * NCOEF + 1] = cmk(0.0, 0.0);
  c[(J - 1) * NCOEF + 2] = r_next;
  for (int j = J - 2; j >= 0; --j) {
    double2 kj = c[j * NCOEF + 0], kn = c[(j + 1) * NCOEF + 0];
    double2 y = cdiv(kn * (cmk(1.0, 0.0) - r_next), cmk(1.0, 0.0) + r_next);
    double2 rho = cdiv(kj - y, kj + y);
    double h = d.layer_top[j + 1] - d.layer_top[j];
    double2 rj = rho * cexp(cmk(-2.0 * kj.y * h, 2.0 * kj.x * h));
    c[j * NCOEF + 1] = rho;
    c[j * NCOEF + 2] = rj;
    r_next = rj;
  }
  // downward recursion for the downgoing amplitude; jump g'(0+) - g'(0-) = -1
  double2 k0 = c[0];
  double2 amp = cdiv(cmk(0.0, 1.0), cmk(2.0 * k0.x, 2.0 * k0.y));
  for (int j = 0; j < J - 1; ++j) {
    double2 kj = c[j * NCOEF + 0];
    double2 rho = c[j * NCOEF + 1];
    double h = d.layer_top[j + 1] - d.layer_top[j];
    double2 r1 = c[(j + 1) * NCOEF + 2];
    c[j * NCOEF + 2] = amp;
    amp = cdiv(amp * cexp(cmk(-kj.y * h, kj.x * h)) * (cmk(1.0, 0.0) + rho), cmk(1.0, 0.0) + r1);
  }
  c[(J - 1) * NCOEF + 2] = amp;
}

constexpr int EV_WARPS = 4;
constexpr int EV_ZC = 16;   // depths per warp chunk

__global__ void __launch_bounds__(EV_WARPS * 32) green_eval_kernel(Dev d) {
  __shared__ double2 tile[EV_WARPS][32][EV_ZC + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int f = blockIdx.y;
  const int n0 = blockIdx.x * 32;
  const int n = n0 + lane;
  const int J = d.nlayer;
  const bool valid = n < d.nk;
  const double2* c = d.coef + (size_t(f) * d.nk + (valid ? n : 0)) * size_t(J) * NCOEF;
  const double sq = sqrt(d.fc[f].s_abs);
  for (int zc = warp * EV_ZC; zc < d.nz; zc += EV_WARPS * EV_ZC) {
    int cur = -1;
    double2 e1 = cmk(0.0, 0.0), e2 = cmk(0.0, 0.0), E = e1, Ei = e1, amp = e1, rho = e1;
    for (int i = 0; i < EV_ZC && zc + i < d.nz; ++i) {
      int z = zc + i;
      int l = d.z_layer[z];
      if (l != cur) {             // anchor: direct evaluation at layer entry / chunk start
        cur = l;
        double2 kap = c[l * NCOEF + 0];
        rho = c[l * NCOEF + 1];
        amp = c[l * NCOEF + 2];
        E = c[l * NCOEF + 3];
        Ei = c[l * NCOEF + 4];
        double off = d.z_off[z];
        e1 = cexp(cmk(-kap.y * off, kap.x * off));
        if (l < J - 1) {
          double a = 2.0 * (d.layer_top[l + 1] - d.layer_top[l]) - off;
          e2 = cexp(cmk(-kap.y * a, kap.x * a));
        } else {
          e2 = cmk(0.0, 0.0);
          rho = cmk(0.0, 0.0);
        }
      } else {
        e1 = e1 * E;
        e2 = e2 * Ei;
      }
      tile[warp][lane][i] = amp * (e1 + rho * e2);
    }
    __syncwarp();
    // coalesced write-out: two table rows (n) per pass, 16 depths each
    const int zi = lane & 15;
    for (int rr = 0; rr < 32; rr += 2) {
      int nl = rr + (lane >> 4);
      int nn = n0 + nl;
      int z = zc + zi;
      if (nn < d.nk && z < d.nz) {
        double2 v = tile[warp][nl][zi];
        size_t o = (size_t(f) * d.nk + nn) * d.nz + z;
        d.g64[o] = v;
        if (d.g32) d.g32[o] = make_float2(float(sq * v.x), float(sq * v.y));
      }
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_green(const Dev& d, cudaStream_t s) {
  dim3 g1((d.nk + 127) / 128, d.nf);
  green_coef_kernel<<<g1, 128, 0, s>>>(d);
  dim3 g2((d.nk + 31) / 32, d.nf);
  green_eval_kernel<<<g2, EV_WARPS * 32, 0, s>>>(d);
  return cudaGetLastError();
}

}  // namespace edt
