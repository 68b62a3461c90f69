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
// Kernels: green_layer (one thread per (f, n, layer): vertical wavenumber and the layer's
// phase factors, the FP64 transcendentals, fully parallel), green_recursion (one thread
// per (f, n): the two recursions, FP64), then one of two evaluations:
//   green_eval64  (FP64 table, and/or the FP32 table sqrt|s_f| g rounded from it, with the
//                 rounding remainder as a second FP32 table for a double-float pair):
//                 a CTA per (f, block of 32 n); each warp marches a chunk of depths by the
//                 recurrence and stages its tile in shared memory so the table rows are
//                 written coalesced;
//   green_eval32  (FP32 table sqrt|s_f| g for the mixed path): one thread per (f, n, z);
//                 each exponential's phase and decay are formed and range-reduced in FP64
//                 (Cody-Waite for the phase, integer/fraction split for the decay) and
//                 evaluated with FP32 sincos/exp2 of the reduced arguments, ~1e-7 relative.
// For the line inversion with the FP32 residual (GREEN_G32F) and at most 32 layers,
// green_kap32 (one thread per (f, n, layer)) and green_rec32 (one thread per (f, n)) replace
// green_layer and green_recursion: each kappa_j by an FP32 complex square root and one Newton
// step on the FP64 residual w - kappa^2 (the square of the FP32 root is exact in FP64, so the
// (hi, lo) pair carries kappa to ~1e-14 with four FP64 products instead of a complex FP64
// root), exp(i kappa_j h_j) by double-float phase reduction, and both recursions in FP32
// complex arithmetic; the outputs are the FP32 coefficients green_eval32 reads.  GB300's FP64
// rate made the FP64 transcendentals of green_layer and the recursion's FP64 divisions most of
// the depth march.
#include "edt_internal.h"
#include "cplx.cuh"

namespace edt {

namespace {

// coefficient slots per (f, n, layer): kappa, rho, amp, exp(i kappa dz), exp(-i kappa dz),
// exp(i kappa h), 1 / (1 + r_{j+1})
constexpr int NCOEF = 7;
constexpr int C_KAP = 0, C_RHO = 1, C_AMP = 2, C_E = 3, C_EI = 4, C_EH = 5, C_INV1R = 6;
// FP32 copies for the fast evaluation: kappa.x and kappa.y as (hi, lo) pairs, amp, rho
constexpr int NCOEF32 = 8;

// coefficient array layout [f][layer][slot][n]: consecutive wavenumbers are adjacent, so the
// per-(f, n) threads of every kernel below read and write them coalesced
__device__ __forceinline__ size_t cix(const Dev& d, int f, int n, int j, int k) {
  return ((size_t(f) * d.nlayer + j) * NCOEF + k) * d.nk + n;
}

// 1 / b with one real division (|b| is O(1e-3 .. 1e3) for every use here)
__device__ __forceinline__ double2 cinv(double2 b) {
  const double r = 1.0 / (b.x * b.x + b.y * b.y);
  return cmk(b.x * r, -b.y * r);
}

__global__ void green_layer_kernel(Dev d, int want_steps) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int J = d.nlayer;
  const long long total = (long long)d.nf * d.nk * J;
  if (gid >= total) return;
  const int n = int(gid % d.nk);                   // wavenumber fastest: coalesced stores
  const long long fj = gid / d.nk;
  const int j = int(fj % J), f = int(fj / J);
  const FreqConst fc = d.fc[f];
  const double L = double(d.N) * d.dx;
  const double k = d.kval ? d.kval[n] : 2.0 * M_PI * double(n) / L;
  const double2 om = cmk(fc.om_re, fc.om_im);
  const double2 om2 = om * om;
  const double inv_c2 = 1.0 / (d.layer_vel[j] * d.layer_vel[j]);
  const double2 kap = csqrt_upper(cmk(om2.x * inv_c2 - k * k, om2.y * inv_c2));
  double2* c = d.coef;
  c[cix(d, f, n, j, C_KAP)] = kap;
  if (j < J - 1) {
    const double h = d.layer_top[j + 1] - d.layer_top[j];
    c[cix(d, f, n, j, C_EH)] = cexp(cmk(-kap.y * h, kap.x * h));
  } else {
    c[cix(d, f, n, j, C_EH)] = cmk(1.0, 0.0);
  }
  if (want_steps) {
    const double2 E = cexp(cmk(-kap.y * d.dz, kap.x * d.dz));
    c[cix(d, f, n, j, C_E)] = E;
    c[cix(d, f, n, j, C_EI)] = cdiv(cmk(1.0, 0.0), E);
  }
}

__global__ void green_recursion_kernel(Dev d) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (n >= d.nk) return;
  const int J = d.nlayer;
  double2* c = d.coef;
  const double2 one = cmk(1.0, 0.0);
  // upward recursion for the reflection coefficient of the stack below each interface
  double2 r_next = cmk(0.0, 0.0);
  c[cix(d, f, n, J - 1, C_RHO)] = cmk(0.0, 0.0);
  double2 kn = c[cix(d, f, n, J - 1, C_KAP)];
  for (int j = J - 2; j >= 0; --j) {
    const double2 kj = c[cix(d, f, n, j, C_KAP)], eh = c[cix(d, f, n, j, C_EH)];
    const double2 inv1r = cinv(one + r_next);             // 1 / (1 + r_{j+1})
    const double2 y = kn * (one - r_next) * inv1r;
    const double2 rho = (kj - y) * cinv(kj + y);
    c[cix(d, f, n, j, C_RHO)] = rho;
    c[cix(d, f, n, j, C_INV1R)] = inv1r;
    r_next = rho * (eh * eh);
    kn = kj;
  }
  // downward recursion for the downgoing amplitude; jump g'(0+) - g'(0-) = -1
  const double2 k0 = c[cix(d, f, n, 0, C_KAP)];
  double2 amp = cmk(0.0, 0.5) * cinv(k0);
  for (int j = 0; j < J - 1; ++j) {
    c[cix(d, f, n, j, C_AMP)] = amp;
    amp = amp * c[cix(d, f, n, j, C_EH)] * (one + c[cix(d, f, n, j, C_RHO)]) * c[cix(d, f, n, j, C_INV1R)];
  }
  c[cix(d, f, n, J - 1, C_AMP)] = amp;
  if (d.coef32) {
    float* c32 = d.coef32 + (size_t(f) * d.nk + n) * size_t(J) * NCOEF32;
    for (int j = 0; j < J; ++j) {
      const double2 kap = c[cix(d, f, n, j, C_KAP)], a = c[cix(d, f, n, j, C_AMP)], r = c[cix(d, f, n, j, C_RHO)];
      const float kxh = float(kap.x), kyh = float(kap.y);
      float* o = c32 + j * NCOEF32;
      o[0] = kxh; o[1] = float(kap.x - double(kxh));
      o[2] = kyh; o[3] = float(kap.y - double(kyh));
      o[4] = float(a.x); o[5] = float(a.y);
      o[6] = j < J - 1 ? float(r.x) : 0.f; o[7] = j < J - 1 ? float(r.y) : 0.f;
    }
  }
}

// The FP32 recursion's rounding errors (and those of its FP32 exponentials) compound over the
// layers, about a few FP32 ulps per layer in the amplitudes: deeper stacks keep the FP64 march.
constexpr int COEF32_MAX_LAYERS = 32;

// FP32 coefficients, pass 1: one thread per (f, n, layer) -- kappa_j (FP32 root, one Newton
// step on the FP64 residual) and exp(i kappa_j h_j), the latter parked in the amplitude slots
// until the recursion replaces it.
__global__ void green_kap32_kernel(Dev d) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int J = d.nlayer;
  const long long total = (long long)d.nf * d.nk * J;
  if (gid >= total) return;
  const int j = int(gid % J);
  const long long fn = gid / J;
  const int n = int(fn % d.nk), f = int(fn / d.nk);
  const FreqConst fc = d.fc[f];
  const double L = double(d.N) * d.dx;
  const double k = d.kval ? d.kval[n] : 2.0 * M_PI * double(n) / L;
  const double om2r = fc.om_re * fc.om_re - fc.om_im * fc.om_im, om2i = 2.0 * fc.om_re * fc.om_im;
  const double ic2 = 1.0 / (d.layer_vel[j] * d.layer_vel[j]);
  const double wr2 = om2r * ic2 - k * k, wi2 = om2i * ic2;
  const float2 k32 = csqrt_upper32(make_float2(float(wr2), float(wi2)));
  const double rr = wr2 - (double(k32.x) * k32.x - double(k32.y) * k32.y);
  const double ri = wi2 - 2.0 * double(k32.x) * k32.y;
  const float2 dk = (k32.x == 0.f && k32.y == 0.f)
                        ? make_float2(0.f, 0.f)
                        : make_float2(float(rr), float(ri)) * cinv32(make_float2(2.f * k32.x, 2.f * k32.y));
  float2 eh = make_float2(1.f, 0.f);
  if (j + 1 < J) {
    float hh, hl;
    split_ff(d.layer_top[j + 1] - d.layer_top[j], hh, hl);
    eh = expi_ff(k32.x, dk.x, k32.y, hh, hl);            // exp(i kappa_j h_j)
  }
  float4* o = reinterpret_cast<float4*>(d.coef32 + size_t(gid) * NCOEF32);
  o[0] = make_float4(k32.x, dk.x, k32.y, dk.y);
  o[1] = make_float4(eh.x, eh.y, 0.f, 0.f);
}

// Pass 2: one thread per (f, n) -- the upward recursion for rho_j (stored; the amplitude slot
// takes exp(i kappa_j h_j) / (1 + r_{j+1})), then the downward one for the amplitudes, in FP32.
__global__ void __launch_bounds__(128) green_rec32_kernel(Dev d) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (n >= d.nk) return;
  const int J = d.nlayer;
  float4* c4 = reinterpret_cast<float4*>(d.coef32 + (size_t(f) * d.nk + n) * size_t(J) * NCOEF32);
  const float2 one = make_float2(1.f, 0.f);
  // upward: r_{J-1} = 0; y = kappa_{j+1}(1 - r_{j+1})/(1 + r_{j+1}); rho_j = (kappa_j - y)/(kappa_j + y)
  float2 r = make_float2(0.f, 0.f);
  float4 kn4 = c4[2 * (J - 1)];
  float2 kn = make_float2(kn4.x + kn4.y, kn4.z + kn4.w);
  c4[2 * (J - 1) + 1] = make_float4(0.f, 0.f, 0.f, 0.f);   // amplitude set below; rho_{J-1} = 0
  for (int j = J - 2; j >= 0; --j) {
    const float4 kj4 = c4[2 * j], ah = c4[2 * j + 1];
    const float2 kj = make_float2(kj4.x + kj4.y, kj4.z + kj4.w), eh = make_float2(ah.x, ah.y);
    const float2 inv1r = cinv32(one + r);
    const float2 y = kn * (one - r) * inv1r;
    const float2 rho = (kj - y) * cinv32(kj + y);
    r = rho * (eh * eh);
    const float2 ehi = eh * inv1r;                            // exp(i kappa_j h_j) / (1 + r_{j+1})
    c4[2 * j + 1] = make_float4(ehi.x, ehi.y, rho.x, rho.y);
    kn = kj;
  }
  // downward: A_0 = i / (2 kappa_0), A_{j+1} = A_j exp(i kappa_j h_j)(1 + rho_j)/(1 + r_{j+1})
  const float4 k04 = c4[0];
  float2 amp = make_float2(0.f, 0.5f) * cinv32(make_float2(k04.x + k04.y, k04.z + k04.w));
  for (int j = 0; j < J; ++j) {
    const float4 ah = c4[2 * j + 1];                          // (ehi, rho)
    c4[2 * j + 1] = make_float4(amp.x, amp.y, ah.z, ah.w);
    if (j + 1 < J) amp = amp * make_float2(ah.x, ah.y) * (one + make_float2(ah.z, ah.w));
  }
}

constexpr int EV_WARPS = 4;
constexpr int EV_ZC = 16;   // depths per warp chunk

__global__ void __launch_bounds__(EV_WARPS * 32) green_eval64_kernel(Dev d) {
  __shared__ double2 tile[EV_WARPS][32][EV_ZC + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int f = blockIdx.y;
  const int n0 = blockIdx.x * 32;
  const int n = n0 + lane;
  const int J = d.nlayer;
  const bool valid = n < d.nk;
  const double2* c = d.coef;
  const int nn0 = valid ? n : 0;
  const double sq = sqrt(d.fc[f].s_abs);
  for (int zc = warp * EV_ZC; zc < d.nz; zc += EV_WARPS * EV_ZC) {
    int cur = -1;
    double2 e1 = cmk(0.0, 0.0), e2 = e1, E = e1, Ei = e1, amp = e1, rho = e1;
    for (int i = 0; i < EV_ZC && zc + i < d.nz; ++i) {
      const int z = zc + i;
      const int l = d.z_layer[z];
      if (l != cur) {             // anchor: direct evaluation at layer entry / chunk start
        cur = l;
        const double2 kap = c[cix(d, f, nn0, l, C_KAP)];
        rho = c[cix(d, f, nn0, l, C_RHO)];
        amp = c[cix(d, f, nn0, l, C_AMP)];
        E = c[cix(d, f, nn0, l, C_E)];
        Ei = c[cix(d, f, nn0, l, C_EI)];
        const double off = d.z_off[z];
        e1 = cexp(cmk(-kap.y * off, kap.x * off));
        if (l < J - 1) {
          const double a = 2.0 * (d.layer_top[l + 1] - d.layer_top[l]) - off;
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
    const int zi = lane & 15;
    for (int rr = 0; rr < 32; rr += 2) {
      const int nl = rr + (lane >> 4);
      const int nn = n0 + nl;
      const int z = zc + zi;
      if (nn < d.nk && z < d.nz) {
        const double2 v = tile[warp][nl][zi];
        if (d.g64) d.g64[(size_t(f) * d.nk + nn) * d.nz + z] = v;
        if (d.g32) {
          // sqrt|s_f| g rounded to FP32, and (double-float table) the FP32 rounding of the rest
          const double sx = sq * v.x, sy = sq * v.y;
          const float hx = float(sx), hy = float(sy);
          const size_t o32 = (size_t(f) * d.nk + nn) * d.nzs + z;
          d.g32[o32] = make_float2(hx, hy);
          if (d.g32lo) d.g32lo[o32] = make_float2(float(sx - double(hx)), float(sy - double(hy)));
        }
      }
    }
    __syncwarp();
  }
}

// One CTA per table row (f, n), threads over depth; the row's largest |value| goes to rowmax
// (when present) for the FP16 operand scales of the Gram, so that no pass re-reads the table.
__global__ void __launch_bounds__(256) green_eval32_kernel(Dev d) {
  __shared__ float red[8];
  const long long fn = blockIdx.x;
  const int J = d.nlayer;
  const int f = int(fn / d.nk);
  const float sq = d.fc32_sqrt_s[f];
  float mx = 0.f;
  for (int z = threadIdx.x; z < d.nz; z += blockDim.x) {
    const int l = d.z_layer[z];
    const float4 zo = reinterpret_cast<const float4*>(d.z_off32)[z];   // off (hi, lo), 2h - off (hi, lo)
    const float4* c4 = reinterpret_cast<const float4*>(d.coef32 + (fn * J + l) * NCOEF32);
    const float4 k4 = c4[0], ar = c4[1];
    float2 e = expi_ff(k4.x, k4.y, k4.z, zo.x, zo.y);
    if (l < J - 1) {
      const float2 e2 = expi_ff(k4.x, k4.y, k4.z, zo.z, zo.w);
      e = e + make_float2(ar.z, ar.w) * e2;
    }
    const float2 g = make_float2(ar.x, ar.y) * e;
    const float2 v = make_float2(sq * g.x, sq * g.y);
    d.g32[size_t(fn) * d.nzs + z] = v;
    mx = fmaxf(mx, sqrtf(v.x * v.x + v.y * v.y));
  }
  if (!d.rowmax) return;                           // the same in the whole CTA
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < int(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
    d.rowmax[fn] = mx;
  }
}

}  // namespace

cudaError_t launch_green(const Dev& d, cudaStream_t s, int tables) {
  const bool fast32 = tables == GREEN_G32 || tables == GREEN_G32F;
  dim3 g1((d.nk + 127) / 128, d.nf);
  if (tables == GREEN_G32F && d.coef32 && d.nlayer <= COEF32_MAX_LAYERS) {
    const long long nl = (long long)d.nf * d.nk * d.nlayer;
    green_kap32_kernel<<<unsigned((nl + 255) / 256), 256, 0, s>>>(d);
    green_rec32_kernel<<<g1, 128, 0, s>>>(d);
  } else {
    const long long nl = (long long)d.nf * d.nk * d.nlayer;
    green_layer_kernel<<<unsigned((nl + 255) / 256), 256, 0, s>>>(d, fast32 ? 0 : 1);
    green_recursion_kernel<<<g1, 128, 0, s>>>(d);
  }
  if (fast32) {
    green_eval32_kernel<<<unsigned((long long)d.nf * d.nk), 256, 0, s>>>(d);
  } else {
    Dev e = d;
    if (!(tables & (GREEN_G32 | GREEN_G32DF))) e.g32 = nullptr;
    if (!(tables & GREEN_G32DF)) e.g32lo = nullptr;
    if (!(tables & GREEN_G64)) e.g64 = nullptr;
    dim3 g2((d.nk + 31) / 32, d.nf);
    green_eval64_kernel<<<g2, EV_WARPS * 32, 0, s>>>(e);
  }
  return cudaGetLastError();
}

}  // namespace edt
