// Misfit gradients of the line geometry: J = ||F(c0) V - D||^2 of the Born operator (every
// row; the modelling operator has no evanescent cut) and its gradients with respect to the
// model V(x, z) and to the layer velocities c_l of the reference.
//
// Everything is evaluated in the (p, q) spectral domain.  The data transform D -> D2 is N
// times a unitary map in each of its two lateral axes, so with c_J = 1/N^2
//   J = c_J sum_f sum_{p,q} |R2_f(p, q)|^2,   R2 = s_f sum_j g_p g_q Vhat(p - q) - D2
// (eqs. DMV and M read forward, g_n = g(k_n, z_j; omega~_f), Vhat(k_m, z_j) = sum_x V e^{-i k_m x}).
// Differentiating:
//   dJ/dV(x, z_j)  = 2 c_J Re sum_m Ahat(m, j) e^{+i k_m x},
//                    Ahat(m, j) = sum_{f,p} conj(s_f g_p g_{p-m}) R2(p, p - m)      (adjoint Born)
//   dJ/dg_f(n, j)  = 2 c_J s_f [S1(n, j) + S2(n, j)],
//                    S1(n) = sum_q conj(R2(n, q)) g_q Vhat(n - q),
//                    S2(n) = sum_p conj(R2(p, n)) g_p Vhat(p - n)
//                          = sum_m conj(R2^T(n, n - m)) g_{n-m} conj(Vhat(m))  (V real),
// folded onto the table index |n'| (g depends on k only through k^2), then
//   dJ/dc_l = Re sum_{f,k,j} gbar_f(k, j) dg_f(k, j)/dc_l
// by reverse-mode differentiation of the reflectivity recursion of the depth march (the
// march is recomputed here, not stored by the forward pass).
//
// The FP32 table of the mixed path holds sqrt|s_f| g, so s_f g_p g_q = ph_f g32_p g32_q with
// ph_f = s_f/|s_f|, and dJ/dg = sqrt|s_f| dJ/dg32 -> the factor 2 c_J ph_f sqrt|s_f| below.
//
// Kernels per chunk of frequency planes (X holds D2, then R2 in place):
//   grad_residual  (p, q) tiles of 64 x 64, 4 x 4 per thread, depth in chunks of 32 in
//                  shared memory: R2 and the partial sums of |R2|^2;
//   grad_vhat      (m, j) outputs, 8 consecutive m per thread and one j per lane; the
//                  thread walks p, so its 8 legs q = p - m slide by one per step and stay
//                  in registers: Ahat accumulated across frequencies in FP64;
//   grad_gbar      (n, j) outputs, 8 consecutive n per thread walking m (legs q = n - m
//                  slide the same way): S1 and S2 together (the same legs and Vhat) into
//                  the gbar buffer;
// then once, in FP64: grad_march (per (f, k): the recursion forward), grad_field (per
// (f, k, layer): the field's depths of that layer, reversed), grad_reverse (per (f, k): the
// two recursions reversed, then the per-layer sums); the inverse lateral DFT of Ahat and a
// finalize kernel.
#include "edt_internal.h"
#include "cplx.cuh"

#include <algorithm>

namespace edt {

namespace {

__device__ __forceinline__ int tab_index(int n, int N) { return n <= (N >> 1) ? n : N - n; }

// 1 / b with one real division (the depth march's denominators are O(1e-4 .. 1e1))
__device__ __forceinline__ double2 crcp(double2 b) {
  const double r = 1.0 / (b.x * b.x + b.y * b.y);
  return cmk(b.x * r, -b.y * r);
}

// acc += a * b (complex)
__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cmac_conj(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

__global__ void grad_zero_kernel(Dev d) {
  const size_t n = size_t(d.N) * d.nz;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    d.adj[i] = make_double2(0.0, 0.0);
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i <= d.nlayer; i += blockDim.x) d.gacc[i] = 0.0;
}

// ---- residual R2 = ph_f sum_j g32_p g32_q Vhat(p - q) - D2, and sum |R2|^2 ------------------
constexpr int RT = 64, RJC = 32, RTM = 2 * RT - 1;
constexpr size_t RES_SMEM = (size_t(2) * RJC * (RT + 1) + size_t(RJC) * (RTM + 2)) * sizeof(float2);

__global__ void __launch_bounds__(256, 3) grad_residual_kernel(Dev d, int f0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 (*gp)[RT + 1] = reinterpret_cast<float2 (*)[RT + 1]>(smem_raw);
  float2 (*gq)[RT + 1] = reinterpret_cast<float2 (*)[RT + 1]>(smem_raw + size_t(RJC) * (RT + 1) * sizeof(float2));
  float2 (*vh)[RTM + 2] = reinterpret_cast<float2 (*)[RTM + 2]>(smem_raw + size_t(2) * RJC * (RT + 1) * sizeof(float2));
  __shared__ double red[8];
  const int N = d.N, fi = blockIdx.z, f = f0 + fi;
  const int p0 = blockIdx.x * RT, q0 = blockIdx.y * RT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const float2* g = d.g32 + size_t(f) * d.nk * d.nzs;
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
  for (int j0 = 0; j0 < d.nz; j0 += RJC) {
    for (int e = threadIdx.x; e < RT * RJC; e += blockDim.x) {
      const int i = e / RJC, jj = e - i * RJC, j = j0 + jj;
      const bool in = j < d.nz;
      gp[jj][i] = in ? g[size_t(tab_index(p0 + i, N)) * d.nzs + j] : make_float2(0.f, 0.f);
      gq[jj][i] = in ? g[size_t(tab_index(q0 + i, N)) * d.nzs + j] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < RTM * RJC; e += blockDim.x) {
      const int i = e / RJC, jj = e - i * RJC, j = j0 + jj;
      const int m = (p0 - q0 - (RT - 1) + i) & (N - 1);
      const double2 v = j < d.nz ? d.vfull[size_t(m) * d.nz + j] : make_double2(0.0, 0.0);
      vh[jj][i] = make_float2(float(v.x), float(v.y));
    }
    __syncthreads();
#pragma unroll 2
    for (int jj = 0; jj < RJC; ++jj) {
      float2 ga[4], gb[4], v[7];
#pragma unroll
      for (int a = 0; a < 4; ++a) ga[a] = gp[jj][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) gb[b] = gq[jj][ty + 16 * b];
      // p - q = tx - ty + 16 (a - b); slot p - q + RT - 1
#pragma unroll
      for (int t = 0; t < 7; ++t) v[t] = vh[jj][tx - ty + 16 * (t - 3) + RT - 1];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cmac(acc[a][b], ga[a] * gb[b], v[a - b + 3]);
    }
    __syncthreads();
  }
  const FreqConst fc = d.fc[f];
  const float2 ph = make_float2(float(fc.rot_re), float(-fc.rot_im));     // s_f / |s_f|
  float2* X = reinterpret_cast<float2*>(d.X) + size_t(fi) * N * N;
  double jp = 0.0;
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const size_t o = size_t(q0 + ty + 16 * b) * N + p0 + tx + 16 * a;   // X[q][p] = D2(p, q)
      const float2 r = ph * acc[a][b] - X[o];
      X[o] = r;
      jp += double(r.x) * r.x + double(r.y) * r.y;
    }
  const double t = block_sum(jp, red);
  if (threadIdx.x == 0) atomicAdd(d.gacc, t);
}

// ---- Ahat(m, j) += conj(ph_f) sum_p conj(g32_p g32_{p-m}) R2(p, p - m) -----------------------
constexpr int VM = 64, VPC = 32, VQR = VPC + VM - 1, VLT = VQR + 2;   // VLT odd
constexpr size_t VHAT_SMEM = (size_t(VPC) * 33 + size_t(VQR) * 33 + size_t(VPC) * VLT + 1) * sizeof(float2);
static_assert(VLT % 2 == 1, "odd row length: each step's 8 residuals start 16-byte aligned");

__global__ void __launch_bounds__(256, 3) grad_vhat_kernel(Dev d, int f0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 (*gps)[33] = reinterpret_cast<float2 (*)[33]>(smem_raw);
  float2 (*gqs)[33] = reinterpret_cast<float2 (*)[33]>(smem_raw + size_t(VPC) * 33 * sizeof(float2));
  // residual tile transposed, rsT[pl * VLT + qi] = R2(p0 + pl, q(qi)): at step pl a thread's 8
  // legs are the run qi = pl - 8w + 56 .. pl - 8w + 63, whose start pl (VLT + 1) - 8w + 56 is
  // even, so the run is read with four 16-byte broadcast loads
  constexpr size_t RS_OFF = (size_t(VPC + VQR) * 33 + 1) & ~size_t(1);   // even: 16-byte aligned
  float2* rsT = reinterpret_cast<float2*>(smem_raw + RS_OFF * sizeof(float2));
  const int N = d.N, fi = blockIdx.z, f = f0 + fi;
  const int m0 = blockIdx.x * VM, j0 = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = j0 + lane;
  const float2* g = d.g32 + size_t(f) * d.nk * d.nzs;
  const float2* X = reinterpret_cast<const float2*>(d.X) + size_t(fi) * N * N;
  float2 acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = make_float2(0.f, 0.f);
  for (int p0 = 0; p0 < N; p0 += VPC) {
    // rows qi <-> q = p0 - m0 - (VM - 1) + qi (mod N)
    for (int e = threadIdx.x; e < VQR * 32; e += blockDim.x) {
      const int qi = e >> 5, jl = e & 31, jj = j0 + jl;
      const int q = (p0 - m0 - (VM - 1) + qi) & (N - 1);
      gqs[qi][jl] = jj < d.nz ? g[size_t(tab_index(q, N)) * d.nzs + jj] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < VPC * 32; e += blockDim.x) {
      const int pl = e >> 5, jl = e & 31, jj = j0 + jl;
      gps[pl][jl] = jj < d.nz ? g[size_t(tab_index(p0 + pl, N)) * d.nzs + jj] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < VQR * VPC; e += blockDim.x) {
      const int qi = e / VPC, pl = e - qi * VPC;
      const int q = (p0 - m0 - (VM - 1) + qi) & (N - 1);
      rsT[pl * VLT + qi] = X[size_t(q) * N + p0 + pl];
    }
    __syncthreads();
    // thread's m_k = m0 + 8 w + k; at p = p0 + pl its leg q_k = p - m_k sits in row
    // qi = pl - 8 w - k + VM - 1, one row further per step of p: a sliding window
    float2 win[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) win[k] = gqs[VM - 1 - 8 * w - k][lane];
#pragma unroll
    for (int pl = 0; pl < VPC; ++pl) {
      if (pl > 0) {
#pragma unroll
        for (int k = 7; k > 0; --k) win[k] = win[k - 1];
        win[0] = gqs[pl + VM - 1 - 8 * w][lane];
      }
      const float2 gpv = gps[pl][lane];
      const float4* r4 = reinterpret_cast<const float4*>(rsT + pl * VLT + pl + VM - 8 - 8 * w);
#pragma unroll
      for (int h = 0; h < 4; ++h) {                      // legs k = 7 - 2h (.xy) and 6 - 2h (.zw)
        const float4 rr = r4[h];
        cmac_conj(acc[7 - 2 * h], gpv * win[7 - 2 * h], make_float2(rr.x, rr.y));
        cmac_conj(acc[6 - 2 * h], gpv * win[6 - 2 * h], make_float2(rr.z, rr.w));
      }
    }
    __syncthreads();
  }
  if (j < d.nz) {
    const FreqConst fc = d.fc[f];
    const double2 cph = make_double2(fc.rot_re, fc.rot_im);               // conj(s_f)/|s_f|
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double2 v = cph * make_double2(double(acc[k].x), double(acc[k].y));
      double* o = reinterpret_cast<double*>(d.adj + size_t(m0 + 8 * w + k) * d.nz + j);
      atomicAdd(o, v.x);
      atomicAdd(o + 1, v.y);
    }
  }
}

// ---- S1 + S2 at (n, j): sum_m [conj(R2(n, n - m)) Vhat(m) + conj(R2(n - m, n)) conj(Vhat(m))]
//      g32_{n-m}; gbar_f(n, j) = 2 c_J ph_f sqrt|s_f| (S1 + S2) ----------------------------------
constexpr int GA = 64, GMC = 16, GQR = GA + GMC - 1;
constexpr size_t GBAR_SMEM = (size_t(2) * GMC * GA + size_t(GQR) * 33 + size_t(GMC) * 33) * sizeof(float2);

__global__ void __launch_bounds__(256, 3) grad_gbar_kernel(Dev d, int f0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // bs[2][GMC][GA] first (16-byte aligned rows for the float4 reads): [0] R2(n, q), [1] R2(q, n)
  float2 (*bs)[GMC][GA] = reinterpret_cast<float2 (*)[GMC][GA]>(smem_raw);
  float2 (*gqs)[33] = reinterpret_cast<float2 (*)[33]>(smem_raw + size_t(2) * GMC * GA * sizeof(float2));
  float2 (*ws)[33] = reinterpret_cast<float2 (*)[33]>(smem_raw + (size_t(2) * GMC * GA + size_t(GQR) * 33) * sizeof(float2));
  const int N = d.N, fi = blockIdx.z, f = f0 + fi;
  const int a0 = blockIdx.x * GA, j0 = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = j0 + lane;
  const float2* g = d.g32 + size_t(f) * d.nk * d.nzs;
  const float2* X = reinterpret_cast<const float2*>(d.X) + size_t(fi) * N * N;
  float2 acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = make_float2(0.f, 0.f);
  for (int mc = 0; mc < N; mc += GMC) {
    // rows qi <-> q = a0 - mc - (GMC - 1) + qi (mod N)
    for (int e = threadIdx.x; e < GQR * 32; e += blockDim.x) {
      const int qi = e >> 5, jl = e & 31, jj = j0 + jl;
      const int q = (a0 - mc - (GMC - 1) + qi) & (N - 1);
      gqs[qi][jl] = jj < d.nz ? g[size_t(tab_index(q, N)) * d.nzs + jj] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < GMC * 32; e += blockDim.x) {
      const int mi = e >> 5, jl = e & 31, jj = j0 + jl;
      const double2 v = jj < d.nz ? d.vfull[size_t(mc + mi) * d.nz + jj] : make_double2(0.0, 0.0);
      ws[mi][jl] = make_float2(float(v.x), float(v.y));
    }
    for (int e = threadIdx.x; e < GMC * GA; e += blockDim.x) {
      const int mi = e / GA, al = e - mi * GA;
      const int a = a0 + al, q = (a - mc - mi) & (N - 1);
      bs[0][mi][al] = X[size_t(q) * N + a];           // R2(a, q) = X[q][a]
      bs[1][mi][al] = X[size_t(a) * N + q];           // R2(q, a) = X[a][q]
    }
    __syncthreads();
    // thread's n_k = a0 + 8 w + k; at m = mc + mi its leg q_k = n_k - m sits in row
    // qi = 8 w + k - mi + GMC - 1, one row lower per step of m
    float2 win[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) win[k] = gqs[8 * w + k + GMC - 1][lane];
#pragma unroll
    for (int mi = 0; mi < GMC; ++mi) {
      if (mi > 0) {
#pragma unroll
        for (int k = 7; k > 0; --k) win[k] = win[k - 1];
        win[0] = gqs[8 * w - mi + GMC - 1][lane];
      }
      const float2 wv = ws[mi][lane], wc = make_float2(wv.x, -wv.y);
      const float4* b0 = reinterpret_cast<const float4*>(&bs[0][mi][8 * w]);
      const float4* b1 = reinterpret_cast<const float4*>(&bs[1][mi][8 * w]);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const float4 x0 = b0[h], x1 = b1[h];
        cmac_conj(acc[2 * h], make_float2(x0.x, x0.y), win[2 * h] * wv);
        cmac_conj(acc[2 * h], make_float2(x1.x, x1.y), win[2 * h] * wc);
        cmac_conj(acc[2 * h + 1], make_float2(x0.z, x0.w), win[2 * h + 1] * wv);
        cmac_conj(acc[2 * h + 1], make_float2(x1.z, x1.w), win[2 * h + 1] * wc);
      }
    }
    __syncthreads();
  }
  if (j < d.nz) {
    const FreqConst fc = d.fc[f];
    const double sc = 2.0 / (double(N) * N) * sqrt(fc.s_abs);
    const float2 scale = make_float2(float(sc * fc.rot_re), float(-sc * fc.rot_im));
    float2* G = d.gbar + size_t(f) * N * d.nz;
#pragma unroll
    for (int k = 0; k < 8; ++k) G[size_t(a0 + 8 * w + k) * d.nz + j] = scale * acc[k];
  }
}

// ---- dJ/dc_l: reverse-mode differentiation of the depth march ------------------------------
// Per (f, k), FP64.  Forward (recomputed): kappa_l, rho_l, r_l, A_l as in the march
// (upward: y = kappa_{l+1}(1 - r_{l+1})/(1 + r_{l+1}), rho_l = (kappa_l - y)/(kappa_l + y),
// r_l = rho_l E_l, E_l = e^{2 i kappa_l h_l}; downward: A_0 = i/(2 kappa_0),
// A_{l+1} = A_l F_l, F_l = e^{i kappa_l h_l}(1 + rho_l)/(1 + r_{l+1}); field
// g(z) = A_l (P + rho_l Q), P = e^{i kappa_l d}, Q = e^{i kappa_l (2 h_l - d)}, d = z - t_l).
// Every step is holomorphic in its inputs, so with dJ = Re(gbar dg) each input's cotangent
// is the sum over its uses of (output cotangent) x (complex partial derivative).  Reverse
// order: the field, the downward recursion (l descending), the upward one (l ascending),
// finally d kappa_l/d c_l = -omega~^2/(c_l^3 kappa_l).
constexpr int GS_KAP = 0, GS_RHO = 1, GS_R = 2, GS_A = 3, GS_BKAP = 4, GS_BRHO = 5, GS_BA = 6, GS_BR = 7;
constexpr int GS_SLOTS = 8;

__device__ __forceinline__ double2& gs_at(const Dev& d, int f, int l, int slot, int k) {
  return d.gscr[((size_t(f) * d.nlayer + l) * GS_SLOTS + slot) * d.nk + k];
}

// forward march per (f, k): kappa_l, rho_l, r_l, A_l; the cotangent slots cleared
__global__ void __launch_bounds__(128) grad_march_kernel(Dev d) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (k >= d.nk) return;
  const int J = d.nlayer;
  const double2 one = cmk(1.0, 0.0), zero = cmk(0.0, 0.0);
  const FreqConst fc = d.fc[f];
  const double2 om = cmk(fc.om_re, fc.om_im), om2 = om * om;
  const double kx = 2.0 * M_PI * double(k) / (double(d.N) * d.dx);
  for (int l = 0; l < J; ++l) {
    const double ic2 = 1.0 / (d.layer_vel[l] * d.layer_vel[l]);
    gs_at(d, f, l, GS_KAP, k) = csqrt_upper(cmk(om2.x * ic2 - kx * kx, om2.y * ic2));
    gs_at(d, f, l, GS_BR, k) = zero;
  }
  // upward recursion
  double2 rn = zero, kn = gs_at(d, f, J - 1, GS_KAP, k);
  gs_at(d, f, J - 1, GS_R, k) = zero;
  gs_at(d, f, J - 1, GS_RHO, k) = zero;
  for (int l = J - 2; l >= 0; --l) {
    const double h = d.layer_top[l + 1] - d.layer_top[l];
    const double2 kl = gs_at(d, f, l, GS_KAP, k);
    const double2 y = kn * (one - rn) * crcp(one + rn);
    const double2 rho = (kl - y) * crcp(kl + y);
    const double2 E = cexp(cmk(-2.0 * kl.y * h, 2.0 * kl.x * h));
    gs_at(d, f, l, GS_RHO, k) = rho;
    rn = rho * E;
    gs_at(d, f, l, GS_R, k) = rn;
    kn = kl;
  }
  // downward recursion
  double2 A = cmk(0.0, 0.5) * crcp(gs_at(d, f, 0, GS_KAP, k));
  for (int l = 0; l < J; ++l) {
    gs_at(d, f, l, GS_A, k) = A;
    if (l < J - 1) {
      const double h = d.layer_top[l + 1] - d.layer_top[l];
      const double2 kl = gs_at(d, f, l, GS_KAP, k);
      const double2 e1 = cexp(cmk(-kl.y * h, kl.x * h));
      A = A * e1 * (one + gs_at(d, f, l, GS_RHO, k)) * crcp(one + gs_at(d, f, l + 1, GS_R, k));
    }
  }
}

// field, reversed, per (f, k, l): the depths z_j of layer l (a contiguous index range) give
// A_l, rho_l, kappa_l their cotangents; gbar on the table index |n'| = k (rows n = k and
// N - k).  Within the layer P and Q advance by e^{+-i kappa dz} from a direct start.
// gb64: the cotangent already on the table index in FP64 ([nf][nk][nz]), else d.gbar.
__global__ void __launch_bounds__(128) grad_field_kernel(Dev d, const double2* gb64) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int J = d.nlayer;
  if (gid >= (long long)d.nf * J * d.nk) return;
  const int k = int(gid % d.nk);
  const long long fl = gid / d.nk;
  const int l = int(fl % J), f = int(fl / J);
  // depth range of layer l: first j with z_layer[j] >= l and >= l + 1
  auto lower = [&](int v) {
    int lo = 0, hi = d.nz;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (d.z_layer[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
  };
  const int j0 = lower(l), j1 = lower(l + 1);
  double2 bA = cmk(0.0, 0.0), bRho = bA, bK = bA;
  if (j0 < j1) {
    const int N = d.N;
    const double2 kl = gs_at(d, f, l, GS_KAP, k), Al = gs_at(d, f, l, GS_A, k);
    const bool last = l == J - 1;
    const double h = last ? 0.0 : d.layer_top[l + 1] - d.layer_top[l];
    const double2 rho = last ? cmk(0.0, 0.0) : gs_at(d, f, l, GS_RHO, k);
    const double dz = d.dz;
    const double2 Ef = cexp(cmk(-kl.y * dz, kl.x * dz));          // e^{+i kappa dz}
    const double2 Eb = cexp(cmk(kl.y * dz, -kl.x * dz));          // e^{-i kappa dz}
    double dd = d.z_off[j0];
    double2 P = cexp(cmk(-kl.y * dd, kl.x * dd));
    double2 Q = last ? cmk(0.0, 0.0) : cexp(cmk(-kl.y * (2.0 * h - dd), kl.x * (2.0 * h - dd)));
    const float2* G = d.gbar + size_t(f) * N * d.nz;
    const bool two = k > 0 && k < N / 2;
    for (int j = j0; j < j1; ++j) {
      dd = d.z_off[j];
      double2 gbar;
      if (gb64) {
        gbar = gb64[(size_t(f) * d.nk + k) * d.nz + j];
      } else {
        float2 gb = G[size_t(k) * d.nz + j];
        if (two) gb = gb + G[size_t(N - k) * d.nz + j];
        gbar = cmk(double(gb.x), double(gb.y));
      }
      const double2 gA = gbar * Al;
      if (!last) {
        bA = bA + gbar * (P + rho * Q);
        bRho = bRho + gA * Q;
        bK = bK + gA * cmk(0.0, 1.0) * (dd * P + (2.0 * h - dd) * (rho * Q));
        Q = Q * Eb;
      } else {
        bA = bA + gbar * P;
        bK = bK + gA * cmk(0.0, 1.0) * (dd * P);
      }
      P = P * Ef;
    }
  }
  gs_at(d, f, l, GS_BA, k) = bA;
  gs_at(d, f, l, GS_BRHO, k) = bRho;
  gs_at(d, f, l, GS_BKAP, k) = bK;
}

// the two recursions reversed per (f, k), then dJ/dc_l = Re(kappabar_l dkappa_l/dc_l)
// summed over (f, k): warp sums, one partial per warp and layer (added in warp order by the
// finalize kernel, so the result does not depend on the order the warps ran in)
__global__ void __launch_bounds__(128) grad_reverse_kernel(Dev d) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  const int J = d.nlayer;
  const bool live = k < d.nk;
  const int kk = live ? k : 0;
  const double2 one = cmk(1.0, 0.0);
  const FreqConst fc = d.fc[f];
  const double2 om = cmk(fc.om_re, fc.om_im), om2 = om * om;
  if (live) {
    // downward recursion, reversed: A_{l+1} = A_l F_l
    double2 bA1 = gs_at(d, f, J - 1, GS_BA, kk);
    for (int l = J - 2; l >= 0; --l) {
      const double h = d.layer_top[l + 1] - d.layer_top[l];
      const double2 kl = gs_at(d, f, l, GS_KAP, kk), rho = gs_at(d, f, l, GS_RHO, kk);
      const double2 rn = gs_at(d, f, l + 1, GS_R, kk), Al = gs_at(d, f, l, GS_A, kk);
      const double2 e1 = cexp(cmk(-kl.y * h, kl.x * h));
      const double2 inv1r = crcp(one + rn);
      const double2 F = e1 * (one + rho) * inv1r;
      const double2 bF = bA1 * Al;
      const double2 bA = gs_at(d, f, l, GS_BA, kk) + bA1 * F;
      gs_at(d, f, l, GS_BKAP, kk) = gs_at(d, f, l, GS_BKAP, kk) + bF * F * cmk(0.0, h);
      gs_at(d, f, l, GS_BRHO, kk) = gs_at(d, f, l, GS_BRHO, kk) + bF * e1 * inv1r;
      gs_at(d, f, l + 1, GS_BR, kk) = gs_at(d, f, l + 1, GS_BR, kk) - bF * F * inv1r;
      bA1 = bA;
    }
    {
      const double2 k0 = gs_at(d, f, 0, GS_KAP, kk);
      gs_at(d, f, 0, GS_BKAP, kk) = gs_at(d, f, 0, GS_BKAP, kk) + bA1 * cmk(0.0, -0.5) * crcp(k0 * k0);
    }
    // upward recursion, reversed (l ascending: r_l's cotangent is complete when l is reached)
    for (int l = 0; l <= J - 2; ++l) {
      const double h = d.layer_top[l + 1] - d.layer_top[l];
      const double2 kl = gs_at(d, f, l, GS_KAP, kk), kn = gs_at(d, f, l + 1, GS_KAP, kk);
      const double2 rn = gs_at(d, f, l + 1, GS_R, kk), rho = gs_at(d, f, l, GS_RHO, kk);
      const double2 E = cexp(cmk(-2.0 * kl.y * h, 2.0 * kl.x * h));
      const double2 bR = gs_at(d, f, l, GS_BR, kk);
      const double2 bRho = gs_at(d, f, l, GS_BRHO, kk) + bR * E;
      double2 bK = gs_at(d, f, l, GS_BKAP, kk) + bR * rho * E * cmk(0.0, 2.0 * h);
      const double2 iopr = crcp(one + rn);
      const double2 y = kn * (one - rn) * iopr;
      const double2 sm = kl + y, is2 = crcp(sm * sm);
      bK = bK + bRho * (2.0 * y) * is2;
      const double2 bY = bRho * (-2.0 * kl) * is2;
      gs_at(d, f, l, GS_BKAP, kk) = bK;
      gs_at(d, f, l + 1, GS_BKAP, kk) = gs_at(d, f, l + 1, GS_BKAP, kk) + bY * (one - rn) * iopr;
      gs_at(d, f, l + 1, GS_BR, kk) = gs_at(d, f, l + 1, GS_BR, kk) + bY * kn * (-2.0 * (iopr * iopr));
    }
  }
  for (int l = 0; l < J; ++l) {
    double v = 0.0;
    if (live) {
      const double c = d.layer_vel[l];
      const double2 dk = (-1.0 / (c * c * c)) * om2 * crcp(gs_at(d, f, l, GS_KAP, kk));
      v = (gs_at(d, f, l, GS_BKAP, kk) * dk).x;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const size_t wid = (size_t(blockIdx.y) * gridDim.x + blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if ((threadIdx.x & 31) == 0) d.gcpart[wid * J + l] = v;
  }
}

// nw: the reverse kernel's warps (their partials are added in warp order)
__global__ void grad_finalize_kernel(Dev d, double* J, double* gc, int nw) {
  const double cj = 1.0 / (double(d.N) * d.N);
  if (threadIdx.x == 0 && J) J[0] = cj * d.gacc[0];
  for (int l = threadIdx.x; l < d.nlayer; l += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += d.gcpart[size_t(w) * d.nlayer + l];
    gc[l] = t;
  }
}

// ---- adjoint of the inversion D -> V (linear in D: G and lam depend on the rows only) --------
// V = (1/N) Re sum_m Vhat(m) e^{i k_m x} with Vhat(m) = x_+ + i x_- for m = 0..N/2 and the
// conjugate for -m, so dV/dx_+(m) = (c_m/N) cos(k_m x), dV/dx_-(m) = -(c_m/N) sin(k_m x),
// c_m = 1 at the self-paired m (x_- = 0 there) and 2 otherwise: xbar(m) = (c_m/N) DFT(Vbar)(m).
// xbar goes where the forward solve reads b.
__global__ void adj_xbar_kernel(Dev d) {
  const int m = blockIdx.x, N = d.N;
  const bool self = m == 0 || 2 * m == N;
  const double c = (self ? 1.0 : 2.0) / double(N);
  for (int z = threadIdx.x; z < d.nz; z += blockDim.x) {
    const double2 v = d.vfull[size_t(m) * d.nz + z];
    d.b[(size_t(m) * d.nz + z) * 2 + 0] = c * v.x;
    d.b[(size_t(m) * d.nz + z) * 2 + 1] = self ? 0.0 : c * v.y;
  }
}

// r += xbar: with zero right-hand sides the refinement kernel leaves r = -Ahat^T Ahat y, so
// this makes r - lam y = xbar - (Ahat^T Ahat + lam I) y, the residual of the adjoint solve.
__global__ void adj_addb_kernel(Dev d) {
  const size_t n = size_t(d.nsub) * d.nz * 2;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    d.r[i] += d.b[i];
}

// Per kept row (f, p) of m at frequencies [f0, f1), with bbar = (G + lam I)^-1 xbar in d.x:
// b_+- = sum_rows w Re(conj(row) rhs_+-) gives rhsbar = w sum_z row(z) bbar(z); then the
// rotation rhs = rot d, the split d_+ = (a + c)/2, d_- = (a - c)/(2i) with a = D2(p, q),
// c = D2(q, p) (folded rows: a and c the means with D2(-q, -p), D2(-p, -q)) are reversed and
// scattered (atomically) into the chunk's planes X[fi][q][p] = D2bar(p, q).
__global__ void __launch_bounds__(256) adj_rows_kernel(Dev d, int f0, int f1) {
  __shared__ float2 bb[512];                          // (bbar_+, bbar_-) per depth, nz <= 512
  const int m = blockIdx.y, N = d.N, msk = N - 1;
  if (d.status[m] != EDT_OK) return;
  const double* yb = d.x + size_t(m) * d.nz * 2;
  for (int z = threadIdx.x; z < d.nz; z += blockDim.x) bb[z] = make_float2(float(yb[2 * z]), float(yb[2 * z + 1]));
  __syncthreads();
  const long long r0 = d.row_off_mf[size_t(m) * (d.nf + 1) + f0];
  const long long r1 = d.row_off_mf[size_t(m) * (d.nf + 1) + f1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  float2* X = reinterpret_cast<float2*>(d.X);
  // one warp per row, lanes over depth
  for (long long ri = r0 + (long long)blockIdx.x * nwarp + warp; ri < r1; ri += (long long)gridDim.x * nwarp) {
    const uint32_t row = d.rows[ri];
    const int f = row_f(row), p = row_p(row), q = (p - m) & msk;
    const float2* g1 = d.g32 + (size_t(f) * d.nk + tab_index(p, N)) * d.nzs;
    const float2* g2 = d.g32 + (size_t(f) * d.nk + tab_index(q, N)) * d.nzs;
    float2 sp = make_float2(0.f, 0.f), sm = sp;
    for (int z = lane; z < d.nz; z += 32) {
      const float2 t = g1[z] * g2[z], b2 = bb[z];
      sp.x = fmaf(t.x, b2.x, sp.x); sp.y = fmaf(t.y, b2.x, sp.y);
      sm.x = fmaf(t.x, b2.y, sm.x); sm.y = fmaf(t.y, b2.y, sm.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
      sp.x += __shfl_xor_sync(0xffffffffu, sp.x, o);
      sp.y += __shfl_xor_sync(0xffffffffu, sp.y, o);
      sm.x += __shfl_xor_sync(0xffffffffu, sm.x, o);
      sm.y += __shfl_xor_sync(0xffffffffu, sm.y, o);
    }
    if (lane != 0) continue;
    const bool w2 = row_w2(row);
    const FreqConst fc = d.fc[f];
    const float2 crot = make_float2(float(fc.rot_re), float(-fc.rot_im));   // conj(rot)
    const float w = w2 ? 2.f : 1.f;
    const float2 dp = crot * (w * sp), dm = crot * (w * sm);
    // abar = dp/2 + (i/2) dm, cbar = dp/2 - (i/2) dm; folded rows split each in halves
    const float h = w2 ? 0.25f : 0.5f;
    const float2 abar = make_float2(h * (dp.x - dm.y), h * (dp.y + dm.x));
    const float2 cbar = make_float2(h * (dp.x + dm.y), h * (dp.y - dm.x));
    float2* P = X + size_t(f - f0) * N * N;
    auto add = [&](int pp, int qq, float2 v) {             // D2bar(pp, qq) at X[qq][pp]
      float* o = reinterpret_cast<float*>(P + size_t(qq & msk) * N + (pp & msk));
      atomicAdd(o, v.x);
      atomicAdd(o + 1, v.y);
    };
    add(p, q, abar);
    add(q, p, cbar);
    if (w2) {
      add(-q, -p, abar);
      add(-p, -q, cbar);
    }
  }
}

// ---- dL/dc_l through the damped solve ----------------------------------------------------
// Per subproblem m, x solves (Ahat^T Ahat + lam I) x = Ahat^T dhat with lam = alpha tr(Ahat^T
// Ahat) (the Gram's trace, the sum of w |A|^2 over the rows); the kernel rows A = g32_p g32_q
// (g32 = sqrt|s_f| g; the data carry the unit phase of s_f) depend on the reference.  With
// mu = (Ahat^T Ahat + lam I)^-1 xbar, differentiating the normal equations gives the
// cotangent of a complex row (dL = Re sum_z conj(Abar) dA)
//   Abar = w [ sum_k (u_k mu_k + v_k x_k) + gamma A ],
//   u_k = d_k - A . x_k,  v_k = -A . mu_k,  gamma = -2 alpha sum_k mu_k . x_k,
// (k over the two right-hand sides +-; w = 2 for a folded row).  With dA = sqrt|s_f| (g32_q dg_p
// + g32_p dg_q) the table's cotangent in the convention dL = Re sum gbar dg is
//   gbar(f, |p|) += sqrt|s_f| g32_q conj(Abar),   gbar(f, |q|) += sqrt|s_f| g32_p conj(Abar),
// gathered per table row over the rows that read it (row groups built with the plan, in row
// order: no atomics), FP32 products, FP64 sums; then the depth march is reversed as for the
// misfit gradient.
constexpr int IG_WARPS = 8, IG_RPW = 16;             // 128 rows per CTA of the row products

// Per row the products with the depth vectors of its subproblem: mode 0 (before the adjoint
// solve) u_k = d_k - A . x_k with x the forward solution (Vhat), mode 1 v_k = -A . mu_k with mu
// in x; the first CTA of each subproblem also stores the FP32 vectors and, in mode 1, gamma.
__global__ void __launch_bounds__(IG_WARPS * 32) ig_rowdot_kernel(Dev d, int mode) {
  __shared__ float vs[2][512];
  __shared__ double red[IG_WARPS];
  const int m = blockIdx.y, nz = d.nz, N = d.N, msk = N - 1;
  const bool ok = d.status[m] == EDT_OK;
  const long long r0 = d.row_off[m], nr = d.row_off[m + 1] - r0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double bsum = 0.0;
  for (int z = threadIdx.x; z < nz; z += blockDim.x) {
    float a = 0.f, b = 0.f;
    if (ok) {
      if (mode) {
        const double mp = d.x[(size_t(m) * nz + z) * 2], mm = d.x[(size_t(m) * nz + z) * 2 + 1];
        const double2 xv = d.vhat[size_t(m) * nz + z];
        bsum += mp * xv.x + mm * xv.y;
        a = float(mp); b = float(mm);
      } else {
        const double2 xv = d.vhat[size_t(m) * nz + z];
        a = float(xv.x); b = float(xv.y);
      }
    }
    vs[0][z] = a; vs[1][z] = b;
    if (blockIdx.x == 0) {
      float4* o = d.xmu + size_t(m) * nz + z;
      if (mode) { o->z = a; o->w = b; } else { o->x = a; o->y = b; }
    }
  }
  if (mode && blockIdx.x == 0) {
    for (int o = 16; o > 0; o >>= 1) bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
    if (lane == 0) red[warp] = bsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < IG_WARPS; ++w) t += red[w];
      d.gam[m] = ok ? -2.0 * d.alpha * t : 0.0;
    }
  }
  __syncthreads();
  const long long wb = (long long)blockIdx.x * IG_WARPS * IG_RPW + warp * IG_RPW;
  const long long we = min(nr, wb + IG_RPW);
  const float2* rhs = reinterpret_cast<const float2*>(d.rhs);
  for (long long i = wb; i < we; ++i) {
    const long long ri = r0 + i;
    const uint32_t row = d.rows[ri];
    const int f = row_f(row), p = row_p(row), q = (p - m) & msk;
    const float2* gp = d.g32 + (size_t(f) * d.nk + tab_index(p, N)) * d.nzs;
    const float2* gq = d.g32 + (size_t(f) * d.nk + tab_index(q, N)) * d.nzs;
    float2 sp = make_float2(0.f, 0.f), sm = sp;
    for (int z = lane; z < nz; z += 32) {
      const float2 t = gp[z] * gq[z];
      const float a = vs[0][z], b = vs[1][z];
      sp.x = fmaf(t.x, a, sp.x); sp.y = fmaf(t.y, a, sp.y);
      sm.x = fmaf(t.x, b, sm.x); sm.y = fmaf(t.y, b, sm.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
      sp.x += __shfl_xor_sync(0xffffffffu, sp.x, o); sp.y += __shfl_xor_sync(0xffffffffu, sp.y, o);
      sm.x += __shfl_xor_sync(0xffffffffu, sm.x, o); sm.y += __shfl_xor_sync(0xffffffffu, sm.y, o);
    }
    if (lane == 0) {
      float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
      if (ok) {
        if (mode) {
          o = make_float4(-sp.x, -sp.y, -sm.x, -sm.y);
        } else {
          const float2 dp = rhs[2 * ri], dm = rhs[2 * ri + 1];
          o = make_float4(dp.x - sp.x, dp.y - sp.y, dm.x - sm.x, dm.y - sm.y);
        }
      }
      d.rowc[2 * ri + mode] = o;
    }
  }
}

// One warp per table row (f, n), n = 0 .. N/2, lanes over depth (NZL per lane): gbar of that
// row from every row that reads it, in row order; 32 rows summed in FP32, then into FP64.
template <int NZL>
__global__ void __launch_bounds__(256) ig_gather_kernel(Dev d) {
  const long long te = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (te >= (long long)d.nf * d.nk) return;
  const int lane = threadIdx.x & 31, nz = d.nz, N = d.N, msk = N - 1;
  const int f = int(te / d.nk);
  const float2* gs = d.g32 + size_t(te) * d.nzs;
  float2 self[NZL], part[NZL];
  double2 acc[NZL];
#pragma unroll
  for (int t = 0; t < NZL; ++t) {
    const int z = lane + 32 * t;
    self[t] = z < nz ? gs[z] : make_float2(0.f, 0.f);
    part[t] = make_float2(0.f, 0.f);
    acc[t] = make_double2(0.0, 0.0);
  }
  const long long b0 = d.tref_off[te], b1 = d.tref_off[te + 1];
  for (long long i = b0; i < b1; ++i) {
    const int2 rf = d.tref[i];
    const int m = rf.y >> 1, side = rf.y & 1;
    const uint32_t row = d.rows[rf.x];
    const int p = row_p(row), q = (p - m) & msk;
    const float2* go = d.g32 + (size_t(f) * d.nk + tab_index(side ? p : q, N)) * d.nzs;
    const float4 u = d.rowc[2 * size_t(rf.x)], v = d.rowc[2 * size_t(rf.x) + 1];
    const float w = row_w2(row) ? 2.f : 1.f, gam = float(d.gam[m]);
    const float4* xm = d.xmu + size_t(m) * nz;
#pragma unroll
    for (int t = 0; t < NZL; ++t) {
      const int z = lane + 32 * t;
      if (z < nz) {
        const float2 g2 = go[z];
        const float4 xv = xm[z];                       // (x_+, x_-, mu_+, mu_-)
        const float2 A = self[t] * g2;
        float2 ab;
        ab.x = fmaf(u.x, xv.z, fmaf(u.z, xv.w, fmaf(v.x, xv.x, fmaf(v.z, xv.y, gam * A.x))));
        ab.y = fmaf(u.y, xv.z, fmaf(u.w, xv.w, fmaf(v.y, xv.x, fmaf(v.w, xv.y, gam * A.y))));
        ab.x *= w; ab.y *= w;
        part[t].x = fmaf(g2.x, ab.x, fmaf(g2.y, ab.y, part[t].x));      // g2 conj(ab)
        part[t].y = fmaf(g2.y, ab.x, fmaf(-g2.x, ab.y, part[t].y));
      }
    }
    if (((i - b0) & 31) == 31) {
#pragma unroll
      for (int t = 0; t < NZL; ++t) {
        acc[t].x += double(part[t].x); acc[t].y += double(part[t].y);
        part[t] = make_float2(0.f, 0.f);
      }
    }
  }
  const double sq = sqrt(d.fc[f].s_abs);
  double2* out = d.g64 + size_t(te) * nz;
#pragma unroll
  for (int t = 0; t < NZL; ++t) {
    const int z = lane + 32 * t;
    if (z < nz) out[z] = make_double2(sq * (acc[t].x + double(part[t].x)), sq * (acc[t].y + double(part[t].y)));
  }
}

}  // namespace

// The forward solve with k refinement steps is x = sum_{i<=k} (I - Ht^-1 H)^i Ht^-1 b (Ht the
// factored matrix, H = Ahat^T Ahat + lam I from the rows), a symmetric map: its transpose is
// the same iteration applied to xbar, run here with the forward's own kernels.
cudaError_t launch_invert_vjp(const Dev& d0, const void* Vbar, int Vbar_dtype, void* Dbar, int Dbar_dtype,
                              double* gc, int refine, cudaStream_t s) {
  cudaError_t e;
  // the adjoint solve's refinement residual is xbar - (Ahat^T Ahat + lam I) y: the rows'
  // data term is left out (the right-hand sides stay for later calls)
  Dev d = d0;
  d.refine_nodata = 1;
  const dim3 rg(unsigned((std::max(d.rows_max_sub, 1LL) + IG_WARPS * IG_RPW - 1) / (IG_WARPS * IG_RPW)), d.nsub);
  if (gc) {
    ig_rowdot_kernel<<<rg, IG_WARPS * 32, 0, s>>>(d, 0);          // u = d - A x
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = launch_lateral_dft(d, Vbar, Vbar_dtype, s)) != cudaSuccess) return e;
  adj_xbar_kernel<<<d.nsub, 256, 0, s>>>(d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_chol_resolve(d, s)) != cudaSuccess) return e;
  for (int it = 0; it < refine; ++it) {
    if ((e = launch_refine(d, s)) != cudaSuccess) return e;
    adj_addb_kernel<<<152, 256, 0, s>>>(d);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_refine_update(d, s)) != cudaSuccess) return e;
  }
  if (Dbar) {
    for (int f0 = 0; f0 < d.nf; f0 += d.fchunk) {
      const int nfc = std::min(d.fchunk, d.nf - f0);
      if ((e = cudaMemsetAsync(d.X, 0, size_t(nfc) * d.N * d.N * sizeof(float2), s)) != cudaSuccess) return e;
      adj_rows_kernel<<<dim3(32, d.nsub), 256, 0, s>>>(d, f0, f0 + nfc);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = launch_transform_adjoint(d, Dbar, Dbar_dtype, f0, nfc, s)) != cudaSuccess) return e;
    }
  }
  if (gc) {
    ig_rowdot_kernel<<<rg, IG_WARPS * 32, 0, s>>>(d, 1);          // v = -A mu, gamma
    const unsigned gg = unsigned(((long long)d.nf * d.nk + 7) / 8);
    if (d.nz <= 64) ig_gather_kernel<2><<<gg, 256, 0, s>>>(d);
    else if (d.nz <= 128) ig_gather_kernel<4><<<gg, 256, 0, s>>>(d);
    else if (d.nz <= 256) ig_gather_kernel<8><<<gg, 256, 0, s>>>(d);
    else ig_gather_kernel<16><<<gg, 256, 0, s>>>(d);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    grad_zero_kernel<<<152, 256, 0, s>>>(d);
    const dim3 gk((d.nk + 127) / 128, d.nf);
    grad_march_kernel<<<gk, 128, 0, s>>>(d);
    const long long nfl = (long long)d.nf * d.nlayer * d.nk;
    grad_field_kernel<<<unsigned((nfl + 127) / 128), 128, 0, s>>>(d, d.g64);
    grad_reverse_kernel<<<gk, 128, 0, s>>>(d);
    grad_finalize_kernel<<<1, 64, 0, s>>>(d, nullptr, gc, int(gk.x * gk.y * 4));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t prepare_grad(const Dev&) {
  cudaError_t e = cudaFuncSetAttribute(grad_residual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(RES_SMEM));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(grad_vhat_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(VHAT_SMEM));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(grad_gbar_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(GBAR_SMEM));
}

bool grad_supported(const Dev& d) {
  return d.geom == EDT_GEOM_LINE && d.precision == EDT_MIXED && d.N >= 64 && d.nlayer <= GRAD_MAX_LAYERS &&
         d.gscr != nullptr;
}

// Adjoint Born operator of the line geometry, V = F^T D for <D1, D2> = Re sum conj(D1) D2 and
// <V1, V2> = sum V1 V2: the adjoint of the inverse data transform is T / N^2 (T the data
// transform, N times a unitary map per axis), then Vbar_hat(m, z) = sum_f sum_p
// conj(s_f g(k_p, z) g(k_{p-m}, z)) D2(p, p - m) and V(x, z) = Re sum_m Vbar_hat(m, z) e^{+i k_m x}.
// Mixed path: FP32 transform and the misfit gradient's adjoint-Born contraction (FP64 sums
// across frequencies); FP64 path: FP64 transform and a direct FP64 contraction.
cudaError_t launch_adjoint(const Dev& d, const void* D, int D_dtype, void* V, int V_dtype, cudaStream_t s) {
  cudaError_t e;
  const int N = d.N;
  const double scale = 1.0 / (double(N) * N);
  if (d.precision == EDT_FP64) {
    if ((e = cudaMemsetAsync(d.vfull, 0, sizeof(double2) * size_t(N) * d.nz, s)) != cudaSuccess) return e;
    for (int f0 = 0; f0 < d.nf; f0 += d.fchunk) {
      const int nfc = std::min(d.fchunk, d.nf - f0);
      if ((e = launch_adjoint64_chunk(d, D, D_dtype, f0, nfc, s)) != cudaSuccess) return e;
    }
    return launch_lateral_idft_real(d, d.vfull, scale, V, V_dtype, s);
  }
  grad_zero_kernel<<<152, 256, 0, s>>>(d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int f0 = 0; f0 < d.nf; f0 += d.fchunk) {
    const int nfc = std::min(d.fchunk, d.nf - f0);
    if ((e = launch_transform<float>(d, D, D_dtype, f0, nfc, s)) != cudaSuccess) return e;
    grad_vhat_kernel<<<dim3(N / VM, (d.nz + 31) / 32, nfc), 256, VHAT_SMEM, s>>>(d, f0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return launch_lateral_idft_real(d, d.adj, scale, V, V_dtype, s);
}

cudaError_t launch_misfit_grad(const Dev& d, const void* V, int V_dtype, const void* D, int D_dtype,
                               double* J, void* gV, double* gc, cudaStream_t s) {
  cudaError_t e;
  grad_zero_kernel<<<152, 256, 0, s>>>(d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_lateral_dft(d, V, V_dtype, s)) != cudaSuccess) return e;
  const int N = d.N;
  for (int f0 = 0; f0 < d.nf; f0 += d.fchunk) {
    const int nfc = std::min(d.fchunk, d.nf - f0);
    if ((e = launch_transform<float>(d, D, D_dtype, f0, nfc, s)) != cudaSuccess) return e;
    grad_residual_kernel<<<dim3(N / RT, N / RT, nfc), 256, RES_SMEM, s>>>(d, f0);
    const dim3 gj(N / VM, (d.nz + 31) / 32, nfc);
    grad_vhat_kernel<<<gj, 256, VHAT_SMEM, s>>>(d, f0);
    grad_gbar_kernel<<<gj, 256, GBAR_SMEM, s>>>(d, f0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const dim3 gk((d.nk + 127) / 128, d.nf);
  grad_march_kernel<<<gk, 128, 0, s>>>(d);
  const long long nfl = (long long)d.nf * d.nlayer * d.nk;
  grad_field_kernel<<<unsigned((nfl + 127) / 128), 128, 0, s>>>(d, nullptr);
  grad_reverse_kernel<<<gk, 128, 0, s>>>(d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_lateral_idft_real(d, d.adj, 2.0 / (double(N) * N), gV, V_dtype, s)) != cudaSuccess) return e;
  grad_finalize_kernel<<<1, 64, 0, s>>>(d, J, gc, int(gk.x * gk.y * 4));
  return cudaGetLastError();
}

}  // namespace edt
