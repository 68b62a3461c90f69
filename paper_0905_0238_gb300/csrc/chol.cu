// Damped normal-equation solves (G + lam I) x_+- = b_+-, lam = alpha * trace(G): the native
// FP64 factorisation, the per-request blocked factorisation of the streaming batches, and the
// refinement's FP32 correction solves.
//
// Zeroth-order Tikhonov damping is the regularisation the paper's Discussion proposes in
// place of its truncated SVD.
//
// Native FP64 (the FP64 path and chol_df = 2): one block per midpoint wavenumber m (two
// resident per SM, so one problem's serial panel steps overlap another's trailing update on the
// FP64 pipe): blocked right-looking Cholesky with 32-column panels, in place on the L2-resident
// matrix -- the diagonal block factored by one warp in shared memory, the panel by
// row-per-thread triangular solves, the trailing lower triangle by 4x4 FP64 register tiles.
// Then forward and backward substitution for the two right-hand sides with each 32x32 diagonal
// block staged in shared memory and solved by one warp with shuffles, and the off-diagonal
// updates by thread-per-row dot products (forward) or coalesced column sweeps (backward).
//
// Streaming batches (per-request sizes): the blocked factorisation in double-float over many
// launches, every launch covering all active requests (see the blocked-Cholesky section).
//
// A non-positive or non-finite pivot marks the subproblem EDT_ENOTPD and zeroes its solution.
// The solve applied to r - lam x, with r = Ahat^T (dhat - Ahat x) accumulated by the refinement
// kernel, gives one step of iterative refinement on the normal equations.
#include "edt_internal.h"
#include "cplx.cuh"
#include "dfloat.cuh"
#include "blksolve.cuh"

namespace edt {

namespace {

constexpr int NB = 32, LDP = NB + 1;

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int(blockDim.x) + 31) / 32; ++w) t += red[w];
    red[32] = t;
  }
  __syncthreads();
  t = red[32];
  __syncthreads();
  return t;
}

// Solve L L^T x = sb in place (two right-hand sides, sb[i][0..1]); L lower in A (ld n).
__device__ void chol_solve_2rhs(const double* A, const double* dinv, int n, double* sb,
                                double (*sL)[LDP]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nblk = (n + NB - 1) / NB;
  // forward: L y = b
  for (int bk = 0; bk < nblk; ++bk) {
    const int k0 = bk * NB, kb = min(NB, n - k0);
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
      const int i = e / kb, j = e - i * kb;
      sL[i][j] = j <= i ? A[size_t(k0 + i) * n + k0 + j] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      double v0 = lane < kb ? sb[(k0 + lane) * 2] : 0.0, v1 = lane < kb ? sb[(k0 + lane) * 2 + 1] : 0.0;
      for (int j = 0; j < kb; ++j) {
        const double ij = dinv[k0 + j];
        const double y0 = __shfl_sync(0xffffffffu, v0, j) * ij;
        const double y1 = __shfl_sync(0xffffffffu, v1, j) * ij;
        if (lane == j) { v0 = y0; v1 = y1; }
        if (lane > j && lane < kb) { v0 -= sL[lane][j] * y0; v1 -= sL[lane][j] * y1; }
      }
      if (lane < kb) { sb[(k0 + lane) * 2] = v0; sb[(k0 + lane) * 2 + 1] = v1; }
    }
    __syncthreads();
    for (int i = k0 + kb + threadIdx.x; i < n; i += blockDim.x) {   // b_i -= L[i][blk] . y
      double s0 = sb[i * 2], s1 = sb[i * 2 + 1];
      const double* Ai = A + size_t(i) * n + k0;
      for (int l = 0; l < kb; ++l) {
        const double a = Ai[l];
        s0 -= a * sb[(k0 + l) * 2];
        s1 -= a * sb[(k0 + l) * 2 + 1];
      }
      sb[i * 2] = s0; sb[i * 2 + 1] = s1;
    }
    __syncthreads();
  }
  // backward: L^T x = y
  for (int bk = nblk - 1; bk >= 0; --bk) {
    const int k0 = bk * NB, kb = min(NB, n - k0);
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
      const int i = e / kb, j = e - i * kb;
      sL[i][j] = j <= i ? A[size_t(k0 + i) * n + k0 + j] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      double v0 = lane < kb ? sb[(k0 + lane) * 2] : 0.0, v1 = lane < kb ? sb[(k0 + lane) * 2 + 1] : 0.0;
      for (int j = kb - 1; j >= 0; --j) {
        const double ij = dinv[k0 + j];
        const double x0 = __shfl_sync(0xffffffffu, v0, j) * ij;
        const double x1 = __shfl_sync(0xffffffffu, v1, j) * ij;
        if (lane == j) { v0 = x0; v1 = x1; }
        if (lane < j) { v0 -= sL[j][lane] * x0; v1 -= sL[j][lane] * x1; }
      }
      if (lane < kb) { sb[(k0 + lane) * 2] = v0; sb[(k0 + lane) * 2 + 1] = v1; }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k0; i += blockDim.x) {   // y_i -= sum_l L[k0+l][i] x_l
      double s0 = sb[i * 2], s1 = sb[i * 2 + 1];
      for (int l = 0; l < kb; ++l) {
        const double a = A[size_t(k0 + l) * n + i];
        s0 -= a * sb[(k0 + l) * 2];
        s1 -= a * sb[(k0 + l) * 2 + 1];
      }
      sb[i * 2] = s0; sb[i * 2 + 1] = s1;
    }
    __syncthreads();
  }
}

// trace_mode 0: trace from the diagonal of G; 1: from d.trace (accumulated by the producer).
// VAR = true: every subproblem m has its own size sub_n[m], its matrices at element offset
// sub_goff[m] of G (and L32) and its vectors at sub_voff[m] (streaming batches).
template <bool VAR>
__global__ void __launch_bounds__(256) chol_kernel(Dev d, int trace_mode) {
  extern __shared__ __align__(16) double sm[];
  const int m = VAR && d.sub_order ? d.sub_order[blockIdx.x] : blockIdx.x;
  const int n = VAR ? d.sub_n[m] : d.nz;
  const size_t go = VAR ? size_t(d.sub_goff[m]) : size_t(m) * n * n;
  const size_t vo = VAR ? size_t(d.sub_voff[m]) : size_t(m) * n;
  double* sP = sm;                          // [n][LDP] panel
  double* sD = sP + size_t(n) * LDP;        // [NB][LDP] diagonal block
  double* sb = sD + NB * LDP;               // [n][2] right-hand sides
  double* red = sb + 2 * n;                 // [33] reduction scratch
  __shared__ int fail;
  __shared__ double sInv[NB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* A = d.G + go;
  const long long nr = d.row_off[m + 1] - d.row_off[m];
  double* xo = d.x + vo * 2;
  if (threadIdx.x == 0) fail = 0;
  if (nr == 0) {
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) xo[i] = 0.0;
    if (threadIdx.x == 0) { d.status[m] = EDT_OK; d.trace[m] = 0.0; }
    return;
  }
  double tr;
  if (trace_mode == 0) {
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += A[size_t(i) * n + i];
    tr = block_sum(t, red);
  } else {
    tr = d.trace[m];
  }
  const double lam = d.alpha * tr;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    A[size_t(i) * n + i] += lam;
    sb[2 * i + 0] = d.b[(vo + i) * 2 + 0];
    sb[2 * i + 1] = d.b[(vo + i) * 2 + 1];
  }
  if (threadIdx.x == 0) d.trace[m] = lam;     // from here on the slot holds lam
  __syncthreads();

  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
      int i = e / kb, j = e - i * kb;
      if (j <= i) sD[i * LDP + j] = A[size_t(k0 + i) * n + k0 + j];
    }
    __syncthreads();
    if (warp == 0) {
      for (int j = 0; j < kb; ++j) {
        const double djj = sD[j * LDP + j];
        if (!(djj > 0.0) || !isfinite(djj)) { if (lane == 0) fail = 1; break; }
        const double inv = rsqrt(djj);          // 1 / L_jj; multiplications replace divisions
        __syncwarp();
        if (lane == j) { sD[j * LDP + j] = djj * inv; sInv[j] = inv; }
        if (lane > j && lane < kb) sD[lane * LDP + j] *= inv;
        __syncwarp();
        if (lane > j && lane < kb) {
          const double lij = sD[lane * LDP + j];
          for (int l = j + 1; l <= lane; ++l) sD[lane * LDP + l] -= lij * sD[l * LDP + j];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (fail) break;
    // the FP32 copy of the factor (refinement's correction solves) is written as each part
    // of L is final; its upper triangle is never read
    float* L32 = d.L32 ? d.L32 + go : nullptr;
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
      int i = e / kb, j = e - i * kb;
      if (j <= i) {
        A[size_t(k0 + i) * n + k0 + j] = sD[i * LDP + j];
        if (L32) L32[size_t(k0 + i) * n + k0 + j] = float(sD[i * LDP + j]);
      }
    }
    for (int j = threadIdx.x; j < kb; j += blockDim.x) {
      d.dinv[vo + k0 + j] = sInv[j];
      if (L32) d.dinv32[vo + k0 + j] = float(sInv[j]);
    }
    const int t0 = k0 + kb, t = n - t0;
    // panel: row i of the block column solves x L_kk^T = a
    for (int i = threadIdx.x; i < t; i += blockDim.x) {
      double x[NB];
      double* Ai = A + size_t(t0 + i) * n + k0;
#pragma unroll
      for (int j = 0; j < NB; ++j) x[j] = j < kb ? Ai[j] : 0.0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j < kb) {
          double s = x[j];
#pragma unroll
          for (int l = 0; l < j; ++l) s -= x[l] * sD[j * LDP + l];
          x[j] = s * sInv[j];
        }
      }
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (j < kb) { Ai[j] = x[j]; sP[i * LDP + j] = x[j]; }
      if (L32) {
        float* Li = L32 + size_t(t0 + i) * n + k0;
#pragma unroll
        for (int j = 0; j < NB; ++j)
          if (j < kb) Li[j] = float(x[j]);
      }
    }
    __syncthreads();
    // trailing lower triangle: A[i][j] -= sum_l P[i][l] P[j][l], 4x4 tiles
    const int nbt = (t + 3) / 4;
    const int npair = nbt * (nbt + 1) / 2;
    for (int pt = threadIdx.x; pt < npair; pt += blockDim.x) {
      int bi = int((sqrtf(8.0f * pt + 1.0f) - 1.0f) * 0.5f);
      while (bi * (bi + 1) / 2 > pt) --bi;
      while ((bi + 1) * (bi + 2) / 2 <= pt) ++bi;
      const int bj = pt - bi * (bi + 1) / 2;
      double acc[4][4] = {};
      for (int l = 0; l < kb; ++l) {
        double pi[4], pj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int ii = bi * 4 + u, jj = bj * 4 + u;
          pi[u] = ii < t ? sP[ii * LDP + l] : 0.0;
          pj[u] = jj < t ? sP[jj * LDP + l] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fma(pi[u], pj[v], acc[u][v]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int ii = bi * 4 + u, jj = bj * 4 + v;
          if (ii < t && jj <= ii) A[size_t(t0 + ii) * n + t0 + jj] -= acc[u][v];
        }
    }
    __syncthreads();
  }
  if (fail) {
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) xo[i] = 0.0;
    if (threadIdx.x == 0) d.status[m] = EDT_ENOTPD;
    return;
  }
  chol_solve_2rhs(A, d.dinv + vo, n, sb, reinterpret_cast<double (*)[LDP]>(sD));
  bool bad = false;
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) {
    xo[i] = sb[i];
    if (!isfinite(sb[i])) bad = true;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) d.status[m] = bad ? EDT_ENONFINITE : EDT_OK;
}

// Solve L L^T y = sb in FP32 with the rounded factor (the refinement's correction: the
// residual r - lam x carries the FP64 information, the correction only needs the factor to
// a few digits; cond(G + lam I) * 2^-24 bounds its relative error).  Same blocking as the
// FP64 solve.
__device__ void chol_solve32_2rhs(const float* A, const float* dinv, int n, float* sb, float (*sL)[LDP]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nblk = (n + NB - 1) / NB;
  for (int bk = 0; bk < nblk; ++bk) {
    const int k0 = bk * NB, kb = min(NB, n - k0);
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
      const int i = e / kb, j = e - i * kb;
      sL[i][j] = j <= i ? A[size_t(k0 + i) * n + k0 + j] : 0.f;
    }
    __syncthreads();
    if (warp == 0) {
      float v0 = lane < kb ? sb[(k0 + lane) * 2] : 0.f, v1 = lane < kb ? sb[(k0 + lane) * 2 + 1] : 0.f;
      for (int j = 0; j < kb; ++j) {
        const float ij = dinv[k0 + j];
        const float y0 = __shfl_sync(0xffffffffu, v0, j) * ij;
        const float y1 = __shfl_sync(0xffffffffu, v1, j) * ij;
        if (lane == j) { v0 = y0; v1 = y1; }
        if (lane > j && lane < kb) { v0 = fmaf(-sL[lane][j], y0, v0); v1 = fmaf(-sL[lane][j], y1, v1); }
      }
      if (lane < kb) { sb[(k0 + lane) * 2] = v0; sb[(k0 + lane) * 2 + 1] = v1; }
    }
    __syncthreads();
    for (int i = k0 + kb + threadIdx.x; i < n; i += blockDim.x) {
      float s0 = sb[i * 2], s1 = sb[i * 2 + 1];
      const float* Ai = A + size_t(i) * n + k0;
      for (int l = 0; l < kb; ++l) {
        const float a = Ai[l];
        s0 = fmaf(-a, sb[(k0 + l) * 2], s0);
        s1 = fmaf(-a, sb[(k0 + l) * 2 + 1], s1);
      }
      sb[i * 2] = s0; sb[i * 2 + 1] = s1;
    }
    __syncthreads();
  }
  for (int bk = nblk - 1; bk >= 0; --bk) {
    const int k0 = bk * NB, kb = min(NB, n - k0);
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
      const int i = e / kb, j = e - i * kb;
      sL[i][j] = j <= i ? A[size_t(k0 + i) * n + k0 + j] : 0.f;
    }
    __syncthreads();
    if (warp == 0) {
      float v0 = lane < kb ? sb[(k0 + lane) * 2] : 0.f, v1 = lane < kb ? sb[(k0 + lane) * 2 + 1] : 0.f;
      for (int j = kb - 1; j >= 0; --j) {
        const float ij = dinv[k0 + j];
        const float x0 = __shfl_sync(0xffffffffu, v0, j) * ij;
        const float x1 = __shfl_sync(0xffffffffu, v1, j) * ij;
        if (lane == j) { v0 = x0; v1 = x1; }
        if (lane < j) { v0 = fmaf(-sL[j][lane], x0, v0); v1 = fmaf(-sL[j][lane], x1, v1); }
      }
      if (lane < kb) { sb[(k0 + lane) * 2] = v0; sb[(k0 + lane) * 2 + 1] = v1; }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k0; i += blockDim.x) {
      float s0 = sb[i * 2], s1 = sb[i * 2 + 1];
      for (int l = 0; l < kb; ++l) {
        const float a = A[size_t(k0 + l) * n + i];
        s0 = fmaf(-a, sb[(k0 + l) * 2], s0);
        s1 = fmaf(-a, sb[(k0 + l) * 2 + 1], s1);
      }
      sb[i * 2] = s0; sb[i * 2 + 1] = s1;
    }
    __syncthreads();
  }
}

// Refinement update with the FP32 factor: x += (LL^T)^-1 (r - lam x); r - lam x in FP64,
// rounded to FP32 for the solve, the correction added to x in FP64.
template <bool VAR>
__global__ void __launch_bounds__(256) chol_refine32_kernel(Dev d) {
  extern __shared__ __align__(16) float sb32[];
  __shared__ float sL[NB][LDP];
  const int m = blockIdx.x;
  const int n = VAR ? d.sub_n[m] : d.nz;
  const size_t go = VAR ? size_t(d.sub_goff[m]) : size_t(m) * n * n;
  const size_t vo = VAR ? size_t(d.sub_voff[m]) : size_t(m) * n;
  double* xo = d.x + vo * 2;
  if (d.row_off[m + 1] == d.row_off[m] || d.status[m] != EDT_OK) {
    if (d.status[m] != EDT_OK)
      for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) xo[i] = 0.0;
    return;
  }
  const double lam = d.trace[m];
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x)
    sb32[i] = float(d.r[vo * 2 + i] - lam * xo[i]);
  __syncthreads();
  chol_solve32_2rhs(d.L32 + go, d.dinv32 + vo, n, sb32, sL);
  bool bad = false;
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) {
    const double v = xo[i] + double(sb32[i]);
    xo[i] = v;
    if (!isfinite(v)) bad = true;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0 && bad) d.status[m] = EDT_ENONFINITE;
}

// The same refinement update after a double-float factorisation, whose FP32 copy also holds
// each diagonal block's inverse in the block's strict upper triangle: coalesced block
// substitutions (see blk_solve_2rhs).
template <bool VAR>
__global__ void __launch_bounds__(256) chol_refine32x_kernel(Dev d) {
  extern __shared__ __align__(16) float sbx[];    // [2 n] right-hand sides, scratch
  const int m = blockIdx.x;
  const int n = VAR ? d.sub_n[m] : d.nz;
  const size_t go = VAR ? size_t(d.sub_goff[m]) : size_t(m) * n * n;
  const size_t vo = VAR ? size_t(d.sub_voff[m]) : size_t(m) * n;
  double* xo = d.x + vo * 2;
  if (d.row_off[m + 1] == d.row_off[m] || d.status[m] != EDT_OK) {
    if (d.status[m] != EDT_OK)
      for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) xo[i] = 0.0;
    return;
  }
  const double lam = d.trace[m];
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x)
    sbx[i] = float(d.r[vo * 2 + i] - lam * xo[i]);
  __syncthreads();
  blk_solve_2rhs<F32Arith, 256>(d.L32 + go, d.dinv32 + vo, n, sbx, sbx + 2 * n);
  bool bad = false;
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) {
    const double v = xo[i] + double(sbx[i]);
    xo[i] = v;
    if (!isfinite(v)) bad = true;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0 && bad) d.status[m] = EDT_ENONFINITE;
}

// mode 0: x = (LL^T)^-1 b; mode 1 (refinement): x += (LL^T)^-1 (r - lam x).
template <bool VAR>
__global__ void __launch_bounds__(256) chol_solve_kernel(Dev d, int mode) {
  extern __shared__ __align__(16) double sb[];
  __shared__ double sL[NB][LDP];
  const int m = blockIdx.x;
  const int n = VAR ? d.sub_n[m] : d.nz;
  const size_t go = VAR ? size_t(d.sub_goff[m]) : size_t(m) * n * n;
  const size_t vo = VAR ? size_t(d.sub_voff[m]) : size_t(m) * n;
  double* xo = d.x + vo * 2;
  const bool has_rows = d.row_off[m + 1] > d.row_off[m];
  if (!has_rows || d.status[m] != EDT_OK) {
    if (mode == 0 || d.status[m] != EDT_OK)
      for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) xo[i] = 0.0;
    return;
  }
  const double lam = d.trace[m];
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x)
    sb[i] = mode == 0 ? d.b[vo * 2 + i] : d.r[vo * 2 + i] - lam * xo[i];
  __syncthreads();
  chol_solve_2rhs(d.G + go, d.dinv + vo, n, sb, sL);
  bool bad = false;
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) {
    const double v = mode == 0 ? sb[i] : xo[i] + sb[i];
    xo[i] = v;
    if (!isfinite(v)) bad = true;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0 && bad) d.status[m] = EDT_ENONFINITE;
}

// ------------------------------------------------------------------ blocked Cholesky, several
// launches per factorisation: step k (columns k0 = 32 k .. k0 + 31) is one panel launch (one CTA
// per active subproblem: the diagonal block factored and inverted, the panel rows multiplied by
// the inverse) and one update launch over 64 x 64 tiles of every active subproblem's trailing
// lower triangle, so a large factorisation spreads over many SMs instead of running on one.
// The matrix is held in double-float (float2 (hi, lo) per entry, in the 8 bytes an FP64 entry
// would take) and every step computes in double-float on the FP32 pipes: about 48 significant
// bits against FP64's 53, at a small fraction of the cost on a part whose FP64 rate is 1/64 of
// its FP32 rate.  The conversions FP64 <-> double-float run on the FP64 unit too, so the matrix
// is converted once, by its producer, not on every access.
constexpr int UT = 64;

template <bool VAR>
__device__ __forceinline__ void sub_geom(const Dev& d, int m, int& n, size_t& go, size_t& vo) {
  n = VAR ? d.sub_n[m] : d.nz;
  go = VAR ? size_t(d.sub_goff[m]) : size_t(m) * n * n;
  vo = VAR ? size_t(d.sub_voff[m]) : size_t(m) * n;
}

// Step 0 of every active subproblem: lam = alpha * trace added to the diagonal, then the first
// diagonal block (later diagonal blocks are factored by the previous step's update launch).
// trace_mode 0: trace from the diagonal of G; 1: from trace[m] (the producer's trace).
template <bool VAR>
__global__ void __launch_bounds__(256) cb_diag0_kernel(Dev d, const int* act, int trace_mode) {
  __shared__ DfDiagScratch sh;
  __shared__ double red[40];
  const int m = act[blockIdx.x];
  int n;
  size_t go, vo;
  sub_geom<VAR>(d, m, n, go, vo);
  if (d.status[m] != EDT_OK) return;
  float2* A = reinterpret_cast<float2*>(d.G) + go;
  double tr;
  if (trace_mode == 0) {
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += df_val(A[size_t(i) * n + i]);
    tr = block_sum(t, red);
  } else {
    tr = d.trace[m];
  }
  const double lam = d.alpha * tr;
  const float2 lamf = df_of(lam);
  for (int i = threadIdx.x; i < n; i += blockDim.x) A[size_t(i) * n + i] = df_add(A[size_t(i) * n + i], lamf);
  __syncthreads();
  if (threadIdx.x == 0) d.trace[m] = lam;
  df_diag_block(A, d.L32 ? d.L32 + go : nullptr, d.dinv + vo, d.dinv32 + vo, d.status + m, n, 0, sh);
}

// Panel rows of step k0: one CTA per 32-row chunk of an active subproblem's rows below the
// diagonal block (cpre: prefix sums of the chunk counts over the active list).  x = a X^T,
// x_j = sum_{l <= j} a_l X_jl, all outputs independent: the chunk sits transposed in shared
// memory (rows read and written coalesced), warp h computes the outputs j = h + 8 q of the 32
// rows (lane = row), X is read by broadcast.
template <bool VAR>
__global__ void __launch_bounds__(256) cb_prow_kernel(Dev d, int k0, const int* act, const long long* cpre,
                                                      int nact) {
  __shared__ float2 sA[NB * LDP], sX[NB * LDP];   // sA: [l][row]; sX: [j][l]
  int lo = 0, hi = nact - 1;
  const long long t = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cpre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const int m = act[lo];
  int n;
  size_t go, vo;
  sub_geom<VAR>(d, m, n, go, vo);
  if (d.status[m] != EDT_OK) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int kb = min(NB, n - k0);
  const int r0 = k0 + kb + NB * int(t - cpre[lo]), nr = min(NB, n - r0);
  const float2* Ac = reinterpret_cast<const float2*>(d.G) + go;
  float2* A = reinterpret_cast<float2*>(d.G) + go;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = warp + 8 * q;                    // a warp: one row's 32 columns (coalesced)
    sA[lane * LDP + r] = r < nr && lane < kb ? Ac[size_t(r0 + r) * n + k0 + lane] : make_float2(0.f, 0.f);
    // X_{r, lane}: below the diagonal from the upper triangle (at (lane, r)), the diagonal
    // from dinv
    sX[r * LDP + lane] = r < kb && lane < r ? Ac[size_t(k0 + lane) * n + k0 + r]
                         : (r < kb && lane == r ? df_of(d.dinv[vo + k0 + r]) : make_float2(0.f, 0.f));
  }
  __syncthreads();
  float2 out[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = warp + 8 * q;
    float2 acc = make_float2(0.f, 0.f);
    for (int l = 0; l <= j; ++l) df_acc(acc, sA[l * LDP + lane], sX[j * LDP + l]);
    out[q] = df_norm(acc);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) sA[(warp + 8 * q) * LDP + lane] = out[q];
  __syncthreads();
  float* L32 = d.L32 ? d.L32 + go : nullptr;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = warp + 8 * q;
    if (r < nr && lane < kb) {
      const float2 v = sA[lane * LDP + r];
      A[size_t(r0 + r) * n + k0 + lane] = v;
      if (L32) L32[size_t(r0 + r) * n + k0 + lane] = v.x;
    }
  }
}

// One 64 x 64 tile (bi, bj <= bi) of the trailing lower triangle: C -= P_bi P_bj^T, the
// 32-term dot products accumulated in double-float.  Thread (ty, tx) owns rows ty + 16 u and
// columns tx + 16 v (u, v < 4): interleaved, so the shared panel reads are conflict-free and
// the global rows coalesced.  The CTA of tile (0, 0), whose rows and columns hold the next
// step's diagonal block, factors that block after its own update (no other tile writes it).
constexpr int ULD = UT + 1;
union UpdateSmem {
  struct { float2 I[NB * ULD], J[NB * ULD]; } p;  // transposed panel rows: [l][i]
  DfDiagScratch dg;
};
template <bool VAR>
__global__ void __launch_bounds__(256) cb_update_df_kernel(Dev d, int k0, const int* act,
                                                           const long long* tpre, int nact) {
  __shared__ UpdateSmem sm;
  float2* sI = sm.p.I;
  float2* sJ = sm.p.J;
  // CTAs 0 .. nt0 - 1 take the tiles (0, 0) of the nt0 subproblems that have tiles (the active
  // list is ordered by size, so those come first), so that the diagonal-block factorisations
  // they carry start with the launch; the other tiles follow, subproblem by subproblem.
  int lo = 0, hi = nact;
  while (lo < hi) {                                // nt0: the first subproblem without tiles
    const int mid = (lo + hi) >> 1;
    if (tpre[mid + 1] > tpre[mid]) lo = mid + 1; else hi = mid;
  }
  const int nt0 = lo;
  const long long t = blockIdx.x;
  int e;
  if (t < nt0) {
    lo = int(t);
    e = 0;
  } else {
    const long long u = t - nt0;                   // among the tiles after each first one
    lo = 0;
    hi = nt0 - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tpre[mid] - mid <= u) lo = mid; else hi = mid - 1;
    }
    e = int(u - (tpre[lo] - lo)) + 1;
  }
  const int m = act[lo];
  int n;
  size_t go, vo;
  sub_geom<VAR>(d, m, n, go, vo);
  if (d.status[m] != EDT_OK) return;
  const int kb = min(NB, n - k0), t0 = k0 + kb;
  int bi = int((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
  while (bi * (bi + 1) / 2 > e) --bi;
  while ((bi + 1) * (bi + 2) / 2 <= e) ++bi;
  const int bj = e - bi * (bi + 1) / 2;
  const int r0 = t0 + bi * UT, c0 = t0 + bj * UT;
  float2* A = reinterpret_cast<float2*>(d.G) + go;
  {
    constexpr int NL = UT * NB / 256;               // 8 elements of each panel per thread
    float2 vi[NL], vj[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int x = threadIdx.x + 256 * q, i = x / NB, l = x - i * NB;   // a warp: one row's 32 columns
      vi[q] = r0 + i < n && l < kb ? A[size_t(r0 + i) * n + k0 + l] : make_float2(0.f, 0.f);
      vj[q] = c0 + i < n && l < kb ? A[size_t(c0 + i) * n + k0 + l] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int x = threadIdx.x + 256 * q, i = x / NB, l = x - i * NB;
      sI[l * ULD + i] = vi[q];
      sJ[l * ULD + i] = vj[q];
    }
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool diag = bi == bj;
  float2 acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = make_float2(0.f, 0.f);
  for (int l = 0; l < kb; ++l) {
    float2 pi[4], pj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { pi[u] = sI[l * ULD + ty + 16 * u]; pj[u] = sJ[l * ULD + tx + 16 * u]; }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (r0 + ty + 16 * u < n)                                 // rows past n: nothing to update
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (!(diag && u < v)) df_acc(acc[u][v], pi[u], pj[v]);   // above the diagonal: unused
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int row = r0 + ty + 16 * u, col = c0 + tx + 16 * v;
      if (row < n && col <= row && !(diag && u < v)) {
        float2* c = A + size_t(row) * n + col;
        *c = df_add(*c, df_neg(df_norm(acc[u][v])));
      }
    }
  if (bi == 0) {                                   // the same in every thread of the CTA
    __syncthreads();                               // the tile's writes visible, panels released
    df_diag_block(A, d.L32 ? d.L32 + go : nullptr, d.dinv + vo, d.dinv32 + vo, d.status + m, n, t0, sm.dg);
  }
}

// x = (LL^T)^-1 b in double-float after the blocked factorisation (the inverse diagonal
// blocks in the upper triangles; see blk_solve_2rhs); b and x FP64.
template <bool VAR>
__global__ void __launch_bounds__(256) chol_solve_df_kernel(Dev d) {
  extern __shared__ __align__(16) float2 sbd[];   // [2 n] right-hand sides, [n] 1 / L_ii, scratch
  const int m = blockIdx.x;
  int n;
  size_t go, vo;
  sub_geom<VAR>(d, m, n, go, vo);
  double* xo = d.x + vo * 2;
  if (d.row_off[m + 1] == d.row_off[m] || d.status[m] != EDT_OK) {
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) xo[i] = 0.0;
    return;
  }
  float2* sInv = sbd + 2 * n;
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) sbd[i] = df_of(d.b[vo * 2 + i]);
  for (int i = threadIdx.x; i < n; i += blockDim.x) sInv[i] = df_of(d.dinv[vo + i]);
  __syncthreads();
  blk_solve_2rhs<DfArith, 256>(reinterpret_cast<const float2*>(d.G) + go, sInv, n, sbd, sInv + n);
  bool bad = false;
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) {
    const double v = df_val(sbd[i]);
    xo[i] = v;
    if (!isfinite(v)) bad = true;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0 && bad) d.status[m] = EDT_ENONFINITE;
}

__global__ void trace_diag_kernel(Dev d) {
  __shared__ double red[40];
  const int m = blockIdx.x, n = d.nz;
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += d.G[size_t(m) * n * n + size_t(i) * n + i];
  t = block_sum(t, red);
  if (threadIdx.x == 0) d.trace[m] = t;
}

}  // namespace

cudaError_t launch_trace_diag(const Dev& d, cudaStream_t s) {
  trace_diag_kernel<<<d.nsub, 256, 0, s>>>(d);
  return cudaGetLastError();
}

int chol_launches(int nz) { return 1; }

static size_t chol_smem(int nz) { return (size_t(nz) * LDP + NB * LDP + 2 * nz + 40) * sizeof(double); }

cudaError_t prepare_chol(const Dev& d) {
  cudaError_t e = cudaFuncSetAttribute(chol_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(chol_smem(d.nz)));
  if (e != cudaSuccess) return e;
  return prepare_chol_dfloat(d);
}

cudaError_t launch_chol_solve(const Dev& d, int trace_mode, cudaStream_t s, const CholLookahead* la) {
  if (d.chol_df) return launch_chol_dfloat(d, trace_mode, s, la);
  chol_kernel<false><<<d.nsub, 256, chol_smem(d.nz), s>>>(d, trace_mode);
  return cudaGetLastError();
}

cudaError_t launch_chol_resolve(const Dev& d, cudaStream_t s) {
  if (d.chol_df) return launch_chol_dfloat_resolve(d, s);
  chol_solve_kernel<false><<<d.nsub, 256, size_t(2 * d.nz) * sizeof(double), s>>>(d, 0);
  return cudaGetLastError();
}

cudaError_t launch_refine_update(const Dev& d, cudaStream_t s) {
  if (d.L32 && d.chol_df)
    chol_refine32x_kernel<false><<<d.nsub, 256, size_t(2 * d.nz + blk_solve_scratch<F32Arith, 256>()) * sizeof(float),
                                   s>>>(d);
  else if (d.L32) chol_refine32_kernel<false><<<d.nsub, 256, size_t(2 * d.nz) * sizeof(float), s>>>(d);
  else chol_solve_kernel<false><<<d.nsub, 256, size_t(2 * d.nz) * sizeof(double), s>>>(d, 1);
  return cudaGetLastError();
}

// Streaming batches: subproblem m has size sub_n[m] <= nmax; lam = trace[m] (trace_mode 1
// with alpha = 1: the caller accumulates alpha * trace).
cudaError_t prepare_chol_var(int nmax) {
  return cudaFuncSetAttribute(chol_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(chol_smem(nmax)));
}

int chol_block_cols() { return NB; }

cudaError_t launch_chol_var(const Dev& d, int nmax, cudaStream_t s) {
  chol_kernel<true><<<d.nsub, 256, chol_smem(nmax), s>>>(d, 1);
  return cudaGetLastError();
}

// Blocked form: a step-0 diagonal launch, then per step a panel-row launch and an update
// launch (which also factors the next diagonal blocks), then the solves; d.G holds double-float
// entries (a float2 in each 8-byte slot) and the solution is FP64.  act + k * nsub lists the
// subproblems active at step k (n > 32 k, rows > 0), nact[k] of them; tpre + k * (nsub + 1) the
// prefix sums of their trailing tile counts (ntile[k] tiles in the update launch), cpre the
// same for their 32-row panel chunks (nchunk[k] in the panel-row launch).
template <bool VAR>
static cudaError_t blocked(const Dev& d, int nmax, int nstep, const int* act, const int* nact,
                           const long long* tpre, const long long* ntile, const long long* cpre,
                           const long long* nchunk, int trace_mode, cudaStream_t s) {
  if (nstep > 0 && nact[0] > 0) cb_diag0_kernel<VAR><<<nact[0], 256, 0, s>>>(d, act, trace_mode);
  for (int k = 0; k < nstep; ++k) {
    if (nact[k] == 0) continue;
    if (nchunk[k] > 0)
      cb_prow_kernel<VAR><<<unsigned(nchunk[k]), 256, 0, s>>>(d, k * NB, act + size_t(k) * d.nsub,
                                                              cpre + size_t(k) * (d.nsub + 1), nact[k]);
    if (ntile[k] > 0)
      cb_update_df_kernel<VAR><<<unsigned(ntile[k]), 256, 0, s>>>(d, k * NB, act + size_t(k) * d.nsub,
                                                                  tpre + size_t(k) * (d.nsub + 1), nact[k]);
  }
  chol_solve_df_kernel<VAR><<<d.nsub, 256, size_t(3 * nmax + blk_solve_scratch<DfArith, 256>()) * sizeof(float2),
                              s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_chol_blocked(const Dev& d, bool var, int nmax, int nstep, const int* act_dev,
                                const int* nact_host, const long long* tpre_dev,
                                const long long* ntile_host, const long long* cpre_dev,
                                const long long* nchunk_host, int trace_mode, cudaStream_t s) {
  return var ? blocked<true>(d, nmax, nstep, act_dev, nact_host, tpre_dev, ntile_host, cpre_dev, nchunk_host,
                             trace_mode, s)
             : blocked<false>(d, nmax, nstep, act_dev, nact_host, tpre_dev, ntile_host, cpre_dev, nchunk_host,
                              trace_mode, s);
}

int chol_blocked_tiles(int n, int k0) {
  const int t0 = k0 + (n - k0 < NB ? n - k0 : NB);
  const int T = (n - t0 + UT - 1) / UT;
  return T > 0 ? T * (T + 1) / 2 : 0;
}

int chol_blocked_chunks(int n, int k0) {
  const int t0 = k0 + (n - k0 < NB ? n - k0 : NB);
  return n > t0 ? (n - t0 + NB - 1) / NB : 0;
}

cudaError_t launch_refine_update_var(const Dev& d, int nmax, cudaStream_t s) {
  chol_refine32x_kernel<true><<<d.nsub, 256, size_t(2 * nmax + blk_solve_scratch<F32Arith, 256>()) * sizeof(float),
                                s>>>(d);
  return cudaGetLastError();
}

}  // namespace edt
