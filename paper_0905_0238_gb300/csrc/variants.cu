// The paper's solver variants (Section "Numerical Examples") on the FP64 path.
//
//  * Vertical-wavenumber disk: the unknowns of midpoint wavenumber k_m are restricted to the
//    depth vectors whose vertical wavenumber k_z satisfies k_m^2 + k_z^2 <= K^2,
//    K = factor omega_max / c0.  With the orthonormal real basis P (constant, cos and sin of
//    2 pi l j / nz for l = 1, 2, ..., and (-1)^j for even nz, in that order) the kept columns are
//    a leading block P_p, and the restricted normal equations are
//        G' = P_p^T G P_p,   b' = P_p^T b,   x = P_p x'.
//  * Truncated SVD: with Ahat^T Ahat = W Lambda W^T (Lambda = S^2 for the singular values S of
//    Ahat, W its right singular vectors) the solution V S~^-1 U^T dhat is
//        x = sum over lambda_j >= sigma^2 of w_j (w_j^T Ahat^T dhat) / lambda_j,
//    computed from the eigenpairs of the FP64 normal matrix by cyclic two-sided Jacobi rotations
//    in parallel (round-robin) order, matrix and eigenvectors in shared memory.
#include "edt_internal.h"

namespace edt {

namespace {

// T[m] = G[m] P_p (nz x p), one thread per element
__global__ void kzv_t_kernel(Dev d) {
  const int m = blockIdx.y;
  const int n = d.nz, p = d.kz_p[m];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * p) return;
  const int i = e / p, c = e - i * p;
  const double* G = d.G + size_t(m) * n * n + size_t(i) * n;
  double s = 0.0;
  for (int k = 0; k < n; ++k) s = fma(G[k], d.kz_P[size_t(k) * n + c], s);
  d.kz_T[size_t(m) * n * n + size_t(i) * p + c] = s;
}

// G'[m] = P_p^T T[m] (p x p) and b'[m] = P_p^T b[m] (p x 2)
__global__ void kzv_g_kernel(Dev d) {
  const int m = blockIdx.y;
  const int n = d.nz, p = d.kz_p[m];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < p * p) {
    const int a = e / p, c = e - a * p;
    const double* T = d.kz_T + size_t(m) * n * n;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fma(d.kz_P[size_t(i) * n + a], T[size_t(i) * p + c], s);
    d.kz_G[size_t(m) * n * n + size_t(a) * p + c] = s;
  } else if (e < p * p + 2 * p) {
    const int a = (e - p * p) >> 1, side = (e - p * p) & 1;
    const double* b = d.b + size_t(m) * n * 2;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fma(d.kz_P[size_t(i) * n + a], b[i * 2 + side], s);
    d.kz_b[(size_t(m) * n + a) * 2 + side] = s;
  }
}

// x[m] = P_p x'[m] (nz x 2)
__global__ void kzv_back_kernel(Dev d) {
  const int m = blockIdx.y;
  const int n = d.nz, p = d.kz_p[m];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * n) return;
  const int i = e >> 1, side = e & 1;
  double s = 0.0;
  for (int a = 0; a < p; ++a) s = fma(d.kz_P[size_t(i) * n + a], d.kz_x[(size_t(m) * n + a) * 2 + side], s);
  d.x[(size_t(m) * n + i) * 2 + side] = s;
}

constexpr int JAC_THREADS = 256;
constexpr int JAC_MAX_SWEEPS = 20;

// One CTA per subproblem: eigen-decomposition of the p x p normal matrix (G, or G' of the disk)
// by cyclic Jacobi, then the truncated-SVD solution for both right-hand sides.
// src: matrices at m * nz * nz with leading dimension p; rhs, out: [m][nz][2].
__global__ void __launch_bounds__(JAC_THREADS) tsvd_jacobi_kernel(Dev d, const double* src, const double* rhs,
                                                                 double* out) {
  extern __shared__ __align__(16) double sm[];
  const int m = blockIdx.x;
  const int n = d.nz;
  const int p = d.kz_p ? d.kz_p[m] : n;
  const int ld = p + 1;
  double* A = sm;                         // [p][ld]
  double* W = A + size_t(p) * ld;         // [p][ld] eigenvectors (columns)
  double* cs = W + size_t(p) * ld;        // [2][p/2 + 1] rotation cosines and sines
  double* red = cs + 2 * (p / 2 + 1);     // [32]
  int* pj = reinterpret_cast<int*>(red + 32);   // [2][p/2 + 1] pair indices (i < j), -1: none;
                                                // then the sweep's rotation flag
  const bool has_rows = d.row_off[m + 1] > d.row_off[m];
  double* xo = out + size_t(m) * n * 2;
  if (!has_rows || p == 0) {
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) xo[i] = 0.0;
    if (threadIdx.x == 0) d.status[m] = EDT_OK;
    return;
  }
  const double* S = src + size_t(m) * n * n;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e - i * p;
    A[i * ld + j] = S[size_t(i) * p + j];
    W[i * ld + j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  const int P2 = (p + 1) & ~1;            // players of the round-robin (a dummy when p is odd)
  const int npair = P2 / 2;
  // a pair is rotated while |a_ij| > 1e-14 sqrt(a_ii a_jj) (relative to its own diagonal, which
  // keeps small eigenvalues of the positive semi-definite matrix accurate; well above the FP64
  // rounding of a rotation, so the sweeps end); the sweeps stop when one rotates no pair
  int* rotated = pj + 2 * (p / 2 + 1);
  for (int sweep = 0; sweep < JAC_MAX_SWEEPS; ++sweep) {
    if (threadIdx.x == 0) *rotated = 0;
    __syncthreads();
    for (int r = 0; r < P2 - 1; ++r) {
      // round r: player 0 fixed, the others rotate; pair k = (pos[k], pos[P2 - 1 - k])
      for (int k = threadIdx.x; k < npair; k += blockDim.x) {
        auto pos = [&](int t) { return t == 0 ? 0 : 1 + (t - 1 + r) % (P2 - 1); };
        int a = pos(k), b = pos(P2 - 1 - k);
        if (a > b) { const int t = a; a = b; b = t; }
        double c = 1.0, s = 0.0;
        bool rot = false;
        if (b < p) {
          const double apq = A[a * ld + b];
          const double app = A[a * ld + a], aqq = A[b * ld + b];
          if (fabs(apq) > 1e-14 * sqrt(fabs(app * aqq))) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = fabs(tau) < 1e150 ? (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau))
                                               : 0.5 / tau;
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            rot = true;
          }
        }
        if (rot) *rotated = 1;
        pj[k] = rot ? a : -1; pj[npair + k] = b;
        cs[k] = c; cs[npair + k] = s;
      }
      __syncthreads();
      // A <- A J and W <- W J: columns a, b of every pair (disjoint columns)
      for (int e = threadIdx.x; e < npair * p; e += blockDim.x) {
        const int k = e / p, row = e - k * p;
        const int a = pj[k], b = pj[npair + k];
        if (a < 0) continue;
        const double c = cs[k], s = cs[npair + k];
        const double x = A[row * ld + a], y = A[row * ld + b];
        A[row * ld + a] = c * x - s * y;
        A[row * ld + b] = s * x + c * y;
        const double u = W[row * ld + a], v = W[row * ld + b];
        W[row * ld + a] = c * u - s * v;
        W[row * ld + b] = s * u + c * v;
      }
      __syncthreads();
      // A <- J^T A: rows a, b of every pair (disjoint rows)
      for (int e = threadIdx.x; e < npair * p; e += blockDim.x) {
        const int k = e / p, col = e - k * p;
        const int a = pj[k], b = pj[npair + k];
        if (a < 0) continue;
        const double c = cs[k], s = cs[npair + k];
        const double x = A[a * ld + col], y = A[b * ld + col];
        A[a * ld + col] = c * x - s * y;
        A[b * ld + col] = s * x + c * y;
      }
      __syncthreads();
    }
    if (!*rotated) break;
    __syncthreads();
  }
  // threshold on the eigenvalues lambda = s^2: tol > 0 absolute on s, < 0 relative to s_max,
  // 0: every positive s
  double lmax = 0.0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) lmax = fmax(lmax, A[i * ld + i]);
  for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lmax;
  __syncthreads();
  lmax = 0.0;
  for (int w = 0; w < int(blockDim.x >> 5); ++w) lmax = fmax(lmax, red[w]);
  const double tol = d.tsvd_tol;
  const double thr = tol > 0.0 ? tol * tol : (tol < 0.0 ? tol * tol * lmax : 0.0);
  // z = Lambda~^-1 W^T b (kept eigenvalues only) in the last 2p doubles of A (A's entries are no
  // longer needed once its diagonal is saved), then x' = W z
  const double* bm = rhs + size_t(m) * n * 2;
  double* zv = A + size_t(p) * ld - 2 * p;
  // the eigenvalues go to W's padding column W[i][p] (ld = p + 1)
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += blockDim.x) W[i * ld + p] = A[i * ld + i];
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * p; e += blockDim.x) {
    const int i = e >> 1, side = e & 1;
    double sacc = 0.0;
    for (int k = 0; k < p; ++k) sacc = fma(W[k * ld + i], bm[k * 2 + side], sacc);
    const double lam = W[i * ld + p];
    zv[e] = (thr > 0.0 ? lam >= thr : lam > 0.0) ? sacc / lam : 0.0;
  }
  __syncthreads();
  bool bad = false;
  for (int e = threadIdx.x; e < 2 * p; e += blockDim.x) {
    const int i = e >> 1, side = e & 1;
    double sacc = 0.0;
    for (int k = 0; k < p; ++k) sacc = fma(W[i * ld + k], zv[k * 2 + side], sacc);
    xo[e] = sacc;
    if (!isfinite(sacc)) bad = true;
  }
  for (int e = 2 * p + threadIdx.x; e < 2 * n; e += blockDim.x) xo[e] = 0.0;
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) d.status[m] = bad ? EDT_ENONFINITE : EDT_OK;
}

}  // namespace

size_t tsvd_smem_bytes(int p) {
  return (2 * size_t(p) * (p + 1) + 2 * size_t(p / 2 + 1) + 32) * sizeof(double) + (2 * size_t(p / 2 + 1) + 1) * sizeof(int);
}

cudaError_t prepare_variants(int nz) {
  if (nz > TSVD_MAX_NZ) return cudaSuccess;
  return cudaFuncSetAttribute(tsvd_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(tsvd_smem_bytes(nz)));
}

cudaError_t launch_solve_variant(const Dev& d, cudaStream_t s) {
  const int n = d.nz;
  if (d.kz_p) {
    // lam = alpha trace(G) of the unrestricted system
    cudaError_t e = launch_trace_diag(d, s);
    if (e != cudaSuccess) return e;
    kzv_t_kernel<<<dim3((n * n + 255) / 256, d.nsub), 256, 0, s>>>(d);
    kzv_g_kernel<<<dim3((n * n + 2 * n + 255) / 256, d.nsub), 256, 0, s>>>(d);
    if (d.solver == EDT_SOLVE_TSVD) {
      tsvd_jacobi_kernel<<<d.nsub, JAC_THREADS, tsvd_smem_bytes(n), s>>>(d, d.kz_G, d.kz_b, d.kz_x);
    } else {
      // damped: per-subproblem Cholesky of G' + lam I (size p(m)) in the projected arrays
      Dev v = d;
      v.G = d.kz_G; v.b = d.kz_b; v.x = d.kz_x; v.dinv = d.kz_T; v.L32 = nullptr; v.dinv32 = nullptr;
      v.sub_n = d.kz_p; v.sub_goff = d.kz_goff; v.sub_voff = d.kz_voff; v.sub_order = nullptr;
      e = launch_chol_var(v, n, s);
      if (e != cudaSuccess) return e;
    }
    kzv_back_kernel<<<dim3((2 * n + 255) / 256, d.nsub), 256, 0, s>>>(d);
  } else {
    tsvd_jacobi_kernel<<<d.nsub, JAC_THREADS, tsvd_smem_bytes(n), s>>>(d, d.G, d.b, d.x);
  }
  return cudaGetLastError();
}

}  // namespace edt
