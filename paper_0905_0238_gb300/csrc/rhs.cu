// Right-hand sides of the split systems (eq. Split), gathered from the transformed data.
//
// For row (f, p) of midpoint index m, q = (p - m) mod N, the paired row of -k_m is (q, p):
//   d_+ = (D2(p,q) + D2(q,p)) / 2,     d_- = (D2(p,q) - D2(q,p)) / (2 i).
// A folded row (weight 2) also stands for its reciprocal partner (-q, -p), whose kernel
// row is identical (g depends on |k| only); its data enter as the mean of the two rows,
// which leaves the normal equations unchanged.  Finally the complex prefactor of the
// kernel is moved onto the data: rows are built as |s_f| g_p g_q and the data are rotated
// by conj(s_f)/|s_f| (a unit-modulus row scaling, which leaves the least-squares problem
// unchanged).  X holds D2(p, q) at X[f - f0][q][p] for the current chunk of frequencies.
#include "edt_internal.h"
#include "cplx.cuh"

namespace edt {

namespace {

template <typename T>
__global__ void rhs_kernel(Dev d, int f0, int f1) {
  using T2 = cplx_t<T>;
  const int m = blockIdx.y;
  const long long* mo = d.row_off_mf + size_t(m) * (d.nf + 1);
  const long long r0 = mo[f0], nr = mo[f1] - r0;            // this chunk's rows of subproblem m
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  const int N = d.N, msk = N - 1;
  const uint32_t row = d.rows[r0 + i];
  const int f = row_f(row), p = row_p(row);
  const int q = (p - m) & msk;
  const T2* X = reinterpret_cast<const T2*>(d.X) + size_t(f - f0) * N * N;   // chunk-local plane
  T2 a = X[size_t(q) * N + p];           // D2(p, q)
  T2 b = X[size_t(p) * N + q];           // D2(q, p)
  if (row_w2(row)) {
    const int np = (-p) & msk, nq = (-q) & msk;
    T2 a2 = X[size_t(np) * N + nq];      // D2(-q, -p)
    T2 b2 = X[size_t(nq) * N + np];      // D2(-p, -q)
    a = cmk(T(0.5) * (a.x + a2.x), T(0.5) * (a.y + a2.y));
    b = cmk(T(0.5) * (b.x + b2.x), T(0.5) * (b.y + b2.y));
  }
  T2 dp = cmk(T(0.5) * (a.x + b.x), T(0.5) * (a.y + b.y));
  T2 dm = cmk(T(0.5) * (a.y - b.y), T(-0.5) * (a.x - b.x));
  const FreqConst fc = d.fc[f];
  T2 rot = cmk(T(fc.rot_re), T(fc.rot_im));
  T2* out = reinterpret_cast<T2*>(d.rhs) + 2 * size_t(r0 + i);
  const T2 rp = dp * rot, rm = dm * rot;
  out[0] = rp;
  out[1] = rm;
}

// Operand metadata of the tensor-core Gram: the FP32 table rows g(|k_p|), g(|k_q|) of each
// row (table row indices) and sqrt of its weight (weight-2 rows enter the Gram scaled by
// sqrt 2).
__global__ void gent_static_kernel(Dev d) {
  const int m = blockIdx.y;
  const long long r0 = d.row_off[m], nr = d.row_off[m + 1] - r0;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  const int N = d.N;
  const uint32_t row = d.rows[r0 + i];
  const int f = row_f(row), p = row_p(row), q = (p - m) & (N - 1);
  const int np = p <= N / 2 ? p : N - p, nq = q <= N / 2 ? q : N - q;
  GramRow g;
  g.rp = unsigned(size_t(f) * d.nk + np);
  g.rq = unsigned(size_t(f) * d.nk + nq);
  g.bp = (unsigned long long)g.rp * d.nzs * sizeof(float2);
  g.bq = (unsigned long long)g.rq * d.nzs * sizeof(float2);
  g.sw = row_w2(row) ? 1.41421356237309515f : 1.0f;
  g.pad = 0.f;
  d.gent[r0 + i] = g;
}

}  // namespace

cudaError_t launch_gent_static(const Dev& d, cudaStream_t s) {
  dim3 g(unsigned((d.rows_max_sub + 255) / 256), d.nsub);
  gent_static_kernel<<<g, 256, 0, s>>>(d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rhs(const Dev& d, int f0, int nfc, cudaStream_t s) {
  // a subproblem has at most nfc * N rows at these frequencies
  dim3 g(unsigned((nfc * (long long)d.N + 255) / 256), d.nsub);
  rhs_kernel<T><<<g, 256, 0, s>>>(d, f0, f0 + nfc);
  return cudaGetLastError();
}
template cudaError_t launch_rhs<float>(const Dev&, int, int, cudaStream_t);
template cudaError_t launch_rhs<double>(const Dev&, int, int, cudaStream_t);

}  // namespace edt
