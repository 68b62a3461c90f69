// Lateral transforms: the shot/receiver data transform, the inverse transform back to
// (x, z), and the spectral Born forward model.
//
// Data transform (the discrete form of the Fourier transform over midpoint and offset in
// Section "Two dimensions"):  D2(p, q) = sum_is sum_ir D(is, ir) e^{-i k_p x_ir} e^{+i k_q x_is}.
// Pass 1 transforms every receiver line (contiguous rows, sign -), pass 2 every source
// column (stride N, sign +), leaving X[f][q][p] = D2(p, q).  The FP32 path uses register-
// resident warp FFTs (one warp per line); the FP64 path and N < 32 use shared-memory
// radix-4 FFTs.  Twiddles come from a host-computed table.
//
// Inverse transform: Vhat(k_m) for 0 <= m <= N/2 from the split solutions x_+/x_-,
// completed by Vhat(-k_m) = conj Vhat(k_m) (eq. VSym), then
// V(x, z) = (1/N) sum_m Vhat(k_m, z) e^{+i k_m x}, real part.
//
// Forward model (eqs. DMV/M read forward): D2(p, q) = s_f sum_j g(k_p,z_j) g(k_q,z_j)
// Vhat(k_p - k_q, z_j), then the inverse of the data transform.
#include "edt_internal.h"
#include "cplx.cuh"
#include "wfft.cuh"

#include <algorithm>

namespace edt {

namespace {

__device__ __forceinline__ int bitrev(int i, int logn) { return int(__brev(unsigned(i)) >> (32 - logn)); }
// shared-memory index with one pad element per 16: bit-reversed stores and strided
// butterflies then spread over the banks instead of hitting one
__device__ __forceinline__ int pd(int e) { return e + (e >> 4); }
__host__ __device__ __forceinline__ int padded_len(int n) { return n + (n >> 4); }
__host__ __device__ __forceinline__ int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

template <typename T> __device__ __forceinline__ const cplx_t<T>* twid(const Dev& d);
template <> __device__ __forceinline__ const float2* twid<float>(const Dev& d) { return d.tw32; }
template <> __device__ __forceinline__ const double2* twid<double>(const Dev& d) { return d.tw64; }

template <typename T2> __device__ __forceinline__ T2 load_c(const void* p, int dtype, size_t i);
template <> __device__ __forceinline__ float2 load_c<float2>(const void* p, int dtype, size_t i) {
  if (dtype == EDT_C64) return reinterpret_cast<const float2*>(p)[i];
  double2 v = reinterpret_cast<const double2*>(p)[i];
  return make_float2(float(v.x), float(v.y));
}
template <> __device__ __forceinline__ double2 load_c<double2>(const void* p, int dtype, size_t i) {
  if (dtype == EDT_C128) return reinterpret_cast<const double2*>(p)[i];
  float2 v = reinterpret_cast<const float2*>(p)[i];
  return make_double2(double(v.x), double(v.y));
}
template <typename T2> __device__ __forceinline__ void store_c(void* p, int dtype, size_t i, T2 v) {
  if (dtype == EDT_C64) reinterpret_cast<float2*>(p)[i] = make_float2(float(v.x), float(v.y));
  else reinterpret_cast<double2*>(p)[i] = make_double2(double(v.x), double(v.y));
}

// In-place decimation-in-time FFT of `batch` sequences of length N = 2^logn held in
// shared memory in bit-reversed order; sequence b starts at s + b * bstride and element e
// sits at pd(e).  sign = -1 uses e^{-2 pi i k/N}, sign = +1 its conjugate.  One radix-2
// stage when logn is odd, then pairs of radix-2 stages fused into radix-4 butterflies (one
// barrier per pair).  Each thread owns one butterfly position q and walks a share of the
// sequences, so its two twiddles are loaded once per stage and reused across the batch.
template <typename T, typename T2>
__device__ void block_fft(T2* s, int N, int logn, int batch, int bstride, const T2* tw, int sign) {
  int lh = 0;                       // log2 of the current half-size h
  if (logn & 1) {                   // radix-2 stage, h = 1 (twiddle 1)
    const int lq = logn - 1, total = batch << lq;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int b = t >> lq, j = t & ((1 << lq) - 1);
      T2* base = s + b * bstride;
      const int i0 = pd(2 * j), i1 = pd(2 * j + 1);
      const T2 u = base[i0], v = base[i1];
      base[i0] = u + v;
      base[i1] = u - v;
    }
    __syncthreads();
    lh = 1;
  }
  const int nq = N >> 2;                                   // radix-4 butterflies per sequence
  const int ngrp = max(1, int(blockDim.x) / max(nq, 1));   // thread groups over sequences
  for (; lh < logn; lh += 2) {      // fused stages h and 2h
    const int h = 1 << lh;
    for (int t = threadIdx.x; t < nq * ngrp; t += blockDim.x) {
      const int q = t % nq, g = t / nq;
      const int jj = q & (h - 1), blk = q >> lh;    // jj < h, block of 4h
      const int e0 = (blk << (lh + 2)) + jj;
      const int i0 = pd(e0), i1 = pd(e0 + h), i2 = pd(e0 + 2 * h), i3 = pd(e0 + 3 * h);
      T2 w1 = tw[jj << (logn - 1 - lh)];            // W_{2h}^jj
      T2 w2 = tw[jj << (logn - 2 - lh)];            // W_{4h}^jj
      if (sign > 0) { w1.y = -w1.y; w2.y = -w2.y; }
      for (int b = g; b < batch; b += ngrp) {
        T2* base = s + b * bstride;
        const T2 x0 = base[i0], x1 = base[i1] * w1, x2 = base[i2], x3 = base[i3] * w1;
        const T2 y0 = x0 + x1, y1 = x0 - x1, y2 = x2 + x3, y3 = x2 - x3;
        const T2 a = w2 * y2;
        T2 c = w2 * y3;                             // times W_4 = -i (sign -) or +i (sign +)
        c = sign < 0 ? cmk(c.y, -c.x) : cmk(-c.y, c.x);
        base[i0] = y0 + a;
        base[i2] = y0 - a;
        base[i1] = y1 + c;
        base[i3] = y1 - c;
      }
    }
    __syncthreads();
  }
}

// Row FFTs: rows of length N at stride N; each block handles `rpb` consecutive rows.
template <typename T>
__global__ void fft_rows_kernel(Dev d, const void* in, int in_dtype, void* out, int out_dtype,
                                long long nrows, int rpb, int sign, T scale) {
  using T2 = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* s = reinterpret_cast<T2*>(smem_raw);
  const int N = d.N, logn = ilog2(N);
  const long long r0 = (long long)blockIdx.x * rpb;
  const int nr = int(min((long long)rpb, nrows - r0));
  const int ld = padded_len(N);
  for (int e = threadIdx.x; e < nr * N; e += blockDim.x) {
    const int r = e >> logn, i = e & (N - 1);
    s[r * ld + pd(bitrev(i, logn))] = load_c<T2>(in, in_dtype, size_t(r0) * N + e);
  }
  __syncthreads();
  block_fft<T, T2>(s, N, logn, nr, ld, twid<T>(d), sign);
  for (int e = threadIdx.x; e < nr * N; e += blockDim.x) {
    const int r = e >> logn, i = e & (N - 1);
    T2 v = s[r * ld + pd(i)];
    store_c<T2>(out, out_dtype, size_t(r0) * N + e, cmk(v.x * scale, v.y * scale));
  }
}

// Column FFTs of [planes][N][N] (transform along the first index), in place; each block
// takes `cpb` adjacent columns of one plane (a 128-byte row segment).
template <typename T>
__global__ void fft_cols_kernel(Dev d, cplx_t<T>* X, int cpb, int sign, T scale) {
  using T2 = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* s = reinterpret_cast<T2*>(smem_raw);
  const int N = d.N, logn = ilog2(N), ld = padded_len(N) + 1;
  const int c0 = blockIdx.x * cpb;
  T2* P = X + size_t(blockIdx.y) * N * N;
  for (int e = threadIdx.x; e < N * cpb; e += blockDim.x) {
    int r = e / cpb, c = e - r * cpb;
    s[c * ld + pd(bitrev(r, logn))] = P[size_t(r) * N + c0 + c];
  }
  __syncthreads();
  block_fft<T, T2>(s, N, logn, cpb, ld, twid<T>(d), sign);
  for (int e = threadIdx.x; e < N * cpb; e += blockDim.x) {
    int r = e / cpb, c = e - r * cpb;
    T2 v = s[c * ld + pd(r)];
    P[size_t(r) * N + c0 + c] = cmk(v.x * scale, v.y * scale);
  }
}

constexpr int WR_WARPS = 8;   // rows per block in the row kernel

template <int P>
__global__ void __launch_bounds__(WR_WARPS * 32) wfft_rows_kernel(Dev d, const void* in, int in_dtype,
                                                                 float2* out, long long nrows, int sign,
                                                                 float scale) {
  constexpr int N = 32 * P;
  __shared__ float2 sm[WR_WARPS][N + N / 16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long row = (long long)blockIdx.x * WR_WARPS + warp;
  if (row >= nrows) return;
  float2 r[P];
#pragma unroll
  for (int a = 0; a < P; ++a) r[a] = load_c<float2>(in, in_dtype, size_t(row) * N + 32 * a + lane);
  warp_fft<P>(r, d.tw32, N, sign, lane);
  const int brl = rbits(lane, 5) * P;
#pragma unroll
  for (int k1 = 0; k1 < P; ++k1) sm[warp][pd(k1 + brl)] = r[k1];
  __syncwarp();
  float2* o = out + size_t(row) * N;
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const float2 v = sm[warp][pd(32 * j + lane)];
    o[32 * j + lane] = make_float2(v.x * scale, v.y * scale);
  }
}

// Columns of [planes][N][N] in place, WC columns per block, one warp per column.
template <int P, int WC>
__global__ void __launch_bounds__(WC * 32) wfft_cols_kernel(Dev d, float2* X, int sign, float scale) {
  constexpr int N = 32 * P;
  constexpr int LD = N + N / 16 + 1;                         // odd stride: columns on distinct banks
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);        // [WC][LD]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = blockIdx.x * WC;
  float2* Pl = X + size_t(blockIdx.y) * N * N;
  for (int e = threadIdx.x; e < N * WC; e += blockDim.x) {
    const int rr = e / WC, c = e - rr * WC;
    tile[c * LD + pd(rr)] = Pl[size_t(rr) * N + c0 + c];
  }
  __syncthreads();
  float2 r[P];
#pragma unroll
  for (int a = 0; a < P; ++a) r[a] = tile[warp * LD + pd(32 * a + lane)];
  warp_fft<P>(r, d.tw32, N, sign, lane);
  const int brl = rbits(lane, 5) * P;
#pragma unroll
  for (int k1 = 0; k1 < P; ++k1) tile[warp * LD + pd(k1 + brl)] = r[k1];
  __syncthreads();
  for (int e = threadIdx.x; e < N * WC; e += blockDim.x) {
    const int rr = e / WC, c = e - rr * WC;
    const float2 v = tile[c * LD + pd(rr)];
    Pl[size_t(rr) * N + c0 + c] = make_float2(v.x * scale, v.y * scale);
  }
}

template <int P>
cudaError_t wfft_rows_launch(const Dev& d, const void* in, int in_dtype, float2* out, long long nrows,
                             int sign, float scale, cudaStream_t st) {
  const long long nb = (nrows + WR_WARPS - 1) / WR_WARPS;
  wfft_rows_kernel<P><<<unsigned(nb), WR_WARPS * 32, 0, st>>>(d, in, in_dtype, out, nrows, sign, scale);
  return cudaGetLastError();
}

template <int P>
cudaError_t wfft_cols_launch(const Dev& d, float2* X, int planes, int sign, float scale, cudaStream_t st) {
  constexpr int N = 32 * P, WC = P >= 32 ? 8 : 16;
  const size_t smem = size_t(WC) * (N + N / 16 + 1) * sizeof(float2);
  dim3 g(N / WC, planes);
  wfft_cols_kernel<P, WC><<<g, WC * 32, smem, st>>>(d, X, sign, scale);
  return cudaGetLastError();
}

template <int P>
cudaError_t wfft_cols_prepare() {
  constexpr int N = 32 * P, WC = P >= 32 ? 8 : 16;
  const size_t smem = size_t(WC) * (N + N / 16 + 1) * sizeof(float2);
  return cudaFuncSetAttribute(wfft_cols_kernel<P, WC>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

// FP32 row / column transforms for N >= 32 (warp FFT); false if N is outside that range
bool wfft_rows(const Dev& d, const void* in, int in_dtype, float2* out, long long nrows, int sign,
               float scale, cudaStream_t st, cudaError_t* e) {
  switch (d.N) {
    case 32: *e = wfft_rows_launch<1>(d, in, in_dtype, out, nrows, sign, scale, st); return true;
    case 64: *e = wfft_rows_launch<2>(d, in, in_dtype, out, nrows, sign, scale, st); return true;
    case 128: *e = wfft_rows_launch<4>(d, in, in_dtype, out, nrows, sign, scale, st); return true;
    case 256: *e = wfft_rows_launch<8>(d, in, in_dtype, out, nrows, sign, scale, st); return true;
    case 512: *e = wfft_rows_launch<16>(d, in, in_dtype, out, nrows, sign, scale, st); return true;
    case 1024: *e = wfft_rows_launch<32>(d, in, in_dtype, out, nrows, sign, scale, st); return true;
    default: return false;
  }
}
bool wfft_cols(const Dev& d, float2* X, int planes, int sign, float scale, cudaStream_t st, cudaError_t* e) {
  switch (d.N) {
    case 32: *e = wfft_cols_launch<1>(d, X, planes, sign, scale, st); return true;
    case 64: *e = wfft_cols_launch<2>(d, X, planes, sign, scale, st); return true;
    case 128: *e = wfft_cols_launch<4>(d, X, planes, sign, scale, st); return true;
    case 256: *e = wfft_cols_launch<8>(d, X, planes, sign, scale, st); return true;
    case 512: *e = wfft_cols_launch<16>(d, X, planes, sign, scale, st); return true;
    case 1024: *e = wfft_cols_launch<32>(d, X, planes, sign, scale, st); return true;
    default: return false;
  }
}

template <typename T>
cudaError_t rows_fft(const Dev& d, const void* in, int in_dtype, void* out, int out_dtype,
                     long long nrows, int sign, T scale, cudaStream_t st) {
  using T2 = cplx_t<T>;
  int rpb = (int(sizeof(T)) == 4 ? 4096 : 2048) / d.N;
  if (rpb < 1) rpb = 1;
  size_t smem = size_t(rpb) * padded_len(d.N) * sizeof(T2);
  long long nb = (nrows + rpb - 1) / rpb;
  fft_rows_kernel<T><<<unsigned(nb), 256, smem, st>>>(d, in, in_dtype, out, out_dtype, nrows, rpb,
                                                      sign, scale);
  return cudaGetLastError();
}

template <typename T>
cudaError_t cols_fft(const Dev& d, cplx_t<T>* X, int planes, int sign, T scale, cudaStream_t st) {
  using T2 = cplx_t<T>;
  int cpb = 128 / int(sizeof(T2));
  if (cpb > d.N) cpb = d.N;
  size_t smem = size_t(cpb) * (padded_len(d.N) + 1) * sizeof(T2);
  dim3 g(d.N / cpb, planes);
  fft_cols_kernel<T><<<g, 256, smem, st>>>(d, X, cpb, sign, scale);
  return cudaGetLastError();
}

}  // namespace

cudaError_t fft2_f64(const Dev& d, double2* X, int planes, int ny, int sign, double scale, cudaStream_t s) {
  cudaError_t e = rows_fft<double>(d, X, EDT_C128, X, EDT_C128, (long long)planes * ny, sign, scale, s);
  if (e != cudaSuccess || ny == 1) return e;
  return cols_fft<double>(d, X, planes, sign, 1.0, s);
}

namespace {

// ---- inverse transform ------------------------------------------------------------------
constexpr int INV_ZT = 2;   // depths per CTA: 128 CTAs for 256 depths (8 left most SMs idle)

__global__ void inverse_kernel(Dev d, void* V, int V_dtype) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* s = reinterpret_cast<double2*>(smem_raw);
  const int N = d.N, logn = ilog2(N), ld = padded_len(N) + 1, half = N / 2;
  const int z0 = blockIdx.x * INV_ZT;
  const int nzt = min(INV_ZT, d.nz - z0);
  for (int e = threadIdx.x; e < (half + 1) * nzt; e += blockDim.x) {
    int m = e / nzt, t = e - m * nzt;
    int z = z0 + t;
    const double* xm = d.x + (size_t(m) * d.nz + z) * 2;
    double re = xm[0];
    double im = (m == 0 || m == half) ? 0.0 : xm[1];
    if (d.status[m] != EDT_OK) { re = 0.0; im = 0.0; }
    d.vhat[size_t(m) * d.nz + z] = make_double2(re, im);
    s[t * ld + pd(bitrev(m, logn))] = make_double2(re, im);
    if (m > 0 && m < half) s[t * ld + pd(bitrev(N - m, logn))] = make_double2(re, -im);
  }
  __syncthreads();
  block_fft<double, double2>(s, N, logn, nzt, ld, d.tw64, +1);
  const double inv = 1.0 / double(N);
  for (int e = threadIdx.x; e < N * nzt; e += blockDim.x) {
    int xi = e / nzt, t = e - xi * nzt;
    double v = s[t * ld + pd(xi)].x * inv;
    size_t o = size_t(xi) * d.nz + z0 + t;
    if (V_dtype == EDT_F64) reinterpret_cast<double*>(V)[o] = v;
    else reinterpret_cast<float*>(V)[o] = float(v);
  }
}

// ---- forward model -------------------------------------------------------------------------
// Vhat(k_m, z) = sum_x V(x, z) e^{-i k_m x} for all m: one block per z tile.
__global__ void lateral_dft_kernel(Dev d, const void* V, int V_dtype) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* s = reinterpret_cast<double2*>(smem_raw);
  const int N = d.N, logn = ilog2(N), ld = padded_len(N) + 1;
  const int z0 = blockIdx.x * INV_ZT;
  const int nzt = min(INV_ZT, d.nz - z0);
  for (int e = threadIdx.x; e < N * nzt; e += blockDim.x) {
    int xi = e / nzt, t = e - xi * nzt;
    size_t o = size_t(xi) * d.nz + z0 + t;
    double v = V_dtype == EDT_F64 ? reinterpret_cast<const double*>(V)[o]
                                  : double(reinterpret_cast<const float*>(V)[o]);
    s[t * ld + pd(bitrev(xi, logn))] = make_double2(v, 0.0);
  }
  __syncthreads();
  block_fft<double, double2>(s, N, logn, nzt, ld, d.tw64, -1);
  for (int e = threadIdx.x; e < N * nzt; e += blockDim.x) {
    int m = e / nzt, t = e - m * nzt;
    d.vfull[size_t(m) * d.nz + z0 + t] = s[t * ld + pd(m)];
  }
}

// D2[f][q][p] = s_f sum_j g(|p'|, j) g(|q'|, j) Vhat((p - q) mod N, j): 16 x 16 (p, q) tile
// per block, depth in chunks of 32 staged in shared memory.
template <typename T>
__global__ void born_spectral_kernel(Dev d, cplx_t<T>* X, int f0) {
  using T2 = cplx_t<T>;
  constexpr int TP = 16, ZC = 32;
  __shared__ double2 gp[TP][ZC], gq[TP][ZC], vh[2 * TP][ZC];
  const int N = d.N, f = f0 + blockIdx.z;   // X holds the chunk's planes only
  const int p0 = blockIdx.x * TP, q0 = blockIdx.y * TP;
  const int tp = threadIdx.x & (TP - 1), tq = threadIdx.x / TP;
  double2 acc = make_double2(0.0, 0.0);
  const double2* g = d.g64 + size_t(f) * d.nk * d.nz;
  for (int zc = 0; zc < d.nz; zc += ZC) {
    for (int e = threadIdx.x; e < TP * ZC; e += blockDim.x) {
      int i = e / ZC, j = e - i * ZC, z = zc + j;
      int pa = p0 + i, qa = q0 + i;
      int np = pa <= N / 2 ? pa : N - pa, nq = qa <= N / 2 ? qa : N - qa;
      gp[i][j] = z < d.nz ? g[size_t(np) * d.nz + z] : make_double2(0.0, 0.0);
      gq[i][j] = z < d.nz ? g[size_t(nq) * d.nz + z] : make_double2(0.0, 0.0);
    }
    for (int e = threadIdx.x; e < 2 * TP * ZC; e += blockDim.x) {
      int i = e / ZC, j = e - i * ZC, z = zc + j;
      int m = (p0 - q0 - (TP - 1) + i) & (N - 1);     // m = p - q covers [p0-q0-15, p0-q0+15]
      vh[i][j] = z < d.nz ? d.vfull[size_t(m) * d.nz + z] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int mi = tp - tq + (TP - 1);
#pragma unroll 4
    for (int j = 0; j < ZC; ++j) acc = acc + gp[tp][j] * gq[tq][j] * vh[mi][j];
    __syncthreads();
  }
  const FreqConst fc = d.fc[f];
  double2 om = make_double2(fc.om_re, fc.om_im);
  double2 sf = (d.dz / d.dx) * (om * om);
  acc = sf * acc;
  X[size_t(blockIdx.z) * N * N + size_t(q0 + tq) * N + p0 + tp] = cmk(T(acc.x), T(acc.y));
}

// out[x][z] = scale Re sum_m in[m][z] e^{+i k_m x}: one block per z tile, every m given.
__global__ void lateral_idft_kernel(Dev d, const double2* in, double scale, void* out, int out_dtype) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* s = reinterpret_cast<double2*>(smem_raw);
  const int N = d.N, logn = ilog2(N), ld = padded_len(N) + 1;
  const int z0 = blockIdx.x * INV_ZT;
  const int nzt = min(INV_ZT, d.nz - z0);
  for (int e = threadIdx.x; e < N * nzt; e += blockDim.x) {
    const int m = e / nzt, t = e - m * nzt;
    s[t * ld + pd(bitrev(m, logn))] = in[size_t(m) * d.nz + z0 + t];
  }
  __syncthreads();
  block_fft<double, double2>(s, N, logn, nzt, ld, d.tw64, +1);
  for (int e = threadIdx.x; e < N * nzt; e += blockDim.x) {
    const int xi = e / nzt, t = e - xi * nzt;
    const double v = s[t * ld + pd(xi)].x * scale;
    const size_t o = size_t(xi) * d.nz + z0 + t;
    if (out_dtype == EDT_F64) reinterpret_cast<double*>(out)[o] = v;
    else reinterpret_cast<float*>(out)[o] = float(v);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_transform(const Dev& d, const void* D, int D_dtype, int f0, int nfc, cudaStream_t s) {
  using T2 = cplx_t<T>;
  const int out_dtype = sizeof(T) == 4 ? EDT_C64 : EDT_C128;
  const size_t esz = D_dtype == EDT_C64 ? sizeof(float2) : sizeof(double2);
  const void* Dc = static_cast<const char*>(D) + size_t(f0) * d.N * d.N * esz;
  const long long nrows = (long long)nfc * d.N;
  cudaError_t e = cudaSuccess;
  if (sizeof(T) == 4 && wfft_rows(d, Dc, D_dtype, reinterpret_cast<float2*>(d.X), nrows, -1, 1.f, s, &e)) {
    if (e != cudaSuccess) return e;
    wfft_cols(d, reinterpret_cast<float2*>(d.X), nfc, +1, 1.f, s, &e);
    return e;
  }
  e = rows_fft<T>(d, Dc, D_dtype, d.X, out_dtype, nrows, -1, T(1), s);
  if (e != cudaSuccess) return e;
  return cols_fft<T>(d, reinterpret_cast<T2*>(d.X), nfc, +1, T(1), s);
}
template cudaError_t launch_transform<float>(const Dev&, const void*, int, int, int, cudaStream_t);
template cudaError_t launch_transform<double>(const Dev&, const void*, int, int, int, cudaStream_t);

// Opt-in shared-memory sizes of this file's kernels, set once per context (outside any
// stream capture).
cudaError_t prepare_fft(const Dev& d) {
  const int N = d.N;
  const int rpb32 = std::max(1, 4096 / N), rpb64 = std::max(1, 2048 / N);
  const int cpb32 = std::min(N, 16), cpb64 = std::min(N, 8);
  const size_t inv = size_t(INV_ZT) * (padded_len(N) + 1) * sizeof(double2);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(fft_rows_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(size_t(rpb32) * padded_len(N) * sizeof(float2)))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(fft_rows_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(size_t(rpb64) * padded_len(N) * sizeof(double2)))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(fft_cols_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(size_t(cpb32) * (padded_len(N) + 1) * sizeof(float2)))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(fft_cols_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(size_t(cpb64) * (padded_len(N) + 1) * sizeof(double2)))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(inv))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(lateral_dft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(inv))) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(lateral_idft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(inv))) !=
      cudaSuccess)
    return e;
  switch (N) {
    case 32: return wfft_cols_prepare<1>();
    case 64: return wfft_cols_prepare<2>();
    case 128: return wfft_cols_prepare<4>();
    case 256: return wfft_cols_prepare<8>();
    case 512: return wfft_cols_prepare<16>();
    case 1024: return wfft_cols_prepare<32>();
    default: return cudaSuccess;
  }
}

cudaError_t launch_inverse(const Dev& d, void* V, int V_dtype, cudaStream_t s) {
  size_t smem = size_t(INV_ZT) * (padded_len(d.N) + 1) * sizeof(double2);
  inverse_kernel<<<(d.nz + INV_ZT - 1) / INV_ZT, 256, smem, s>>>(d, V, V_dtype);
  return cudaGetLastError();
}

cudaError_t launch_lateral_dft(const Dev& d, const void* V, int V_dtype, cudaStream_t s) {
  size_t smem = size_t(INV_ZT) * (padded_len(d.N) + 1) * sizeof(double2);
  lateral_dft_kernel<<<(d.nz + INV_ZT - 1) / INV_ZT, 256, smem, s>>>(d, V, V_dtype);
  return cudaGetLastError();
}

cudaError_t launch_lateral_idft_real(const Dev& d, const double2* in, double scale, void* out,
                                     int out_dtype, cudaStream_t s) {
  size_t smem = size_t(INV_ZT) * (padded_len(d.N) + 1) * sizeof(double2);
  lateral_idft_kernel<<<(d.nz + INV_ZT - 1) / INV_ZT, 256, smem, s>>>(d, in, scale, out, out_dtype);
  return cudaGetLastError();
}

template <typename T>
cudaError_t forward_chunk(const Dev& d, void* D, int D_dtype, int f0, int nfc, cudaStream_t s) {
  using T2 = cplx_t<T>;
  const int xdtype = sizeof(T) == 4 ? EDT_C64 : EDT_C128;
  const size_t esz = D_dtype == EDT_C64 ? sizeof(float2) : sizeof(double2);
  void* Dc = static_cast<char*>(D) + size_t(f0) * d.N * d.N * esz;
  dim3 g(d.N / 16, d.N / 16, nfc);
  born_spectral_kernel<T><<<g, 256, 0, s>>>(d, reinterpret_cast<T2*>(d.X), f0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // inverse of the data transform: undo pass 2 (sign -, 1/N), then pass 1 (sign +, 1/N)
  if ((e = cols_fft<T>(d, reinterpret_cast<T2*>(d.X), nfc, -1, T(1) / T(d.N), s)) != cudaSuccess) return e;
  return rows_fft<T>(d, d.X, xdtype, Dc, D_dtype, (long long)nfc * d.N, +1, T(1) / T(d.N), s);
}

// Adjoint of the data transform on the chunk's planes X[fi][q][p] (FP32): the conjugate
// transpose of pass 2 (sign -, unscaled) then of pass 1 (sign +, unscaled) into D[f0 + fi].
cudaError_t launch_transform_adjoint(const Dev& d, void* D, int D_dtype, int f0, int nfc, cudaStream_t s) {
  const size_t esz = D_dtype == EDT_C64 ? sizeof(float2) : sizeof(double2);
  void* Dc = static_cast<char*>(D) + size_t(f0) * d.N * d.N * esz;
  cudaError_t e = cols_fft<float>(d, reinterpret_cast<float2*>(d.X), nfc, -1, 1.f, s);
  if (e != cudaSuccess) return e;
  return rows_fft<float>(d, d.X, EDT_C64, Dc, D_dtype, (long long)nfc * d.N, +1, 1.f, s);
}

// Adjoint of the spectral Born model on one chunk of FP64 planes X[fi][q][p] = D2(p, q):
// vfull[m][z] += sum_f sum_p conj(s_f g(k_p, z) g(k_{p-m}, z)) D2(p, p - m), one thread per
// (m, z) (a warp over 32 consecutive depths of one m: table reads coalesced, the D2 value
// broadcast).
__global__ void __launch_bounds__(256) born_adjoint64_kernel(Dev d, int f0, int nfc) {
  const int N = d.N, msk = N - 1;
  const int z = blockIdx.y * 32 + (threadIdx.x & 31);
  const int m = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (z >= d.nz || m >= N) return;
  const double2* X = reinterpret_cast<const double2*>(d.X);
  double2 acc = make_double2(0.0, 0.0);
  for (int fi = 0; fi < nfc; ++fi) {
    const int f = f0 + fi;
    const FreqConst fc = d.fc[f];
    const double2 om = make_double2(fc.om_re, fc.om_im);
    const double2 sf = (d.dz / d.dx) * (om * om);
    const double2* g = d.g64 + size_t(f) * d.nk * d.nz;
    const double2* Xf = X + size_t(fi) * N * N;
    double2 sum = make_double2(0.0, 0.0);
    for (int p = 0; p < N; ++p) {
      const int q = (p - m) & msk;
      const int np = p <= N / 2 ? p : N - p, nq = q <= N / 2 ? q : N - q;
      const double2 a = g[size_t(np) * d.nz + z] * g[size_t(nq) * d.nz + z];
      const double2 x = Xf[size_t(q) * N + p];
      sum = sum + make_double2(a.x * x.x + a.y * x.y, a.x * x.y - a.y * x.x);   // conj(a) x
    }
    acc = acc + make_double2(sf.x * sum.x + sf.y * sum.y, sf.x * sum.y - sf.y * sum.x);   // conj(s_f) sum
  }
  double2* out = d.vfull + size_t(m) * d.nz + z;
  *out = *out + acc;
}

cudaError_t launch_adjoint64_chunk(const Dev& d, const void* D, int D_dtype, int f0, int nfc, cudaStream_t s) {
  cudaError_t e = launch_transform<double>(d, D, D_dtype, f0, nfc, s);
  if (e != cudaSuccess) return e;
  born_adjoint64_kernel<<<dim3((d.N + 7) / 8, (d.nz + 31) / 32), 256, 0, s>>>(d, f0, nfc);
  return cudaGetLastError();
}

cudaError_t launch_forward(const Dev& d, const void* V, int V_dtype, void* D, int D_dtype,
                           cudaStream_t s) {
  size_t smem = size_t(INV_ZT) * (padded_len(d.N) + 1) * sizeof(double2);
  lateral_dft_kernel<<<(d.nz + INV_ZT - 1) / INV_ZT, 256, smem, s>>>(d, V, V_dtype);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the spectrum X holds one chunk of frequency planes at a time
  for (int f0 = 0; f0 < d.nf; f0 += d.fchunk) {
    const int nfc = std::min(d.fchunk, d.nf - f0);
    e = d.precision == EDT_FP64 ? forward_chunk<double>(d, D, D_dtype, f0, nfc, s)
                                : forward_chunk<float>(d, D, D_dtype, f0, nfc, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace edt
