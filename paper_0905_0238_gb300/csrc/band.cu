// Band-limited data transform and right-hand-side gather of the mixed-precision path.
//
// Only wavenumbers that survive the evanescent cut enter any system: row (f, p) of midpoint
// index m is kept when |p'| c_min < cutoff f L and |q'| c_min < cutoff f L (p', q' the
// signed indices), so at frequency f every element of the transformed plane that is read,
// D2(p, q) with its partners D2(q, p), D2(-q, -p), D2(-p, -q), has both indices in the band
// B_f = {n' : |n'| c_min < cutoff f L}, a symmetric interval [lo_f, lo_f + w_f).  The
// transform of the plane is therefore computed only where it is needed:
//
//  1. rows: every receiver line D[f][is][.] gets the full FFT over ir (sign -), but only
//     the band p' in B_f is stored, as Y_f[is][p' - lo_f] (w_f values per line);
//  2. columns: only the w_f band columns of Y_f get the FFT over is (sign +), and only the
//     band q' in B_f is stored: Xc_f[q' - lo_f][p' - lo_f] = D2(p, q);
//  3. gather: one thread per row of the chunk reads its four elements of Xc_f, forms
//     d_+/d_- (eq. Split, folded partner averaged in) and writes the right-hand sides
//     (16 bytes per row; the Gram's row metadata is fixed by the plan and written once).
//
// Planes are processed in chunks whose Y and Xc fit in L2 together, so the intermediate
// spectra of a chunk are written and read back on chip: HBM sees the data read once and the
// right-hand sides written once.  With the cut disabled B_f is the whole index range and the
// same code computes the full transform.
#include "edt_internal.h"
#include "cplx.cuh"
#include "wfft.cuh"

namespace edt {

namespace {

__device__ __forceinline__ int sidx_of(int k, int N) { return k <= (N >> 1) ? k : k - N; }
// tile index with one pad element per 16 (spreads strided accesses over the banks)
__device__ __forceinline__ int pd16(int e) { return e + (e >> 4); }
__device__ __forceinline__ float2 to_c64(float2 v) { return v; }
__device__ __forceinline__ float2 to_c64(double2 v) { return make_float2(float(v.x), float(v.y)); }

// FFT policies: lines of N = 512 use the radix-8 form, other N the shuffle form.
// MINB_*: blocks per SM the register allocation is bounded for (1: unbounded)
struct PolicyRadix8 {
  static constexpr int N = 512, P = 16, SCRATCH = Fft512::SCRATCH, MINB_ROWS = 4, MINB_COLS = 3;
  __device__ static __forceinline__ int in_idx(int l, int j) { return Fft512::idx(l, j); }
  __device__ static __forceinline__ int out_idx(int l, int j) { return Fft512::idx(l, j); }
  template <int SG>
  __device__ static __forceinline__ void run(float2 (&v)[P], float2* buf, const float2* tws,
                                             const float2*, int l) {
    Fft512::run<SG>(v, buf, tws, l);
  }
};

template <int PP>
struct PolicyShuffle {
  static constexpr int N = 32 * PP, P = PP, SCRATCH = 0, MINB_ROWS = 1, MINB_COLS = 1;
  __device__ static __forceinline__ int in_idx(int l, int j) { return 32 * j + l; }
  __device__ static __forceinline__ int out_idx(int l, int j) { return j + PP * rbits(l, 5); }
  template <int SG>
  __device__ static __forceinline__ void run(float2 (&v)[P], float2*, const float2*,
                                             const float2* tw, int l) {
    warp_fft<PP>(v, tw, N, SG, l);
  }
};

constexpr int BR_WARPS = 8;    // receiver lines per block in the row pass
// band columns per block in the column pass: 4, 8 or 16 (the autotuner's choice)

template <class F>
__device__ __forceinline__ void fill_twiddles(float2* tws, const float2* tw32) {
  if (F::SCRATCH == 0) return;                     // the shuffle form reads the global table
  for (int e = threadIdx.x; e < F::N; e += blockDim.x) tws[Fft512::tpad(e)] = tw_at(tw32, e, F::N);
}

// Pass 1: FFT over ir of the receiver lines of planes [f0, f0 + nfc); band outputs only.
template <class F, typename TIN>
__global__ void __launch_bounds__(BR_WARPS * 32, F::MINB_ROWS) band_rows_kernel(Dev d, const TIN* D, int f0,
                                                                                int nfc) {
  constexpr int N = F::N, LN = clog2(N);
  __shared__ float2 tws[F::SCRATCH > 0 ? Fft512::TWS : 1];
  __shared__ float2 scratch[BR_WARPS][F::SCRATCH > 0 ? F::SCRATCH : 1];
  fill_twiddles<F>(tws, d.tw32);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long line = (long long)blockIdx.x * BR_WARPS + warp;
  if (line >= (long long)nfc * N) return;
  const int f = f0 + int(line >> LN), is = int(line & (N - 1));
  const BandInfo b = d.band[f];
  if (b.w == 0) return;
  float2 v[F::P];
  const TIN* Dl = D + (size_t(f) * N + is) * N;
#pragma unroll
  for (int j = 0; j < F::P; ++j) v[j] = to_c64(Dl[F::in_idx(lane, j)]);
  F::template run<-1>(v, scratch[warp], tws, d.tw32, lane);
  float2* Y = d.Yc + b.yoff + size_t(is) * b.w;
#pragma unroll
  for (int j = 0; j < F::P; ++j) {
    const int pb = sidx_of(F::out_idx(lane, j), N) - b.lo;
    if (unsigned(pb) < unsigned(b.w)) Y[pb] = v[j];
  }
}

// Pass 2: FFT over is of BC_COLS band columns of one plane (block table entry (f, pb0)),
// staged through a shared tile so that both the loads and the band stores are row-wise.
template <class F>
__host__ __device__ constexpr int cols_ld() {
  // column stride of the tile: holds a column at pd(e) = e + e/16 and the radix-8 exchange
  // buffer; odd, so the row-wise staging loops spread over the banks
  return ((F::N + F::N / 16 > F::SCRATCH ? F::N + F::N / 16 : F::SCRATCH) | 1);
}

template <class F, int BC_COLS>
__global__ void __launch_bounds__(BC_COLS * 32, (F::MINB_COLS * 8) / BC_COLS > 0 ? (F::MINB_COLS * 8) / BC_COLS : 1)
band_cols_kernel(Dev d, int blk0) {
  constexpr int N = F::N, LD = cols_ld<F>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);            // [BC_COLS][LD]
  float2* tws = tile + BC_COLS * LD;                              // radix-8 twiddle table
  fill_twiddles<F>(tws, d.tw32);
  const int2 bi = d.bcol[blk0 + blockIdx.x];
  const BandInfo b = d.band[bi.x];
  const int pb0 = bi.y, ncol = min(BC_COLS, b.w - pb0);
  const float2* Y = d.Yc + b.yoff;
  {
    // N * BC_COLS elements, BC_COLS * 32 threads: all loads of a thread issued before its
    // shared stores
    constexpr int PER = N / 32;
    const int c = threadIdx.x % BC_COLS, is0 = threadIdx.x / BC_COLS;
    float2 y[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i)
      y[i] = c < ncol ? Y[size_t(is0 + 32 * i) * b.w + pb0 + c] : make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < PER; ++i) tile[c * LD + pd16(is0 + 32 * i)] = y[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* col = tile + warp * LD;
  if (warp < ncol) {
    float2 v[F::P];
#pragma unroll
    for (int j = 0; j < F::P; ++j) v[j] = col[pd16(F::in_idx(lane, j))];
    F::template run<+1>(v, col, tws, d.tw32, lane);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < F::P; ++j) col[pd16(F::out_idx(lane, j))] = v[j];
  }
  __syncthreads();
  float2* Xo = d.Xc + b.xoff;
  for (int e = threadIdx.x; e < b.w * BC_COLS; e += blockDim.x) {
    const int qb = e / BC_COLS, c = e - qb * BC_COLS;
    if (c < ncol) Xo[size_t(qb) * b.w + pb0 + c] = tile[c * LD + pd16((b.lo + qb) & (N - 1))];
  }
}

// Pass 3: right-hand sides, one thread per row of the chunk (rows of subproblem m at the
// chunk's frequencies are contiguous; cpre[m] counts the chunk's rows of subproblems < m).
constexpr int MAX_NSUB = 1024 / 2 + 1;

__global__ void __launch_bounds__(256) band_rhs_kernel(Dev d, const long long* cpre_g, long long nrow,
                                                       int f0) {
  __shared__ long long cpre[MAX_NSUB + 1];
  for (int i = threadIdx.x; i <= d.nsub; i += blockDim.x) cpre[i] = cpre_g[i];
  __syncthreads();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrow) return;
  int lo = 0, hi = d.nsub;                            // cpre[lo] <= t < cpre[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (cpre[mid] <= t) lo = mid; else hi = mid;
  }
  const int m = lo, N = d.N, msk = N - 1;
  const long long ri = d.row_off_mf[size_t(m) * (d.nf + 1) + f0] + (t - cpre[m]);
  const uint32_t row = d.rows[ri];
  const int f = row_f(row), p = row_p(row), q = (p - m) & msk;
  const BandInfo b = d.band[f];
  const float2* X = d.Xc + b.xoff;
  auto at = [&](int pp, int qq) {                     // D2(pp, qq), both indices in the band
    return X[size_t(sidx_of(qq & msk, N) - b.lo) * b.w + (sidx_of(pp & msk, N) - b.lo)];
  };
  float2 a = at(p, q), c = at(q, p);
  if (row_w2(row)) {
    const float2 a2 = at(-q, -p), c2 = at(-p, -q);
    a = make_float2(0.5f * (a.x + a2.x), 0.5f * (a.y + a2.y));
    c = make_float2(0.5f * (c.x + c2.x), 0.5f * (c.y + c2.y));
  }
  const float2 dp = make_float2(0.5f * (a.x + c.x), 0.5f * (a.y + c.y));
  const float2 dm = make_float2(0.5f * (a.y - c.y), -0.5f * (a.x - c.x));
  const FreqConst fc = d.fc[f];
  const float2 rot = make_float2(float(fc.rot_re), float(fc.rot_im));
  const float2 rp = dp * rot, rm = dm * rot;
  reinterpret_cast<float4*>(d.rhs)[ri] = make_float4(rp.x, rp.y, rm.x, rm.y);
}

template <class F>
size_t cols_smem(int bc) {
  return (size_t(bc) * cols_ld<F>() + (F::SCRATCH > 0 ? Fft512::TWS : 0)) * sizeof(float2);
}

template <class F>
cudaError_t run_chunk(const Dev& d, const BandChunk& ch, const void* D, int D_dtype, cudaStream_t s) {
  const int nfc = ch.f1 - ch.f0;
  const long long lines = (long long)nfc * F::N;
  const unsigned nb = unsigned((lines + BR_WARPS - 1) / BR_WARPS);
  if (D_dtype == EDT_C64)
    band_rows_kernel<F, float2><<<nb, BR_WARPS * 32, 0, s>>>(d, static_cast<const float2*>(D), ch.f0, nfc);
  else
    band_rows_kernel<F, double2><<<nb, BR_WARPS * 32, 0, s>>>(d, static_cast<const double2*>(D), ch.f0, nfc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ch.nbcol > 0) {
    const unsigned nb2 = unsigned(ch.nbcol);
    const size_t sm = cols_smem<F>(d.tune_bc);
    if (d.tune_bc == 4) band_cols_kernel<F, 4><<<nb2, 4 * 32, sm, s>>>(d, ch.bcol0);
    else if (d.tune_bc == 16) band_cols_kernel<F, 16><<<nb2, 16 * 32, sm, s>>>(d, ch.bcol0);
    else band_cols_kernel<F, 8><<<nb2, 8 * 32, sm, s>>>(d, ch.bcol0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ch.nrow > 0) {
    band_rhs_kernel<<<unsigned((ch.nrow + 255) / 256), 256, 0, s>>>(d, d.cpre + size_t(ch.ci) * (d.nsub + 1),
                                                                   ch.nrow, ch.f0);
    e = cudaGetLastError();
  }
  return e;
}

template <class F>
cudaError_t prepare_policy() {
  cudaError_t e = cudaFuncSetAttribute(band_cols_kernel<F, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(cols_smem<F>(4)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(band_cols_kernel<F, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(cols_smem<F>(8)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(band_cols_kernel<F, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(cols_smem<F>(16)));
  return e;
}

}  // namespace

bool band_supported(int N) { return N >= 32 && N <= 1024; }


cudaError_t launch_band_chunk(const Dev& d, const BandChunk& ch, const void* D, int D_dtype, cudaStream_t s) {
  switch (d.N) {
    case 32: return run_chunk<PolicyShuffle<1>>(d, ch, D, D_dtype, s);
    case 64: return run_chunk<PolicyShuffle<2>>(d, ch, D, D_dtype, s);
    case 128: return run_chunk<PolicyShuffle<4>>(d, ch, D, D_dtype, s);
    case 256: return run_chunk<PolicyShuffle<8>>(d, ch, D, D_dtype, s);
    case 512: return run_chunk<PolicyRadix8>(d, ch, D, D_dtype, s);
    case 1024: return run_chunk<PolicyShuffle<32>>(d, ch, D, D_dtype, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t prepare_band(const Dev& d) {
  switch (d.N) {
    case 32: return prepare_policy<PolicyShuffle<1>>();
    case 64: return prepare_policy<PolicyShuffle<2>>();
    case 128: return prepare_policy<PolicyShuffle<4>>();
    case 256: return prepare_policy<PolicyShuffle<8>>();
    case 512: return prepare_policy<PolicyRadix8>();
    case 1024: return prepare_policy<PolicyShuffle<32>>();
    default: return cudaSuccess;
  }
}

}  // namespace edt
