// Window geometry: finite half-offset aperture on an nx x ny periodic midpoint grid
// (Section "A practical 3D geometry", with the aperture sinc of eq. M kept as the window's
// Dirichlet kernel).  ny = 1 is the 2D line survey with a finite aperture.
//
// Kernel rows (per frequency f, for every kept row (pair, f, j) and depth z):
//   M(k_m; f, j, z) = c_f sum_y exp(i k_m.y) U_j(y, z),
//   U_j(y, z)       = sum_w exp(-2 pi i j.w/W) G(y - w, z) G(y + w, z),
// with G(y, z) = (1/(L_x L_y)) sum_a exp(i k_a.y) g(|k_a|, z) and c_f = omega~^2 dx dy dz.
// This is the row of the decoupled system (eq. DMV): summing the midpoint transform of the
// Born data over the window, y -> y + w turns the product G(2w - y) G(y) of the kernel of
// half-offset w into G(y - w) G(y + w) and the midpoint phase exp(-i k_m.w) cancels, so the
// window transform acts on U before one transform over y gives every k_m at once.
// Stages per frequency: fa_gspace (spectrum from the table, inverse 2D FFT -> G), fa_u
// (products and the window transform per y), fa_mrows (2D FFT of U_j per (j, z) plane,
// then the kept rows of that plane are written into the row table A32[row][z]).
//
// Data: the window transform of D[f][m][w] per midpoint (fa_dwin, written transposed as
// Dw[f][j][m]), then per (f, j) plane the midpoint FFT and the split right-hand sides of
// the kept rows, d_+ = (d(k_m) + d(-k_m))/2, d_- = (d(k_m) - d(-k_m))/(2i) (eq. Split).
//
// Inverse: Vhat(k_m) = x_+ + i x_- of each pair, Vhat(-k_m) = conj (eq. VSym), inverse 2D
// FFT per depth in FP64, V[y][x][z] = Re / (nx ny).
#include "edt_internal.h"
#include "cplx.cuh"
#include "wfft.cuh"

#include <algorithm>

namespace edt {

namespace {

constexpr int FA_THREADS = 512;   // plane kernels
constexpr int FW_THREADS = 256;   // window-transform kernels

__host__ __device__ constexpr int plane_ld(int nx) { return nx + 1; }   // odd row stride

// 2D transform of one plane s[ny][ld] in shared memory, nx = 32 PX, ny = 32 PY (PY = 0:
// ny = 1).  Warps take rows, then columns, each line a register-resident warp FFT; the
// twiddle table is that of length nx (ny == nx when PY > 0).
template <int PX, int PY, int SG>
__device__ void plane_fft2(float2* s, int ld, const float2* tw) {
  constexpr int NX = 32 * PX, NY = PY > 0 ? 32 * PY : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < NY; r += nw) {
    float2 v[PX];
#pragma unroll
    for (int a = 0; a < PX; ++a) v[a] = s[r * ld + 32 * a + lane];
    warp_fft<PX>(v, tw, NX, SG, lane);
    const int br = rbits(lane, 5) * PX;
#pragma unroll
    for (int k = 0; k < PX; ++k) s[r * ld + k + br] = v[k];
  }
  __syncthreads();
  if (PY > 0) {
    constexpr int QY = PY > 0 ? PY : 1;
    for (int c = warp; c < NX; c += nw) {
      float2 v[QY];
#pragma unroll
      for (int a = 0; a < QY; ++a) v[a] = s[(32 * a + lane) * ld + c];
      warp_fft<QY>(v, tw, NY, SG, lane);
      const int br = rbits(lane, 5) * QY;
#pragma unroll
      for (int k = 0; k < QY; ++k) s[(k + br) * ld + c] = v[k];
    }
    __syncthreads();
  }
}

// ---- small in-register DFTs of the window (sign -, natural order) --------------------
// cos and sin of 2 pi k / 16
__device__ __forceinline__ float2 w16(int k) {
  constexpr float C[16] = {1.f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                           0.f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                           -1.f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                           0.f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
  return make_float2(C[k & 15], -C[(k + 12) & 15]);        // e^{-2 pi i k/16} = (cos, -sin)
}

template <int W> __device__ __forceinline__ void reg_dft(float2 (&a)[W]);
template <> __device__ __forceinline__ void reg_dft<1>(float2 (&)[1]) {}
template <> __device__ __forceinline__ void reg_dft<2>(float2 (&a)[2]) {
  const float2 u = a[0], v = a[1];
  a[0] = u + v; a[1] = u - v;
}
template <> __device__ __forceinline__ void reg_dft<4>(float2 (&a)[4]) {
  const float2 b0 = a[0] + a[2], b1 = a[0] - a[2], b2 = a[1] + a[3], b3 = rot4<-1>(a[1] - a[3]);
  a[0] = b0 + b2; a[2] = b0 - b2; a[1] = b1 + b3; a[3] = b1 - b3;
}
template <> __device__ __forceinline__ void reg_dft<8>(float2 (&a)[8]) { dft8<-1>(a); }
template <> __device__ __forceinline__ void reg_dft<16>(float2 (&a)[16]) {
  float2 e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) { e[i] = a[2 * i]; o[i] = a[2 * i + 1]; }
  dft8<-1>(e);
  dft8<-1>(o);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float2 t = o[k] * w16(k);
    a[k] = e[k] + t;
    a[k + 8] = e[k] - t;
  }
}

// signed-index DFT over a window of W samples: out[j] = sum_w exp(-2 pi i j w/W) in[w] with
// j, w in [-W/2, W/2): the plain DFT of (-1)^w in[w], times (-1)^j (-1)^(W/2) (W >= 2).
__host__ __device__ constexpr bool alt_sign_end(int W) { return W >= 2 && ((W / 2) & 1); }
__device__ __forceinline__ float2 neg_if(float2 v, bool n) { return n ? make_float2(-v.x, -v.y) : v; }

// ---- kernel rows -----------------------------------------------------------------------
// G(y, z) for one frequency: CTA per z.
template <int PX, int PY>
__global__ void __launch_bounds__(FA_THREADS) fa_gspace_kernel(Dev d, int f) {
  constexpr int NX = 32 * PX, NY = PY > 0 ? 32 * PY : 1, LD = plane_ld(NX);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  const int z = blockIdx.x, hx = NX / 2 + 1;
  const float2* g = d.g32 + size_t(f) * d.nk * d.nzs + z;
  for (int e = threadIdx.x; e < NX * NY; e += blockDim.x) {
    const int ay = e / NX, ax = e - ay * NX;
    const int qy = min(ay, NY - ay), qx = min(ax, NX - ax);
    s[ay * LD + ax] = g[size_t(qy * hx + qx) * d.nzs];
  }
  __syncthreads();
  plane_fft2<PX, PY, +1>(s, LD, d.tw32);
  const float sc = float(1.0 / (double(NX) * NY * d.dx * d.dy));
  float2* G = d.Gs + size_t(z) * NX * NY;
  for (int e = threadIdx.x; e < NX * NY; e += blockDim.x) {
    const int y = e / NX, x = e - y * NX;
    const float2 v = s[y * LD + x];
    G[e] = make_float2(sc * v.x, sc * v.y);
  }
}

// Exchange buffer of the two-pass window transforms: [jx][unit][wy] with an odd unit stride
// when WY > 1, so that both the row-wise writes and the column-wise reads spread over banks.
template <int WX, int WY> struct ExLayout {
  static constexpr int UPB = FW_THREADS / WY, US = WY > 1 ? WY + 1 : 1, S = UPB * US;
  static constexpr int SIZE = WX * S;
  __device__ static __forceinline__ int at(int jx, int u, int iwy) { return jx * S + u * US + iwy; }
};

// U_j(y, z) for one frequency: CTA per (y row, z), window transform per y in registers.
template <int WX, int WY>
__global__ void __launch_bounds__(FW_THREADS) fa_u_kernel(Dev d) {
  using L = ExLayout<WX, WY>;
  constexpr int UPB = L::UPB;                              // y points per pass
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* ex = reinterpret_cast<float2*>(smem_raw);       // exchange, L::SIZE
  float2* Grow = ex + L::SIZE;                            // [WY + 1][nx]: rows yy - WY/2 .. yy + WY/2
  const int nx = d.N, ny = d.ny, yy = blockIdx.x, z = blockIdx.y;
  const float2* G = d.Gs + size_t(z) * d.nxy;
  for (int e = threadIdx.x; e < (WY + 1) * nx; e += blockDim.x) {
    const int t = e / nx, x = e - t * nx;
    const int row = ((yy + t - WY / 2) % ny + ny) % ny;
    Grow[e] = G[size_t(row) * nx + x];
  }
  __syncthreads();
  for (int x0 = 0; x0 < nx; x0 += UPB) {
    {
      const int ux = threadIdx.x / WY, iwy = threadIdx.x - ux * WY, x = x0 + ux;
      if (x < nx) {
        const int wyv = iwy - WY / 2;
        const float2* Gm = Grow + (WY / 2 - wyv) * nx;    // row yy - wy
        const float2* Gp = Grow + (WY / 2 + wyv) * nx;    // row yy + wy
        float2 a[WX];
#pragma unroll
        for (int ix = 0; ix < WX; ++ix) {
          const int wxv = ix - WX / 2;
          const float2 p = Gm[(x - wxv + nx) % nx] * Gp[(x + wxv + nx) % nx];
          a[ix] = neg_if(p, WX >= 2 && (ix & 1));
        }
        reg_dft<WX>(a);
#pragma unroll
        for (int jx = 0; jx < WX; ++jx)
          ex[L::at(jx, ux, iwy)] = neg_if(a[jx], WX >= 2 && ((jx & 1) != alt_sign_end(WX)));
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < UPB * WX; t += blockDim.x) {
      const int jx = t / UPB, ux = t - jx * UPB, x = x0 + ux;   // consecutive threads: consecutive x
      if (x >= nx) continue;
      float2 b[WY];
#pragma unroll
      for (int iwy = 0; iwy < WY; ++iwy) b[iwy] = neg_if(ex[L::at(jx, ux, iwy)], WY >= 2 && (iwy & 1));
      reg_dft<WY>(b);
#pragma unroll
      for (int jy = 0; jy < WY; ++jy) {
        const float2 v = neg_if(b[jy], WY >= 2 && ((jy & 1) != alt_sign_end(WY)));
        d.U[(size_t(jy * WX + jx) * d.nz + z) * d.nxy + size_t(yy) * nx + x] = v;
      }
    }
    __syncthreads();
  }
}

// M(k_m; f, j, z) for one (j, z) plane: 2D FFT of U_j, then the kept rows of (f, j).
template <int PX, int PY>
__global__ void __launch_bounds__(FA_THREADS) fa_mrows_kernel(Dev d, int f, float2 cf) {
  constexpr int NX = 32 * PX, NY = PY > 0 ? 32 * PY : 1, LD = plane_ld(NX);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  const int j = blockIdx.x, z = blockIdx.y;
  const float2* P = d.U + (size_t(j) * d.nz + z) * (NX * NY);
  for (int e = threadIdx.x; e < NX * NY; e += blockDim.x) {
    const int y = e / NX, x = e - y * NX;
    s[y * LD + x] = P[e];
  }
  __syncthreads();
  plane_fft2<PX, PY, +1>(s, LD, d.tw32);
  const int e0 = d.fj_off[f * d.W + j], e1 = d.fj_off[f * d.W + j + 1];
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int2 ent = d.fj_ent[e];
    const int y = ent.x / NX, x = ent.x - y * NX;
    d.A32[size_t(ent.y) * d.nzs + z] = cf * s[y * LD + x];
  }
}

// ---- data ------------------------------------------------------------------------------
// Window transform of D[f][m][wy][wx] for UPB consecutive midpoints, written as Dw[f][j][m].
template <int WX, int WY, typename TIN>
__global__ void __launch_bounds__(FW_THREADS) fa_dwin_kernel(Dev d, const TIN* D) {
  using L = ExLayout<WX, WY>;
  constexpr int W = WX * WY, UPB = L::UPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* ex = reinterpret_cast<float2*>(smem_raw);
  const int f = blockIdx.y, m0 = blockIdx.x * UPB;
  {
    const int um = threadIdx.x / WY, iwy = threadIdx.x - um * WY, m = m0 + um;
    if (m < d.nxy) {
      const TIN* src = D + ((size_t(f) * d.nxy + m) * WY + iwy) * WX;
      float2 a[WX];
#pragma unroll
      for (int ix = 0; ix < WX; ++ix) {
        const TIN v = src[ix];
        a[ix] = neg_if(make_float2(float(v.x), float(v.y)), WX >= 2 && (ix & 1));
      }
      reg_dft<WX>(a);
#pragma unroll
      for (int jx = 0; jx < WX; ++jx)
        ex[L::at(jx, um, iwy)] = neg_if(a[jx], WX >= 2 && ((jx & 1) != alt_sign_end(WX)));
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < UPB * WX; t += blockDim.x) {
    const int jx = t / UPB, um = t - jx * UPB, m = m0 + um;   // consecutive threads: consecutive m
    if (m >= d.nxy) continue;
    float2 b[WY];
#pragma unroll
    for (int iwy = 0; iwy < WY; ++iwy) b[iwy] = neg_if(ex[L::at(jx, um, iwy)], WY >= 2 && (iwy & 1));
    reg_dft<WY>(b);
#pragma unroll
    for (int jy = 0; jy < WY; ++jy)
      d.Dw[(size_t(f) * W + jy * WX + jx) * d.nxy + m] =
          neg_if(b[jy], WY >= 2 && ((jy & 1) != alt_sign_end(WY)));
  }
}

// Midpoint FFT of one (f, j) plane of Dw and the split right-hand sides of its kept rows.
template <int PX, int PY>
__global__ void __launch_bounds__(FA_THREADS) fa_drhs_kernel(Dev d) {
  constexpr int NX = 32 * PX, NY = PY > 0 ? 32 * PY : 1, LD = plane_ld(NX);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  const int j = blockIdx.x, f = blockIdx.y;
  const float2* P = d.Dw + (size_t(f) * d.W + j) * (NX * NY);
  for (int e = threadIdx.x; e < NX * NY; e += blockDim.x) {
    const int y = e / NX, x = e - y * NX;
    s[y * LD + x] = P[e];
  }
  __syncthreads();
  plane_fft2<PX, PY, -1>(s, LD, d.tw32);
  const int e0 = d.fj_off[f * d.W + j], e1 = d.fj_off[f * d.W + j + 1];
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int2 ent = d.fj_ent[e];
    const int y = ent.x / NX, x = ent.x - y * NX;
    const int ny2 = (NY - y) % NY, nx2 = (NX - x) % NX;
    const float2 a = s[y * LD + x], b = s[ny2 * LD + nx2];
    reinterpret_cast<float4*>(d.rhs)[ent.y] =
        make_float4(0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.y - b.y), -0.5f * (a.x - b.x));
  }
}

// ---- inverse ---------------------------------------------------------------------------
// Vhat of every pair and its conjugate at -k_m into vfull[z][m] (FP64), Vhat[pair][z] kept.
__global__ void fa_vfull_kernel(Dev d) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)d.nsub * d.nz) return;
  const int p = int(t / d.nz), z = int(t - (long long)p * d.nz);
  const double* xm = d.x + (size_t(p) * d.nz + z) * 2;
  double re = xm[0], im = xm[1];
  if (d.status[p] != EDT_OK) { re = 0.0; im = 0.0; }
  const int m = d.pair_m[p], nx = d.N, y = m / nx, x = m - y * nx;
  const int mneg = ((d.ny - y) % d.ny) * nx + (nx - x) % nx;
  if (mneg == m) im = 0.0;
  d.vhat[size_t(p) * d.nz + z] = make_double2(re, im);
  d.vfull[size_t(z) * d.nxy + m] = make_double2(re, im);
  d.vfull[size_t(z) * d.nxy + mneg] = make_double2(re, -im);
}

__global__ void fa_vout_kernel(Dev d, void* V, int V_dtype) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)d.nxy * d.nz) return;
  const int m = int(t / d.nz), z = int(t - (long long)m * d.nz);
  const double v = d.vfull[size_t(z) * d.nxy + m].x / double(d.nxy);
  if (V_dtype == EDT_F64) reinterpret_cast<double*>(V)[t] = v;
  else reinterpret_cast<float*>(V)[t] = float(v);
}

// Gram metadata of window rows: row r of the kernel table times the ones row, weight 1;
// the ones row itself.
__global__ void fa_setup_kernel(Dev d, long long nrows) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nrows) {
    GramRow g;
    g.offp = unsigned(t);
    g.offq = unsigned(d.ones_row);
    g.sw = 1.f;
    g.pad = 0.f;
    d.gent[t] = g;
  }
  if (t < d.nz) d.A32[size_t(d.ones_row) * d.nzs + t] = make_float2(1.f, 0.f);
}

template <int WX, int WY>
size_t u_smem(int nx) { return (size_t(ExLayout<WX, WY>::SIZE) + size_t(WY + 1) * nx) * sizeof(float2); }

template <int PX, int PY>
size_t plane_smem() { return size_t(PY > 0 ? 32 * PY : 1) * plane_ld(32 * PX) * sizeof(float2); }

template <int PX, int PY>
cudaError_t rows_for(const Dev& d, int f, float2 cf, cudaStream_t s) {
  const size_t sm = plane_smem<PX, PY>();
  fa_gspace_kernel<PX, PY><<<d.nz, FA_THREADS, sm, s>>>(d, f);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 gu(d.ny, d.nz);
  switch (d.wx * 32 + d.wy) {
#define FA_U(WX, WY) case WX * 32 + WY: fa_u_kernel<WX, WY><<<gu, FW_THREADS, u_smem<WX, WY>(d.N), s>>>(d); break;
    FA_U(1, 1) FA_U(2, 1) FA_U(4, 1) FA_U(8, 1) FA_U(16, 1)
    FA_U(2, 2) FA_U(4, 4) FA_U(8, 8) FA_U(16, 16) FA_U(4, 2) FA_U(8, 4) FA_U(16, 8)
#undef FA_U
    default: return cudaErrorInvalidValue;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  fa_mrows_kernel<PX, PY><<<dim3(d.W, d.nz), FA_THREADS, sm, s>>>(d, f, cf);
  return cudaGetLastError();
}

template <typename TIN>
cudaError_t dwin_for(const Dev& d, const TIN* D, cudaStream_t s) {
  const unsigned nb = unsigned((d.nxy + FW_THREADS / d.wy - 1) / (FW_THREADS / d.wy));
  dim3 g(nb, d.nf);
  switch (d.wx * 32 + d.wy) {
#define FA_D(WX, WY) case WX * 32 + WY: fa_dwin_kernel<WX, WY, TIN><<<g, FW_THREADS, ExLayout<WX, WY>::SIZE * sizeof(float2), s>>>(d, D); break;
    FA_D(1, 1) FA_D(2, 1) FA_D(4, 1) FA_D(8, 1) FA_D(16, 1)
    FA_D(2, 2) FA_D(4, 4) FA_D(8, 8) FA_D(16, 16) FA_D(4, 2) FA_D(8, 4) FA_D(16, 8)
#undef FA_D
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int PX, int PY>
cudaError_t prepare_plane() {
  const int sm = int(plane_smem<PX, PY>());
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(fa_gspace_kernel<PX, PY>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(fa_mrows_kernel<PX, PY>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(fa_drhs_kernel<PX, PY>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

// plane shapes: (nx, ny) = (32 PX, 32 PY), PY = 0 for a line
#define FA_SHAPES(X) X(1, 0) X(2, 0) X(4, 0) X(8, 0) X(16, 0) X(1, 1) X(2, 2) X(4, 4)

}  // namespace

bool fa_supported(int nx, int ny, int wx, int wy) {
  const int px = nx / 32, py = ny == 1 ? 0 : ny / 32;
  bool shape = false;
#define FA_S(PX, PY) shape |= (px == PX && py == PY && nx == 32 * PX && (PY == 0 ? ny == 1 : ny == 32 * PY));
  FA_SHAPES(FA_S)
#undef FA_S
  const int k = wx * 32 + wy;
  const bool win = k == 1 * 32 + 1 || k == 2 * 32 + 1 || k == 4 * 32 + 1 || k == 8 * 32 + 1 ||
                   k == 16 * 32 + 1 || k == 2 * 32 + 2 || k == 4 * 32 + 4 || k == 8 * 32 + 8 ||
                   k == 16 * 32 + 16 || k == 4 * 32 + 2 || k == 8 * 32 + 4 || k == 16 * 32 + 8;
  return shape && win && wx <= nx && wy <= ny;
}

cudaError_t launch_fa_rows(const Dev& d, int f, double2 cf, cudaStream_t s) {
  const float2 c = make_float2(float(cf.x), float(cf.y));
  const int px = d.N / 32, py = d.ny == 1 ? 0 : d.ny / 32;
#define FA_R(PX, PY) if (px == PX && py == PY) return rows_for<PX, PY>(d, f, c, s);
  FA_SHAPES(FA_R)
#undef FA_R
  return cudaErrorInvalidValue;
}

cudaError_t launch_fa_data(const Dev& d, const void* D, int D_dtype, cudaStream_t s) {
  cudaError_t e = D_dtype == EDT_C64 ? dwin_for<float2>(d, static_cast<const float2*>(D), s)
                                     : dwin_for<double2>(d, static_cast<const double2*>(D), s);
  if (e != cudaSuccess) return e;
  const int px = d.N / 32, py = d.ny == 1 ? 0 : d.ny / 32;
#define FA_DR(PX, PY) \
  if (px == PX && py == PY) { \
    fa_drhs_kernel<PX, PY><<<dim3(d.W, d.nf), FA_THREADS, plane_smem<PX, PY>(), s>>>(d); \
    return cudaGetLastError(); \
  }
  FA_SHAPES(FA_DR)
#undef FA_DR
  return cudaErrorInvalidValue;
}

cudaError_t launch_fa_inverse(const Dev& d, void* V, int V_dtype, cudaStream_t s) {
  const long long n1 = (long long)d.nsub * d.nz;
  fa_vfull_kernel<<<unsigned((n1 + 255) / 256), 256, 0, s>>>(d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = fft2_f64(d, d.vfull, d.nz, d.ny, +1, 1.0, s)) != cudaSuccess) return e;
  const long long n2 = (long long)d.nxy * d.nz;
  fa_vout_kernel<<<unsigned((n2 + 255) / 256), 256, 0, s>>>(d, V, V_dtype);
  return cudaGetLastError();
}

cudaError_t launch_fa_setup(const Dev& d, long long nrows, cudaStream_t s) {
  const long long n = std::max<long long>(nrows, d.nz);
  fa_setup_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(d, nrows);
  return cudaGetLastError();
}

cudaError_t prepare_fa(const Dev& d) {
  const int px = d.N / 32, py = d.ny == 1 ? 0 : d.ny / 32;
  cudaError_t e = cudaSuccess;
  switch (d.wx * 32 + d.wy) {
#define FA_A(WX, WY) case WX * 32 + WY: \
    e = cudaFuncSetAttribute(fa_u_kernel<WX, WY>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(u_smem<WX, WY>(d.N))); \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fa_dwin_kernel<WX, WY, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ExLayout<WX, WY>::SIZE * sizeof(float2))); \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fa_dwin_kernel<WX, WY, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ExLayout<WX, WY>::SIZE * sizeof(float2))); \
    break;
    FA_A(1, 1) FA_A(2, 1) FA_A(4, 1) FA_A(8, 1) FA_A(16, 1)
    FA_A(2, 2) FA_A(4, 4) FA_A(8, 8) FA_A(16, 16) FA_A(4, 2) FA_A(8, 4) FA_A(16, 8)
#undef FA_A
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
#define FA_P(PX, PY) if (px == PX && py == PY) return prepare_plane<PX, PY>();
  FA_SHAPES(FA_P)
#undef FA_P
  return cudaErrorInvalidValue;
}

}  // namespace edt
