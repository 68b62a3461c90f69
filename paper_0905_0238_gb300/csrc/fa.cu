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
// (products and the window transform per y), fa_mrows (2D FFT of U_j per (j, z) plane, from
// its rows 0..ny/2 since U_j is centrosymmetric; clusters of ZC consecutive depths, then the
// kept rows of (f, j) are written into the row table A32[row][z] ZC depths at a time from the
// cluster's distributed shared memory).
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
#include <cooperative_groups.h>

namespace edt {

namespace {

// threads of the plane kernels: a 2D plane fills shared memory (one CTA per SM), so it takes
// the most warps a CTA can have; a line is one warp's FFT
template <int PY> __host__ __device__ constexpr int plane_threads() { return PY > 0 ? 1024 : 128; }
// the kernel-row planes are half planes (below): two CTAs of 512 threads share an SM
template <int PY> __host__ __device__ constexpr int mrows_threads() { return PY > 0 ? 512 : 128; }
constexpr int FW_THREADS = 256;   // window-transform kernels

// Plane layout in shared memory: element (y, x) at y * ld + 2 (y/16) + x + 2 (x/16) with
// ld = 1 mod 16, so that along a row and along a column element i sits at i + 2 (i/16)
// modulo 16 complex slots (32 banks).  Every access pattern of the 16-thread line FFT below
// (stride-16 loads, the paired reads of its second pass, the natural-order stores) then
// sends the 16 lanes of each 8-byte phase to 16 distinct slot pairs: no bank conflicts.
__host__ __device__ constexpr int plane_ld(int nx) { return (nx + 2 * (nx / 16) + 15) / 16 * 16 + 1; }
__host__ __device__ constexpr int plane_words(int nx, int ny) {
  return (ny - 1) * plane_ld(nx) + 2 * ((ny - 1) / 16) + (nx - 1) + 2 * ((nx - 1) / 16) + 1;
}
__device__ __forceinline__ int paddr(int y, int x, int ld) { return y * ld + 2 * (y >> 4) + x + 2 * (x >> 4); }


// 2D transform of one plane in shared memory (layout above), nx = 32 PX, ny = 32 PY (PY = 0:
// ny = 1).  Warps take rows, then columns, each line a register-resident warp FFT; the
// twiddle table is that of length nx (ny == nx when PY > 0).
// Load a contiguous [NY][NX] plane into the shared layout: every thread issues all of its loads
// before its shared stores, so a CTA keeps the whole plane's reads in flight.
template <int NX, int NY, int LD, int T>
__device__ __forceinline__ void load_plane(float2* s, const float2* P) {
  constexpr int TOT = NX * NY;
  if (TOT % T == 0) {
    constexpr int PER = TOT % T == 0 ? TOT / T : 1;
    float2 r[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) r[i] = P[threadIdx.x + i * T];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + i * T, y = e / NX, x = e - y * NX;
      s[paddr(y, x, LD)] = r[i];
    }
  } else {
    for (int e = threadIdx.x; e < TOT; e += blockDim.x) {
      const int y = e / NX, x = e - y * NX;
      s[paddr(y, x, LD)] = P[e];
    }
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

// In-register DFTs of R points with either sign (the 2D plane transforms)
template <int R, int SG> struct Dft;
template <int SG> struct Dft<2, SG> {
  __device__ static __forceinline__ void run(float2 (&a)[2]) {
    const float2 u = a[0], v = a[1];
    a[0] = u + v; a[1] = u - v;
  }
};
template <int SG> struct Dft<4, SG> {
  __device__ static __forceinline__ void run(float2 (&a)[4]) {
    const float2 b0 = a[0] + a[2], b1 = a[0] - a[2], b2 = a[1] + a[3], b3 = rot4<SG>(a[1] - a[3]);
    a[0] = b0 + b2; a[2] = b0 - b2; a[1] = b1 + b3; a[3] = b1 - b3;
  }
};
template <int SG> struct Dft<8, SG> {
  __device__ static __forceinline__ void run(float2 (&a)[8]) { dft8<SG>(a); }
};
template <int SG> struct Dft<16, SG> {
  __device__ static __forceinline__ void run(float2 (&a)[16]);
};

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

template <int SG>
__device__ __forceinline__ void Dft<16, SG>::run(float2 (&a)[16]) {
  float2 e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) { e[i] = a[2 * i]; o[i] = a[2 * i + 1]; }
  dft8<SG>(e);
  dft8<SG>(o);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float2 t = o[k] * tw_sg<SG>(w16(k));
    a[k] = e[k] + t;
    a[k + 8] = e[k] - t;
  }
}

// N-point FFT (N = 16 R, R in {2, 4, 8}) of one line by a group of 16 threads, t = 0..15,
// in place in shared memory (element i at s[addr(i)]).  With n = 16 a + t and
// k = k1 + R k2: pass 1 takes the R-point DFT over a of x[16 a + t] and applies W_N^{t k1},
// keeping the result in the slots 16 k1 + t; pass 2 takes the 16-point DFT over t for each
// k1, split between the thread pair (2 k1, 2 k1 + 1) as the 8-point DFTs of the even and the
// odd t (the odd half times W_16^k2), exchanged by one shuffle per value, and writes
// X[k1 + R k2] in natural order.  tw: W_N^e (sign -1) for e < N.  A group is a half-warp.
// src: where pass 1 reads the line (null: the shared slots themselves).
// src: where pass 1 reads the line (null: the shared slots themselves); rev: read it
// mirrored, element i at src[(-i) mod N].
template <int R, int SG, class Addr>
__device__ __forceinline__ void group_fft(float2* s, const Addr& addr, int t, const float2* tw,
                                          const float2* src = nullptr, bool rev = false) {
  const unsigned gm = 0xffffu << (threadIdx.x & 16);         // this half-warp
  // slot addresses are affine along each pass (the layout's skew steps at multiples of 16):
  // pass 1 reads slots 16 a + t, pass 2 reads 16 k1 + 2 i + h
  const int a1 = addr(t), s1 = addr(16) - addr(0), s2 = addr(2) - addr(0);
  float2 v[R];
  if (src) {
    constexpr int N = 16 * R;
#pragma unroll
    for (int a = 0; a < R; ++a) v[a] = src[rev ? ((N - 16 * a - t) & (N - 1)) : 16 * a + t];
  } else {
#pragma unroll
    for (int a = 0; a < R; ++a) v[a] = s[a1 + a * s1];
  }
  Dft<R, SG>::run(v);
#pragma unroll
  for (int k1 = 1; k1 < R; ++k1) v[k1] = v[k1] * tw_sg<SG>(tw[t * k1]);
#pragma unroll
  for (int k1 = 0; k1 < R; ++k1) s[a1 + k1 * s1] = v[k1];
  __syncwarp(gm);
  const int k1 = t >> 1, h = t & 1;
  const bool act = k1 < R;
  const int a2 = addr(16 * (act ? k1 : 0) + h);
  float2 u[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) u[i] = act ? s[a2 + i * s2] : make_float2(0.f, 0.f);
  dft8<SG>(u);
  if (h) {
#pragma unroll
    for (int k2 = 1; k2 < 8; ++k2) u[k2] = u[k2] * tw_sg<SG>(w16(k2));
  }
  float2 p[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    p[i].x = __shfl_xor_sync(gm, u[i].x, 1);
    p[i].y = __shfl_xor_sync(gm, u[i].y, 1);
  }
  __syncwarp(gm);                                            // pass-2 reads before the writes
  if (act) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 e = h ? p[i] : u[i], o = h ? u[i] : p[i];
      s[addr(k1 + R * (i + 8 * h))] = h ? e - o : e + o;
    }
  }
  __syncwarp(gm);
}

struct RowAddr {
  int r, ld;
  __device__ __forceinline__ int operator()(int i) const { return paddr(r, i, ld); }
};
struct ColAddr {
  int c, ld;
  __device__ __forceinline__ int operator()(int i) const { return paddr(i, c, ld); }
};

// gsrc: a row-major plane in global memory that the row pass reads directly (its loads then
// overlap other groups' arithmetic); null: the plane is already in s.  grows: rows stored in
// gsrc; a centrosymmetric plane (P(-y) = P(y)) keeps rows 0..NY/2 only and row r > NY/2 is
// row NY - r mirrored.
template <int PX, int PY, int SG>
__device__ void plane_fft2(float2* s, int ld, const float2* tw, const float2* tws,
                           const float2* gsrc = nullptr, int grows = 1 << 30) {
  constexpr int NX = 32 * PX, NY = PY > 0 ? 32 * PY : 1;
  if constexpr (PY > 0) {
    // square plane: one group of 16 threads per line, rows then columns
    constexpr int R = NX / 16;
    const int t = threadIdx.x & 15, grp = threadIdx.x >> 4, ng = blockDim.x >> 4;
    for (int r = grp; r < NY; r += ng) {
      const bool mir = r >= grows;
      group_fft<R, SG>(s, RowAddr{r, ld}, t, tws, gsrc ? gsrc + size_t(mir ? NY - r : r) * NX : nullptr, mir);
    }
    __syncthreads();
    for (int c = grp; c < NX; c += ng) group_fft<R, SG>(s, ColAddr{c, ld}, t, tws);
    __syncthreads();
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < NY; r += nw) {
    float2 v[PX];
#pragma unroll
    for (int a = 0; a < PX; ++a) v[a] = s[paddr(r, 32 * a + lane, ld)];
    warp_fft<PX>(v, tw, NX, SG, lane);
    const int br = rbits(lane, 5) * PX;
#pragma unroll
    for (int k = 0; k < PX; ++k) s[paddr(r, k + br, ld)] = v[k];
  }
  __syncthreads();
}

// 2D transform of a centrosymmetric N x N plane (P(-y) = P(y), so its transform X is
// centrosymmetric too) from its rows 0..N/2, in a half plane of N/2 + 3 rows (layout above):
//   row pass:    rows r = 0..N/2 transformed in place (read from gsrc, row-major N/2+1 rows);
//                V(r, k) for k > N/2 equals V(N - r, N - k) of the rows not stored.
//   column pass: columns c = 0..N/2 only (X(ky, kx) = X(-ky, -kx) gives the rest).  Element
//                e of column c is V(e, c) for e < N/2, else V(N - e, N - c) (column c' =
//                (N - c) mod N), read from the stored rows.  Its 128 slots ("homes") for the
//                in-place transform: e < N/2 at (e, c); e >= N/2 at (e - N/2, c') for
//                0 < c < N/2, and in the spare rows N/2 + 1 (c = 0) and N/2 + 2 (c = N/2).
//                The lines of different columns touch disjoint slots (column c owns rows
//                0..N/2 of columns c and c'), so the groups run without block barriers.
// Result: X(ky, kx) at sym_addr(ky, kx).
template <int N>
__device__ __forceinline__ int sym_addr(int ky, int kx, int ld) {
  constexpr int H = N / 2;
  if (kx > H) { ky = (N - ky) & (N - 1); kx = N - kx; }
  if (ky < H) return paddr(ky, kx, ld);
  if (kx == 0) return paddr(H + 1, ky - H, ld);
  if (kx == H) return paddr(H + 2, ky - H, ld);
  return paddr(ky - H, N - kx, ld);
}
__host__ __device__ constexpr int sym_plane_words(int n) { return plane_words(n, n / 2 + 3); }

// column c of the half plane, N = 16 R, by the 16 threads t of a half-warp (the line FFT of
// group_fft with the home map above; every home address is affine along each access
// sequence, so each is a per-thread base plus a constant step)
template <int R, int SG>
__device__ __forceinline__ void sym_col_fft(float2* s, int c, int ld, int t, const float2* tw) {
  constexpr int N = 16 * R, H = N / 2, HR = R / 2;
  const unsigned gm = 0xffffu << (threadIdx.x & 16);
  const int cm = (N - c) & (N - 1);
  const bool spec = c == 0 || c == H;
  const int srow = c == 0 ? H + 1 : H + 2;
  const int RS = 16 * ld + 2;                                 // 16 rows further
  // pass 1: element 16 a + t; a < R/2 at row 16 a + t of c, else row N - 16 a - t of c'
  const int lo = paddr(t, c, ld), hi = paddr(H - t, cm, ld);
  float2 v[R];
#pragma unroll
  for (int a = 0; a < R; ++a) v[a] = s[a < HR ? lo + a * RS : hi - (a - HR) * RS];
  __syncwarp(gm);                     // columns 0 and N/2 read slots that other lanes store to
  Dft<R, SG>::run(v);
#pragma unroll
  for (int k1 = 1; k1 < R; ++k1) v[k1] = v[k1] * tw_sg<SG>(tw[t * k1]);
  const int h1 = spec ? paddr(srow, t, ld) : paddr(t, cm, ld);   // home of element N/2 + t
  const int hs = spec ? 18 : RS;                                    // 16 elements further
#pragma unroll
  for (int k1 = 0; k1 < R; ++k1) s[k1 < HR ? lo + k1 * RS : h1 + (k1 - HR) * hs] = v[k1];
  __syncwarp(gm);
  // pass 2: the pair (2 k1, 2 k1 + 1) reads elements 16 k1 + 2 i + h
  const int k1 = t >> 1, h = t & 1;
  const bool act = k1 < R;
  const int kk = act ? k1 : 0;
  int b2, s2 = 2 * ld;
  if (kk < HR) b2 = paddr(16 * kk + h, c, ld);
  else if (!spec) b2 = paddr(16 * (kk - HR) + h, cm, ld);
  else { b2 = paddr(srow, 16 * (kk - HR) + h, ld); s2 = 2; }
  float2 u[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) u[i] = act ? s[b2 + i * s2] : make_float2(0.f, 0.f);
  dft8<SG>(u);
  if (h) {
#pragma unroll
    for (int k2 = 1; k2 < 8; ++k2) u[k2] = u[k2] * tw_sg<SG>(w16(k2));
  }
  float2 p[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    p[i].x = __shfl_xor_sync(gm, u[i].x, 1);
    p[i].y = __shfl_xor_sync(gm, u[i].y, 1);
  }
  __syncwarp(gm);
  // outputs X[k1 + R (i + 8 h)]: h = 0 at row k1 + R i of c; h = 1 at row k1 + R i of c'
  // (column k1 + R i of the spare row for c = 0, N/2); the skew term 2 ((R i) >> 4) is the
  // same in both forms because k1 < R
  if (act) {
    int b3, s3 = R * ld;
    if (!h) b3 = paddr(k1, c, ld);
    else if (!spec) b3 = paddr(k1, cm, ld);
    else { b3 = paddr(srow, k1, ld); s3 = R; }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 e = h ? p[i] : u[i], o = h ? u[i] : p[i];
      s[b3 + i * s3 + 2 * ((R * i) >> 4)] = h ? e - o : e + o;
    }
  }
  __syncwarp(gm);
}

// the half-plane transform above; gsrc: rows 0..N/2 of the plane, row-major in global memory
template <int PX, int SG>
__device__ void sym_plane_fft2(float2* s, int ld, const float2* tws, const float2* gsrc) {
  constexpr int N = 32 * PX, R = N / 16, H = N / 2;
  const int t = threadIdx.x & 15, grp = threadIdx.x >> 4, ng = blockDim.x >> 4;
  for (int r = grp; r <= H; r += ng) group_fft<R, SG>(s, RowAddr{r, ld}, t, tws, gsrc + size_t(r) * N);
  __syncthreads();
  for (int c = grp; c <= H; c += ng) sym_col_fft<R, SG>(s, c, ld, t, tws);
  __syncthreads();
}

// W_N^e (sign -1) for e < N in shared memory, from the context's table of length N
__device__ __forceinline__ void plane_twiddles(float2* tws, const float2* tw32, int N) {
  for (int e = threadIdx.x; e < N; e += blockDim.x) tws[e] = tw_at(tw32, e, N);
}

// signed-index DFT over a window of W samples: out[j] = sum_w exp(-2 pi i j w/W) in[w] with
// j, w in [-W/2, W/2): the plain DFT of (-1)^w in[w], times (-1)^j (-1)^(W/2) (W >= 2).
__host__ __device__ constexpr bool alt_sign_end(int W) { return W >= 2 && ((W / 2) & 1); }
__device__ __forceinline__ float2 neg_if(float2 v, bool n) { return n ? make_float2(-v.x, -v.y) : v; }

// ---- kernel rows -----------------------------------------------------------------------
// G(y, z) for one frequency: CTA per z.
template <int PX, int PY>
__global__ void __launch_bounds__(plane_threads<PY>()) fa_gspace_kernel(Dev d, int f) {
  constexpr int NX = 32 * PX, NY = PY > 0 ? 32 * PY : 1, LD = plane_ld(NX);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  const int z = blockIdx.x, hx = NX / 2 + 1;
  const float2* g = d.g32 + size_t(f) * d.nk * d.nzs + z;
  float2* tws = s + plane_words(NX, NY);
  plane_twiddles(tws, d.tw32, NX);
  for (int e = threadIdx.x; e < NX * NY; e += blockDim.x) {
    const int ay = e / NX, ax = e - ay * NX;
    const int qy = min(ay, NY - ay), qx = min(ax, NX - ax);
    s[paddr(ay, ax, LD)] = g[size_t(qy * hx + qx) * d.nzs];
  }
  __syncthreads();
  plane_fft2<PX, PY, +1>(s, LD, d.tw32, tws);
  const float sc = float(1.0 / (double(NX) * NY * d.dx * d.dy));
  float2* G = d.Gs + size_t(z) * NX * NY;
  for (int e = threadIdx.x; e < NX * NY; e += blockDim.x) {
    const int y = e / NX, x = e - y * NX;
    const float2 v = s[paddr(y, x, LD)];
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
// G is even, so U_j(-y) = U_j(y): only the rows y_y = 0..ny/2 are formed and stored, and only
// for the offset wavenumbers j that have kept rows at this frequency (compacted).
template <int WX, int WY>
__global__ void __launch_bounds__(FW_THREADS, 4) fa_u_kernel(Dev d, int f) {
  using L = ExLayout<WX, WY>;
  const int* jmap = d.jmap + size_t(f) * WX * WY;
  constexpr int UPB = L::UPB;                              // y points per pass
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* ex = reinterpret_cast<float2*>(smem_raw);       // exchange, L::SIZE
  float2* Grow = ex + L::SIZE;                            // [WY + 1][nx]: rows yy - WY/2 .. yy + WY/2
  const int nx = d.N, ny = d.ny, yy = blockIdx.x, z = blockIdx.y;
  const float2* G = d.Gs + size_t(z) * d.nxy;
  for (int e = threadIdx.x; e < (WY + 1) * nx; e += blockDim.x) {
    const int t = e / nx, x = e - t * nx;
    const int row = (yy + t - WY / 2 + ny) & (ny - 1);      // ny is a power of two
    Grow[e] = G[size_t(row) * nx + x];
  }
  // the second pass gives each thread the same x offset and KX values of jx in every pass
  // (jx = jx2 + k WY); its stores go to the compacted planes of the active (jx, jy), or nowhere
  constexpr int KX = UPB * WX / FW_THREADS;                // = WX / WY
  static_assert(KX >= 1 && KX * FW_THREADS == UPB * WX, "whole passes");
  const int jx2 = threadIdx.x / UPB, ux2 = threadIdx.x - jx2 * UPB;
  const size_t pstride = size_t(d.nz) * (ny / 2 + 1) * nx;
  float2* Urow = d.U + (size_t(z) * (ny / 2 + 1) + yy) * nx + ux2;
  __shared__ int jat[WX * WY];
  for (int e = threadIdx.x; e < WX * WY; e += blockDim.x) jat[e] = jmap[e];
  __syncthreads();
  // The products are centrosymmetric in w, P(w) = G(y - w) G(y + w) = P(-w), so the
  // x-transform of window row +wy is that of row -wy at the reversed offset wavenumber,
  // plus the one product the window does not hold (w_x = +WX/2 against -WX/2):
  //   A_{+wy}(j) = A_{-wy}(-j) + (-1)^j [P(WX/2, -wy) - P(-WX/2, -wy)];
  // the thread of row -wy (wy = 1 .. WY/2 - 1) writes both rows, row +wy's thread idles.
  for (int x0 = 0; x0 < nx; x0 += UPB) {
    {
      const int iwy = threadIdx.x / UPB, ux = threadIdx.x - iwy * UPB, x = x0 + ux;   // lanes over x
      const int wyv = iwy - WY / 2;
      const bool derived = WY >= 4 && wyv >= 1;
      if (x < nx && !derived) {
        const float2* Gm = Grow + (WY / 2 - wyv) * nx;    // row yy - wy
        const float2* Gp = Grow + (WY / 2 + wyv) * nx;    // row yy + wy
        float2 a[WX];
#pragma unroll
        for (int ix = 0; ix < WX; ++ix) {
          const int wxv = ix - WX / 2;
          const float2 p = Gm[(x - wxv + nx) & (nx - 1)] * Gp[(x + wxv + nx) & (nx - 1)];
          a[ix] = neg_if(p, WX >= 2 && (ix & 1));
        }
        const bool source = WY >= 4 && wyv < 0 && wyv > -WY / 2;
        float2 cr = make_float2(0.f, 0.f);
        if (source)                                       // a[0] = P(-WX/2, wy), unsigned
          cr = Gm[(x - WX / 2 + nx) & (nx - 1)] * Gp[(x + WX / 2 + nx) & (nx - 1)] - a[0];
        reg_dft<WX>(a);
#pragma unroll
        for (int jx = 0; jx < WX; ++jx) a[jx] = neg_if(a[jx], WX >= 2 && ((jx & 1) != alt_sign_end(WX)));
#pragma unroll
        for (int jx = 0; jx < WX; ++jx) ex[L::at(jx, ux, iwy)] = a[jx];
        if (source) {
          const int iwd = WY / 2 - wyv;                   // row +wy
#pragma unroll
          for (int jx = 0; jx < WX; ++jx)
            ex[L::at(jx, ux, iwd)] = a[(WX - jx) & (WX - 1)] + neg_if(cr, ((jx + WX / 2) & 1) != 0);
        }
      }
    }
    __syncthreads();
    if (x0 + ux2 < nx) {                                   // consecutive threads: consecutive x
#pragma unroll
      for (int k = 0; k < KX; ++k) {
        float2 b[WY];
#pragma unroll
        for (int iwy = 0; iwy < WY; ++iwy)
          b[iwy] = neg_if(ex[L::at(jx2 + k * WY, ux2, iwy)], WY >= 2 && (iwy & 1));
        reg_dft<WY>(b);
#pragma unroll
        for (int jy = 0; jy < WY; ++jy) {
          const int ja = jat[jy * WX + jx2 + k * WY];
          if (ja >= 0) Urow[ja * pstride + x0] = neg_if(b[jy], WY >= 2 && ((jy & 1) != alt_sign_end(WY)));
        }
      }
    }
    __syncthreads();
  }
}

// M(k_m; f, j, z) for ZC consecutive depths of one j: a cluster of ZC CTAs, one (j, z) plane
// each (2D FFT of U_j in shared memory; a grid plane as the centrosymmetric half plane, two
// CTAs per SM); then every CTA takes a share of the kept rows of
// (f, j) and reads the ZC depths of each from the cluster's planes (distributed shared
// memory), so each row's depths z0..z0+ZC-1 are written together (8 ZC contiguous bytes).
// ZC: depths per cluster, 2, 4 or 8 (the autotuner's choice).
template <int PX, int PY, int ZC>
__global__ void __cluster_dims__(1, ZC, 1) __launch_bounds__(mrows_threads<PY>(), PY > 0 ? 2 : 1)
fa_mrows_kernel(Dev d, int f, float2 cf) {
  namespace cg = cooperative_groups;
  constexpr int NX = 32 * PX, NY = PY > 0 ? 32 * PY : 1, LD = plane_ld(NX);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  float2* tws = s + (PY > 0 ? sym_plane_words(NX) : plane_words(NX, NY));
  cg::cluster_group cluster = cg::this_cluster();
  // blockIdx.x: position among the frequency's active offset wavenumbers
  const int ja = blockIdx.x, j = d.jact[size_t(f) * d.W + ja];
  const int z = blockIdx.y, rank = int(cluster.block_rank()), z0 = z - rank;
  if (z < d.nz) {                        // every CTA reaches both cluster barriers below
    constexpr int NYH = NY / 2 + 1;      // stored rows of the centrosymmetric plane
    const float2* P = d.U + (size_t(ja) * d.nz + z) * (NYH * NX);
    if constexpr (PY > 0) {
      static_assert(PX == PY, "square planes");
      plane_twiddles(tws, d.tw32, NX);
      __syncthreads();
      sym_plane_fft2<PX, +1>(s, LD, tws, P);
    } else {
      plane_twiddles(tws, d.tw32, NX);
      load_plane<NX, NY, LD, mrows_threads<PY>()>(s, P);
      __syncthreads();
      plane_fft2<PX, PY, +1>(s, LD, d.tw32, tws);
    }
  }
  cluster.sync();
  const float2* ps[ZC];
#pragma unroll
  for (int k = 0; k < ZC; ++k) ps[k] = cluster.map_shared_rank(s, k);
  const int e0 = d.fj_off[f * d.W + j], e1 = d.fj_off[f * d.W + j + 1];
  const int n = e1 - e0, per = (n + ZC - 1) / ZC;
  const int a0 = e0 + rank * per, a1 = min(e1, a0 + per);
  for (int e = a0 + threadIdx.x; e < a1; e += blockDim.x) {
    const int2 ent = d.fj_ent[e];
    const int y = ent.x / NX, x = ent.x - y * NX;
    const int off = PY > 0 ? sym_addr<NX>(y, x, LD) : paddr(y, x, LD);
    float2 v[ZC];
#pragma unroll
    for (int k = 0; k < ZC; ++k) v[k] = z0 + k < d.nz ? cf * ps[k][off] : make_float2(0.f, 0.f);
    float2* dst = d.A32 + size_t(ent.y) * d.nzs + z0;
    if (z0 + ZC <= d.nzs) {
#pragma unroll
      for (int k = 0; k < ZC; k += 2)
        reinterpret_cast<float4*>(dst)[k / 2] = make_float4(v[k].x, v[k].y, v[k + 1].x, v[k + 1].y);
    } else {
#pragma unroll
      for (int k = 0; k < ZC; ++k) if (z0 + k < d.nzs) dst[k] = v[k];
    }
  }
  cluster.sync();                        // peers may still read this CTA's plane
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
__global__ void __launch_bounds__(plane_threads<PY>()) fa_drhs_kernel(Dev d) {
  constexpr int NX = 32 * PX, NY = PY > 0 ? 32 * PY : 1, LD = plane_ld(NX);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  const int j = blockIdx.x, f = blockIdx.y;
  float2* tws = s + plane_words(NX, NY);
  const float2* P = d.Dw + (size_t(f) * d.W + j) * (NX * NY);
  plane_twiddles(tws, d.tw32, NX);
  if (PY > 0) {
    __syncthreads();
    plane_fft2<PX, PY, -1>(s, LD, d.tw32, tws, P);
  } else {
    load_plane<NX, NY, LD, plane_threads<PY>()>(s, P);
    __syncthreads();
    plane_fft2<PX, PY, -1>(s, LD, d.tw32, tws);
  }
  const int e0 = d.fj_off[f * d.W + j], e1 = d.fj_off[f * d.W + j + 1];
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int2 ent = d.fj_ent[e];
    const int y = ent.x / NX, x = ent.x - y * NX;
    const int ny2 = (NY - y) % NY, nx2 = (NX - x) % NX;
    const float2 a = s[paddr(y, x, LD)], b = s[paddr(ny2, nx2, LD)];
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
    g.rp = unsigned(t);
    g.rq = unsigned(d.ones_row);
    g.bp = (unsigned long long)t * d.nzs * sizeof(float2);
    g.bq = (unsigned long long)d.ones_row * d.nzs * sizeof(float2);
    g.sw = 1.f;
    g.pad = 0.f;
    d.gent[t] = g;
  }
  if (t < d.nz) d.A32[size_t(d.ones_row) * d.nzs + t] = make_float2(1.f, 0.f);
}

template <int WX, int WY>
size_t u_smem(int nx) { return (size_t(ExLayout<WX, WY>::SIZE) + size_t(WY + 1) * nx) * sizeof(float2); }

template <int PX, int PY>
size_t plane_smem() { return size_t(plane_words(32 * PX, PY > 0 ? 32 * PY : 1) + 32 * PX) * sizeof(float2); }
template <int PX, int PY>
size_t mrows_smem() {
  return PY > 0 ? size_t(sym_plane_words(32 * PX) + 32 * PX) * sizeof(float2) : plane_smem<PX, PY>();
}

template <int PX, int PY>
cudaError_t rows_for(const Dev& d, int f, int nact, float2 cf, cudaStream_t s) {
  if (nact == 0) return cudaSuccess;     // no kept row at this frequency
  const size_t sm = plane_smem<PX, PY>();
  fa_gspace_kernel<PX, PY><<<d.nz, plane_threads<PY>(), sm, s>>>(d, f);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 gu(d.ny / 2 + 1, d.nz);
  switch (d.wx * 32 + d.wy) {
#define FA_U(WX, WY) case WX * 32 + WY: fa_u_kernel<WX, WY><<<gu, FW_THREADS, u_smem<WX, WY>(d.N), s>>>(d, f); break;
    FA_U(1, 1) FA_U(2, 1) FA_U(4, 1) FA_U(8, 1) FA_U(16, 1)
    FA_U(2, 2) FA_U(4, 4) FA_U(8, 8) FA_U(16, 16) FA_U(4, 2) FA_U(8, 4) FA_U(16, 8)
#undef FA_U
    default: return cudaErrorInvalidValue;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int zc = d.tune_zc;
  const dim3 gm(nact, (d.nz + zc - 1) / zc * zc);
  const size_t smr = mrows_smem<PX, PY>();
  if (zc == 2) fa_mrows_kernel<PX, PY, 2><<<gm, mrows_threads<PY>(), smr, s>>>(d, f, cf);
  else if (zc == 8) fa_mrows_kernel<PX, PY, 8><<<gm, mrows_threads<PY>(), smr, s>>>(d, f, cf);
  else fa_mrows_kernel<PX, PY, 4><<<gm, mrows_threads<PY>(), smr, s>>>(d, f, cf);
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
  const int smr = int(mrows_smem<PX, PY>());
  if ((e = cudaFuncSetAttribute(fa_mrows_kernel<PX, PY, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smr)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(fa_mrows_kernel<PX, PY, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smr)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(fa_mrows_kernel<PX, PY, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smr)) != cudaSuccess) return e;
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

cudaError_t launch_fa_rows(const Dev& d, int f, int nact, double2 cf, cudaStream_t s) {
  const float2 c = make_float2(float(cf.x), float(cf.y));
  const int px = d.N / 32, py = d.ny == 1 ? 0 : d.ny / 32;
#define FA_R(PX, PY) if (px == PX && py == PY) return rows_for<PX, PY>(d, f, nact, c, s);
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
    fa_drhs_kernel<PX, PY><<<dim3(d.W, d.nf), plane_threads<PY>(), plane_smem<PX, PY>(), s>>>(d); \
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
