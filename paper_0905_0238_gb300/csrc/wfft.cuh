// Register-resident FP32 FFTs of one line per warp, shared by the data transforms.
//
// Two forms of the length-N discrete Fourier transform X[k] = sum_n x[n] W^{nk},
// W = e^{sign 2 pi i / N}, each held in P = N / 32 registers per lane:
//
//  * warp_fft<P> (any N = 32 P): lane b holds x[32 a + b] in register a; (1) a P-point DFT
//    over a in registers (radix 2, bit-reversed register order fixed at compile time),
//    (2) the twiddle W^{b k1}, (3) a 32-point decimation-in-frequency DFT across the lanes
//    by shuffles.  Lane l then holds X[k1 + P * bitrev5(l)] in register k1.
//
//  * Fft512 (N = 512 = 8 * 8 * 8): three radix-8 passes in registers with two exchanges
//    through a per-warp shared-memory buffer.  Writing n = 64 n3 + 8 n2 + n1 and
//    k = k1 + 8 k2 + 64 k3, pass 1 takes the 8-point DFTs over n3, pass 2 applies
//    W_64^{n2 k1} and takes the DFTs over n2, pass 3 applies W_512^{n1 (k1 + 8 k2)} and
//    takes the DFTs over n1 (decimation in time, digit by digit).  Register j = 8 h + t of
//    lane l holds x[l + 32 h + 64 t] on entry and X[l + 32 h + 64 t] on exit, so loads and
//    stores of a line are both coalesced.  Twiddles W^t, t < 8, are formed from three table
//    reads (W, W^2, W^4).  Far fewer instructions per line than warp_fft<16>, whose
//    cross-lane stages spend two shuffles and a select per value per stage.
#pragma once

#include <cuda_runtime.h>
#include "cplx.cuh"

namespace edt {

__host__ __device__ constexpr int clog2(int n) { return n <= 1 ? 0 : 1 + clog2(n / 2); }
__device__ __forceinline__ int rbits(int x, int bits) {     // bit reversal of the low `bits` bits
  return bits == 0 ? 0 : int(__brev(unsigned(x)) >> (32 - bits));
}

__device__ __forceinline__ float2 tw_at(const float2* tw, int e, int N) {   // W_N^e, 0 <= e < N
  if (e < (N >> 1)) return tw[e];
  const float2 w = tw[e - (N >> 1)];
  return make_float2(-w.x, -w.y);
}

template <int P>
__device__ __forceinline__ void warp_fft(float2 (&r)[P], const float2* tw, int N, int sign, int lane) {
  constexpr int LP = clog2(P);
  float2 t[P];
#pragma unroll
  for (int a = 0; a < P; ++a) t[rbits(a, LP)] = r[a];
#pragma unroll
  for (int st = 0; st < LP; ++st) {                         // half-size h = 2^st
#pragma unroll
    for (int b = 0; b < P / 2; ++b) {
      const int h = 1 << st;
      const int jj = b & (h - 1), i0 = ((b >> st) << (st + 1)) + jj, i1 = i0 + h;
      float2 w = tw[jj * (N >> (st + 1))];                  // W_{2h}^jj
      if (sign > 0) w.y = -w.y;
      const float2 u = t[i0], v = t[i1] * w;
      t[i0] = u + v;
      t[i1] = u - v;
    }
  }
#pragma unroll
  for (int k1 = 1; k1 < P; ++k1) {                          // W_N^{lane k1}
    float2 w = tw_at(tw, (lane * k1) & (N - 1), N);
    if (sign > 0) w.y = -w.y;
    t[k1] = t[k1] * w;
  }
#pragma unroll
  for (int sh = 4; sh >= 0; --sh) {                         // cross-lane DIF, span 2^sh
    const int j = lane & ((1 << sh) - 1);
    float2 w = tw[j * (N >> (sh + 1))];                     // W_{2^(sh+1)}^j
    if (sign > 0) w.y = -w.y;
    const bool upper = (lane >> sh) & 1;
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      float2 u;
      u.x = __shfl_xor_sync(0xffffffffu, t[k1].x, 1 << sh);
      u.y = __shfl_xor_sync(0xffffffffu, t[k1].y, 1 << sh);
      t[k1] = upper ? (u - t[k1]) * w : t[k1] + u;
    }
  }
#pragma unroll
  for (int a = 0; a < P; ++a) r[a] = t[a];
}

// ---- radix-8 building blocks -------------------------------------------------------------

// i * SG * v (multiplication by W_4 = e^{SG pi i / 2})
template <int SG> __device__ __forceinline__ float2 rot4(float2 v) {
  return SG < 0 ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
}

// In-place 8-point DFT, X[k] = sum_n a[n] e^{SG 2 pi i n k / 8}, natural order in and out:
// 2-point DFTs over (n, n + 4), 4-point DFTs of the even and odd halves, one radix-2 merge.
template <int SG> __device__ __forceinline__ void dft8(float2 (&a)[8]) {
  constexpr float c = 0.70710678118654752f;
  const float2 b0 = a[0] + a[4], b1 = a[0] - a[4];
  const float2 b2 = a[2] + a[6], b3 = a[2] - a[6];
  const float2 b4 = a[1] + a[5], b5 = a[1] - a[5];
  const float2 b6 = a[3] + a[7], b7 = a[3] - a[7];
  const float2 e0 = b0 + b2, e2 = b0 - b2, e1 = b1 + rot4<SG>(b3), e3 = b1 - rot4<SG>(b3);
  const float2 o0 = b4 + b6, o2 = b4 - b6, o1 = b5 + rot4<SG>(b7), o3 = b5 - rot4<SG>(b7);
  // W_8^1 o1 and W_8^3 o3 with W_8 = (1 + SG i) / sqrt 2
  const float2 t1 = SG < 0 ? make_float2(c * (o1.x + o1.y), c * (o1.y - o1.x))
                           : make_float2(c * (o1.x - o1.y), c * (o1.x + o1.y));
  const float2 t3 = SG < 0 ? make_float2(c * (o3.y - o3.x), -c * (o3.x + o3.y))
                           : make_float2(-c * (o3.x + o3.y), c * (o3.x - o3.y));
  const float2 t2 = rot4<SG>(o2);
  a[0] = e0 + o0; a[4] = e0 - o0;
  a[1] = e1 + t1; a[5] = e1 - t1;
  a[2] = e2 + t2; a[6] = e2 - t2;
  a[3] = e3 + t3; a[7] = e3 - t3;
}

template <int SG> __device__ __forceinline__ float2 tw_sg(float2 w) {   // table entries are SG = -1
  return SG < 0 ? w : make_float2(w.x, -w.y);
}

struct Fft512 {
  static constexpr int N = 512, P = 16;
  static constexpr int SCRATCH = 568;                       // float2 per warp (pad1 range)
  // element index held by register j of lane l, on entry and on exit
  __device__ static __forceinline__ int idx(int l, int j) { return l + 32 * (j >> 3) + 64 * (j & 7); }
  // buffer layouts of the two exchanges, chosen so that every 16-lane phase of 8-byte
  // accesses in both directions touches 32 distinct banks
  __device__ static __forceinline__ int pad1(int e) { return e + 8 * (e >> 6); }
  __device__ static __forceinline__ int pad2(int e) { return e + (e >> 4); }

  // twiddle table in shared memory: W_512^e (sign -1) for 0 <= e < 512 at tpad(e), one pad
  // entry per 16 so that the strided reads of passes 2 and 3 hit distinct banks
  static constexpr int TWS = 512 + 32;
  __device__ static __forceinline__ int tpad(int e) { return e + (e >> 4); }

  // W^t for t = 1..7 from the table entries W, W^2, W^4 (four products, each at most two
  // roundings deep, instead of seven table reads)
  template <int SG>
  __device__ static __forceinline__ void powers(float2 (&w)[8], const float2* tws, int e) {
    w[1] = tw_sg<SG>(tws[tpad(e)]);
    w[2] = tw_sg<SG>(tws[tpad(2 * e)]);
    w[4] = tw_sg<SG>(tws[tpad(4 * e)]);
    w[3] = w[1] * w[2];
    w[5] = w[1] * w[4];
    w[6] = w[2] * w[4];
    w[7] = w[3] * w[4];
  }

  // tws: the twiddle table above; buf: SCRATCH float2 of this warp's shared memory.
  template <int SG>
  __device__ static __forceinline__ void run(float2 (&v)[16], float2* buf, const float2* tws, int l) {
    float2 a[8], w[8];
    __syncwarp();                                           // buf may still be read by the caller
    // pass 1: 8-point DFTs over n3 (stride 64) of the lines n1 + 8 n2 = l + 32 h
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int t = 0; t < 8; ++t) a[t] = v[8 * h + t];
      dft8<SG>(a);
#pragma unroll
      for (int t = 0; t < 8; ++t) buf[pad1(l + 32 * h + 64 * t)] = a[t];   // [k1][n2][n1]
    }
    __syncwarp();
    // pass 2: for (n1, k1) = (c & 7, c >> 3), c = l + 32 h: twiddle W_64^{n2 k1}, DFT over n2
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = l + 32 * h, n1 = c & 7, k1 = c >> 3;
      powers<SG>(w, tws, 8 * k1);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const float2 x = buf[pad1(n1 + 8 * t + 64 * k1)];
        a[t] = t == 0 ? x : x * w[t];
      }
      dft8<SG>(a);
#pragma unroll
      for (int t = 0; t < 8; ++t) v[8 * h + t] = a[t];                     // k2 = t
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int t = 0; t < 8; ++t) buf[pad2(l + 32 * h + 64 * t)] = v[8 * h + t];   // [k2][k1][n1]
    __syncwarp();
    // pass 3: for k1 + 8 k2 = l + 32 h: twiddle W_512^{n1 (k1 + 8 k2)}, DFT over n1
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int kk = l + 32 * h;
      powers<SG>(w, tws, kk);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const float2 x = buf[pad2(t + 8 * kk)];
        a[t] = t == 0 ? x : x * w[t];
      }
      dft8<SG>(a);
#pragma unroll
      for (int t = 0; t < 8; ++t) v[8 * h + t] = a[t];                     // X[kk + 64 t]
    }
  }
};

}  // namespace edt
