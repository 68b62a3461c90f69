// Substitutions L L^T x = b with a blocked Cholesky factor whose 32 x 32 diagonal blocks carry
// their inverses, for two right-hand sides at once, by one CTA.
//
// Layout of the factor: L lower, row-major with leading dimension n; the strict upper triangle
// of each diagonal block holds X = L_kk^-1 (X_il at (l, i)); the diagonal of X (1 / L_ii) is
// passed separately.  Every load of the factor is coalesced: lanes run across one row's 32
// columns of a block, warps across rows, and each warp keeps 16 row segments loading at once
// (the factor is usually read from DRAM, and one CTA per system must cover the latency with
// loads in flight).  Each block is one barrier-separated pass:
//   forward   t = b_blk - L[blk, 0:k0] y[0:k0]: one warp per row, lanes over the columns, a
//             shuffle butterfly for the dot product; then y_blk = X t (warp r: right-hand side r,
//             lane: row);
//   backward  t = y_blk - L[k0+kb:n, blk]^T x[k0+kb:n]: lane = column, warps over the rows,
//             the warps' partial sums added in warp order; then x_blk = X^T t.
// Every sum runs in a fixed order, so the result is bitwise reproducible.  Two arithmetic
// forms: double-float (float2 pairs, the factorisation's working precision) and FP32 (the
// refinement's correction solves with the factor's FP32 copy).
#pragma once
#include "dfloat.cuh"

namespace edt {

struct DfArith {
  using T = float2;
  static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void acc(T& s, T a, T b) { df_acc(s, a, b); }
  static __device__ __forceinline__ T add(T a, T b) { return df_add(a, b); }
  static __device__ __forceinline__ T sub(T a, T b) { return df_add(a, df_neg(b)); }
  static __device__ __forceinline__ T norm(T a) { return df_norm(a); }
  // the xor butterfly gives every lane the same sum: TwoSum's error term does not depend on
  // the order of its operands
  static __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      v = df_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
    return v;
  }
};

struct F32Arith {
  using T = float;
  static __device__ __forceinline__ T zero() { return 0.f; }
  static __device__ __forceinline__ void acc(T& s, T a, T b) { s = fmaf(a, b, s); }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
  static __device__ __forceinline__ T norm(T a) { return a; }
  static __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }
};

constexpr int BS_B = 32, BS_LD = 33;

// Shared scratch (elements of Ar::T): sX [32 * 33], red [NT / 32 * 2 * 32].
template <class Ar, int NT>
__host__ __device__ constexpr int blk_solve_scratch() { return BS_B * BS_LD + NT / 32 * 2 * BS_B; }

// Solves L L^T x = b in place: sb[i][r] (shared, [n][2]) holds b on entry and x on return.
// inv_diag: 1 / L_ii ([n], shared or global).  Called by all NT threads of the CTA.
template <class Ar, int NT>
__device__ void blk_solve_2rhs(const typename Ar::T* A, const typename Ar::T* inv_diag, int n,
                               typename Ar::T* sb, typename Ar::T* scratch) {
  using T = typename Ar::T;
  constexpr int NW = NT / 32;
  static_assert(NT % 32 == 0 && NW >= 2, "at least two warps");
  T* sX = scratch;                                          // [i][l] = X_il, l <= i
  T* red = scratch + BS_B * BS_LD;                          // [warp][r][lane]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nblk = (n + BS_B - 1) / BS_B;
  auto stage_x = [&](int k0, int kb) {
    for (int e = threadIdx.x; e < BS_B * BS_B; e += NT) {
      const int l = e >> 5, i = e & 31;                     // consecutive threads: consecutive i
      T v = Ar::zero();
      if (i < kb && l < kb) {
        if (l < i) v = A[size_t(k0 + l) * n + k0 + i];
        else if (l == i) v = inv_diag[k0 + i];
      }
      sX[i * BS_LD + l] = v;
    }
  };
  for (int bk = 0; bk < nblk; ++bk) {                       // forward: L y = b
    const int k0 = bk * BS_B, kb = min(BS_B, n - k0);
    stage_x(k0, kb);
    {
      // rows i = warp + NW q of the block; 4 column chunks of every row in flight at once, so
      // that a warp keeps 4 RPW row segments of 32 entries loading together
      constexpr int RPW = (BS_B + NW - 1) / NW;
      T s0[RPW], s1[RPW];
#pragma unroll
      for (int q = 0; q < RPW; ++q) { s0[q] = Ar::zero(); s1[q] = Ar::zero(); }
      const int nt = k0 / BS_B;                             // 32-column chunks left of the block
      for (int t0 = 0; t0 < nt; t0 += 4) {
        T a[4][RPW];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int q = 0; q < RPW; ++q) {
            const int i = warp + NW * q;
            a[u][q] = i < kb && t0 + u < nt ? A[size_t(k0 + i) * n + BS_B * (t0 + u) + lane] : Ar::zero();
          }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (t0 + u < nt) {
            const int l = BS_B * (t0 + u) + lane;
            const T y0 = sb[2 * l], y1 = sb[2 * l + 1];
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
              Ar::acc(s0[q], a[u][q], y0);
              Ar::acc(s1[q], a[u][q], y1);
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        const int i = warp + NW * q;
        if (i < kb) {                                         // the same in the whole warp
          const T r0 = Ar::warp_sum(Ar::norm(s0[q])), r1 = Ar::warp_sum(Ar::norm(s1[q]));
          if (lane == 0) {
            sb[2 * (k0 + i)] = Ar::sub(sb[2 * (k0 + i)], r0);
            sb[2 * (k0 + i) + 1] = Ar::sub(sb[2 * (k0 + i) + 1], r1);
          }
        }
      }
    }
    __syncthreads();
    if (warp < 2) {                                         // y_blk = X t
      T y = Ar::zero();
      if (lane < kb)
        for (int l = 0; l <= lane; ++l) Ar::acc(y, sX[lane * BS_LD + l], sb[2 * (k0 + l) + warp]);
      __syncwarp();
      if (lane < kb) sb[2 * (k0 + lane) + warp] = Ar::norm(y);
    }
    __syncthreads();
  }
  for (int bk = nblk - 1; bk >= 0; --bk) {                  // backward: L^T x = y
    const int k0 = bk * BS_B, kb = min(BS_B, n - k0);
    stage_x(k0, kb);
    T s0 = Ar::zero(), s1 = Ar::zero();
    if (lane < kb) {
      constexpr int U = 16;                                 // row segments in flight per warp
      for (int i0 = k0 + kb + warp; i0 < n; i0 += U * NW) {
        T a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) a[u] = i0 + NW * u < n ? A[size_t(i0 + NW * u) * n + k0 + lane] : Ar::zero();
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = i0 + NW * u;
          if (i < n) {
            Ar::acc(s0, a[u], sb[2 * i]);
            Ar::acc(s1, a[u], sb[2 * i + 1]);
          }
        }
      }
    }
    red[(warp * 2) * BS_B + lane] = Ar::norm(s0);
    red[(warp * 2 + 1) * BS_B + lane] = Ar::norm(s1);
    __syncthreads();
    if (warp < 2) {                                         // t, then x_blk = X^T t
      T t = Ar::zero();
      for (int w = 0; w < NW; ++w) t = Ar::add(t, red[(w * 2 + warp) * BS_B + lane]);
      if (lane < kb) sb[2 * (k0 + lane) + warp] = Ar::sub(sb[2 * (k0 + lane) + warp], t);
      __syncwarp();
      T x = Ar::zero();
      if (lane < kb)
        for (int i = lane; i < kb; ++i) Ar::acc(x, sX[i * BS_LD + lane], sb[2 * (k0 + i) + warp]);
      __syncwarp();
      if (lane < kb) sb[2 * (k0 + lane) + warp] = Ar::norm(x);
    }
    __syncthreads();
  }
}

}  // namespace edt
