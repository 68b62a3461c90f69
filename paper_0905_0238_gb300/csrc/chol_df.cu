// Damped normal-equation solves (G + lam I) x_+- = b_+-, lam = alpha * trace(G), with the
// factorisation carried in double-float arithmetic on the FP32 pipes.
//
// GB300 runs FP64 at 1/59 of the FP32 rate, so an FP64 Cholesky of 257 systems of 256
// unknowns is bound by the FP64 pipe.  Here every value of the working matrix is held as an
// unevaluated sum h + l of two floats (about 48 significant bits), in place of the FP64
// matrix (the same 8 bytes per element), and the n^3/3 multiply-adds run on the FP32 pipes
// with error-free transformations: each product a_h b_h is split exactly by fma (Dekker's
// TwoProduct with a hardware fma), each addition's rounding error is captured by Knuth's
// TwoSum, and the low parts collect the errors and the cross terms; the pivots' reciprocal
// square roots take an FP32 estimate and one Newton step in double-float.  No FP64 arithmetic
// remains in the factorisation.
//
// Blocked right-looking form over all subproblems at once, so that every step fills the GPU
// (one CTA per subproblem would leave the serial parts of each factorisation on its SM's
// critical path and 257 systems unevenly spread over 152 SMs):
//   * the Gram reduction has written the lower triangle of G + lam I in double-float;
//   * cdf_diag factors and inverts the first 32 x 32 diagonal block of every subproblem
//     (df_diag_block: 256 threads, one barrier per column); per 32-column step cdf_panel
//     multiplies the panel rows by the inverse (x = a L_kk^-T, independent outputs) and
//     cdf_update subtracts P P^T from the trailing lower triangle in 64 x 64 tiles of every
//     subproblem (the panel staged transposed in shared memory, each thread a 4 x 4 interleaved
//     register tile), its tile-(0, 0) CTAs, first in the launch, going on to factor and invert
//     the next diagonal block;
//   * look-ahead: the update of the tile column holding the next diagonal block and panel runs
//     first, and the rest of the update runs on a second stream while the next diagonal block
//     and panel proceed (the latency-bound small launches overlap the throughput-bound tiles);
//   * cdf_final: forward and backward substitution for both right-hand sides in
//     double-float, each diagonal block by its inverse; the factor stays in double-float (the re-solve of the inversion adjoint
//     and the factor export read the pairs), its high parts are written as the FP32 copy for
//     the refinement's correction solves.
// A non-positive or non-finite pivot marks the subproblem EDT_ENOTPD and zeroes its solution.
#include "edt_internal.h"
#include "dfloat.cuh"
#include "blksolve.cuh"
#include "tc_ptx.cuh"

namespace edt {

namespace {

constexpr int FB = 32, FLD = FB + 1, FTHREADS = 256;
constexpr int UT = 64, ULD = UT + 1;   // update tile and its padded shared row

__device__ __forceinline__ bool has_rows(const Dev& d, int m) { return d.row_off[m + 1] > d.row_off[m]; }

// First diagonal block of every subproblem, factored and inverted in double-float (see
// df_diag_block); the later ones are factored by the update launches.  Sets the status and
// the trace slot, which holds lam from here on.
__global__ void __launch_bounds__(256) cdf_diag_kernel(Dev d) {
  __shared__ DfDiagScratch sh;
  const int m = blockIdx.x, n = d.nz;
  if (!has_rows(d, m)) return;
  float2* A = reinterpret_cast<float2*>(d.G + size_t(m) * n * n);
  const bool ok = df_diag_block(A, d.L32 ? d.L32 + size_t(m) * n * n : nullptr, d.dinv + size_t(m) * n,
                                d.dinv32 ? d.dinv32 + size_t(m) * n : nullptr, d.status + m, n, 0, sh);
  if (ok && threadIdx.x == 0) {
    d.trace[m] = d.alpha * d.trace[m];
    d.status[m] = EDT_OK;
  }
}

// Panel rows r0 .. r0 + 31 of subproblem blockIdx.y: x = a L_kk^-T = a X^T, x_j = sum_{l <= j}
// a_l X_jl, all outputs independent.  Warp h of four computes the outputs j = h (mod 4) of all
// 32 rows (lane = row): the rows sit transposed in shared memory (conflict-free), X is read by
// broadcast.
__global__ void __launch_bounds__(128) cdf_panel_kernel(Dev d, int k0) {
  __shared__ float2 sA[FB * FLD], sX[FB * FLD];
  const int m = blockIdx.y, n = d.nz;
  if (!has_rows(d, m) || d.status[m] != EDT_OK) return;
  const int lane = threadIdx.x & 31, h = threadIdx.x >> 5;
  float2* A = reinterpret_cast<float2*>(d.G + size_t(m) * n * n);
  const int r0 = k0 + FB + blockIdx.x * 32, nr = min(32, n - r0);
  {
    constexpr int Q = FB / 4;
    float2 av[Q], xv[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int r = h + 4 * q;                      // a warp: one row's 32 columns (coalesced)
      av[q] = r < nr ? A[size_t(r0 + r) * n + k0 + lane] : make_float2(0.f, 0.f);
      // X_{r, lane} from the upper triangle (at (lane, r)); the diagonal from dinv
      xv[q] = lane < r ? A[size_t(k0 + lane) * n + k0 + r]
                       : (lane == r ? df_of(d.dinv[size_t(m) * n + k0 + r]) : make_float2(0.f, 0.f));
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int r = h + 4 * q;
      sA[lane * FLD + r] = av[q];
      sX[r * FLD + lane] = xv[q];
    }
  }
  __syncthreads();
  float2 out[FB / 4];
#pragma unroll
  for (int q = 0; q < FB / 4; ++q) {
    const int j = h + 4 * q;
    float2 acc = make_float2(0.f, 0.f);
    for (int l = 0; l <= j; ++l) df_acc(acc, sA[l * FLD + lane], sX[j * FLD + l]);
    out[q] = df_norm(acc);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < FB / 4; ++q) sA[(h + 4 * q) * FLD + lane] = out[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < FB / 4; ++q) {
    const int r = h + 4 * q;
    if (r < nr) {
      const float2 v = sA[lane * FLD + r];
      A[size_t(r0 + r) * n + k0 + lane] = v;
      if (d.L32) d.L32[size_t(m) * n * n + size_t(r0 + r) * n + k0 + lane] = v.x;   // FP32 copy
    }
  }
}

// Trailing update of step k0: tile (I, J), I >= J, of 64 x 64 elements of the lower triangle
// of rows / columns t0 = k0 + 32 .. n - 1 of subproblem blockIdx.y loses P_I P_J^T, P the
// step's panel.  Thread (ty, tx) owns rows ty + 16 u and columns tx + 16 v (u, v < 4):
// interleaved, so the shared panel reads are conflict-free and the global rows coalesced.
// part 0: every tile; 1: the first tile column J = 0 (it holds the next step's diagonal block
// and panel); 2: the tiles J >= 1.  Parts 0 and 1 also factor the next step's diagonal block:
// the CTA of tile (0, 0), which holds that block and is its only writer, does so after its own
// update, and those CTAs come first in the launch (1D grid: CTA t < nsub takes tile 0 of
// subproblem t, the others follow) so that the factorisations overlap the remaining tiles.
union UpdateSmem {
  struct { float2 I[FB * ULD], J[FB * ULD]; } p;  // transposed panel rows: [l][i]
  DfDiagScratch dg;
};
__global__ void __launch_bounds__(256) cdf_update_kernel(Dev d, int k0, int part) {
  __shared__ UpdateSmem sm;
  float2* sI = sm.p.I;
  float2* sJ = sm.p.J;
  const int n = d.nz;
  int m, pt;
  if (part == 2) {
    m = blockIdx.y;
    pt = blockIdx.x;
  } else if (int(blockIdx.x) < d.nsub) {
    m = blockIdx.x;
    pt = 0;
  } else {
    m = (blockIdx.x - d.nsub) % d.nsub;
    pt = 1 + (blockIdx.x - d.nsub) / d.nsub;
  }
  if (!has_rows(d, m) || d.status[m] != EDT_OK) return;
  const int t0 = k0 + FB;
  int I, J;
  if (part == 1) {
    I = pt; J = 0;
  } else {
    I = int((sqrtf(8.0f * pt + 1.0f) - 1.0f) * 0.5f);
    while (I * (I + 1) / 2 > pt) --I;
    while ((I + 1) * (I + 2) / 2 <= pt) ++I;
    J = pt - I * (I + 1) / 2;
    if (part == 2) { ++I; ++J; }
  }
  const int r0 = t0 + UT * I, c0 = t0 + UT * J;
  float2* A = reinterpret_cast<float2*>(d.G + size_t(m) * n * n);
  {
    constexpr int NL = UT * FB / 256;              // 8 elements of each panel per thread
    float2 vi[NL], vj[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + 256 * q, i = e / FB, l = e - i * FB;   // a warp: one row's 32 columns
      vi[q] = r0 + i < n ? A[size_t(r0 + i) * n + k0 + l] : make_float2(0.f, 0.f);
      vj[q] = c0 + i < n ? A[size_t(c0 + i) * n + k0 + l] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + 256 * q, i = e / FB, l = e - i * FB;
      sI[l * ULD + i] = vi[q];
      sJ[l * ULD + i] = vj[q];
    }
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool diag = I == J;
  float2 acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = make_float2(0.f, 0.f);
  for (int l = 0; l < FB; ++l) {
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
      const int i = r0 + ty + 16 * u, j = c0 + tx + 16 * v;
      if (i < n && j <= i && !(diag && u < v)) {
        float2* a = A + size_t(i) * n + j;
        *a = df_add(*a, df_neg(df_norm(acc[u][v])));
      }
    }
  if (part != 2 && pt == 0) {                      // the same in every thread of the CTA
    __syncthreads();                               // the tile's writes visible, panels released
    df_diag_block(A, d.L32 ? d.L32 + size_t(m) * n * n : nullptr, d.dinv + size_t(m) * n,
                  d.dinv32 ? d.dinv32 + size_t(m) * n : nullptr, d.status + m, n, t0, sm.dg);
  }
}

// ---- trailing updates on the tensor cores: error-free BF16 slices (Ozaki scheme) ----------
// Tile of 128 rows (I) x 64 columns (J) of the trailing lower triangle: C -= P_I P_J^T with the
// step's double-float panel P (K = 32).  Each panel row r is scaled by 2^-E_r (|P_rk| < 2^E_r)
// and cut into eight signed 7-bit integer slices s_0..s_7 (P_rk = 2^E_r sum_i s_i 2^-7(i+1),
// to the double-float's precision), exact in BF16.  The slice products of one level
// l = i + j, summed over K = 32 and over the level's at most eight pairs, are integers below
// 2^22, so the FP32 accumulators in tensor memory hold them exactly: one accumulator of 64
// columns per level (8 x 64 = 512 columns).  The operands pack two slices per 128-byte row
// (K = 64): A tile u = [s_2u | s_2u+1], B tile c = [t_c | t_c-1], so one K = 64 product adds the
// two pairs (2u, l - 2u) and (2u + 1, l - 2u - 1) of level l: 20 products of K = 64 in all.
// The epilogue adds the levels from the smallest up in double-float, scales by
// 2^(E_r + E_c - 14) and subtracts from C.
constexpr int TCU_M = 128, TCU_N = 64, TCU_A = TCU_M * 128, TCU_B = TCU_N * 128;
constexpr int TCU_SMEM = 1024 + 4 * TCU_A + 8 * TCU_B;

__device__ __forceinline__ void tcu_tiles(int t, int& RT, int& CT) {
  RT = (t + TCU_M - 1) / TCU_M;
  CT = (t + TCU_N - 1) / TCU_N;
}
// number of tiles (I, J), J <= 2 I + 1, J < CT, of part 0 (all), 1 (J = 0) or 2 (J >= 1)
__host__ __device__ inline int tcu_count(int t, int part) {
  const int RT = (t + TCU_M - 1) / TCU_M, CT = (t + TCU_N - 1) / TCU_N;
  if (part == 1) return RT;
  int c = 0;
  for (int I = 0; I < RT; ++I) c += min(2 * I + 2, CT) - (part == 2 ? 1 : 0);
  return c;
}

__device__ __forceinline__ void tcu_put(unsigned char* tile, int row, int kk, float v) {
  *reinterpret_cast<__nv_bfloat16*>(tile + tcx::sw_off(row, kk >> 3) + (kk & 7) * 2) = __float2bfloat16_rn(v);
}

__global__ void __launch_bounds__(256) cdf_update_tc_kernel(Dev d, int k0, int part) {
  using namespace tcx;
  extern __shared__ __align__(1024) unsigned char tcu_raw[];
  __shared__ int sEA[TCU_M], sEB[TCU_N];
  __shared__ uint64_t done;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ DfDiagScratch dg;
  unsigned char* smA = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tcu_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* smB = smA + 4 * TCU_A;
  const int n = d.nz, t = n - k0 - FB, t0 = k0 + FB;
  int m, pt;
  if (part == 2) {
    m = blockIdx.y;
    pt = blockIdx.x;
  } else if (int(blockIdx.x) < d.nsub) {
    m = blockIdx.x;
    pt = 0;
  } else {
    m = (blockIdx.x - d.nsub) % d.nsub;
    pt = 1 + (blockIdx.x - d.nsub) / d.nsub;
  }
  if (!has_rows(d, m) || d.status[m] != EDT_OK) return;
  int I = 0, J = 0;
  {
    int RT, CT;
    tcu_tiles(t, RT, CT);
    if (part == 1) {
      I = pt;
    } else {
      int rem = pt;
      for (I = 0; I < RT; ++I) {
        const int j0 = part == 2 ? 1 : 0, j1 = min(2 * I + 2, CT);
        if (rem < j1 - j0) { J = j0 + rem; break; }
        rem -= j1 - j0;
      }
    }
  }
  const int r0 = t0 + TCU_M * I, c0 = t0 + TCU_N * J;
  float2* A = reinterpret_cast<float2*>(d.G + size_t(m) * n * n);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_slot, 512);
  // operands: every row's values loaded first (24 loads in flight per warp), then per row the
  // exponent and eight slices
  float2 va[TCU_M / 8], vb[TCU_N / 8];
#pragma unroll
  for (int q = 0; q < TCU_M / 8; ++q) {
    const int rg = r0 + warp + 8 * q;
    va[q] = rg < n ? A[size_t(rg) * n + k0 + lane] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int q = 0; q < TCU_N / 8; ++q) {
    const int cg = c0 + warp + 8 * q;
    vb[q] = cg < n ? A[size_t(cg) * n + k0 + lane] : make_float2(0.f, 0.f);
  }
  auto slice_row = [&](float2 a, int& E, float* sl) {
    float mx = fabsf(a.x);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    E = 0;
    if (mx > 0.f) frexpf(mx, &E);                   // mx < 2^E
    float vh = ldexpf(a.x, -E), vl = ldexpf(a.y, -E);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float th = vh * 128.f, tl = vl * 128.f;
      const float si = rintf(th);
      sl[i] = si;
      const float2 r = two_sum(th - si, tl);
      vh = r.x;
      vl = r.y;
    }
  };
#pragma unroll
  for (int q = 0; q < TCU_M / 8; ++q) {
    const int r = warp + 8 * q;
    int E;
    float sl[8];
    slice_row(va[q], E, sl);
#pragma unroll
    for (int i = 0; i < 8; ++i) tcu_put(smA + (i >> 1) * TCU_A, r, 32 * (i & 1) + lane, sl[i]);
    if (lane == 0) sEA[r] = E;
  }
#pragma unroll
  for (int q = 0; q < TCU_N / 8; ++q) {
    const int c = warp + 8 * q;
    int E;
    float sl[8];
    slice_row(vb[q], E, sl);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      tcu_put(smB + i * TCU_B, c, lane, sl[i]);
      if (i < 7) tcu_put(smB + (i + 1) * TCU_B, c, 32 + lane, sl[i]);
    }
    tcu_put(smB, c, 32 + lane, 0.f);
    if (lane == 0) sEB[c] = E;
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  if (threadIdx.x == 0) {
    const uint32_t idesc = idesc_bf16(TCU_M, TCU_N);
    const uint32_t a0 = smem_u32(smA), b0 = smem_u32(smB);
    for (int l = 0; l < 8; ++l)
      for (int u = 0; 2 * u <= l; ++u) {
        const uint32_t aa = a0 + uint32_t(u) * TCU_A, bb = b0 + uint32_t(l - 2 * u) * TCU_B;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(tmem + uint32_t(64 * l), sw128_desc(aa + 32 * kk), sw128_desc(bb + 32 * kk), idesc,
                   (u > 0 || kk > 0) ? 1u : 0u);
      }
    mma_commit(&done);
  }
  __syncwarp();
  const bool ok = mbar_wait(&done, 0u, &abort_flag);
  tc_fence_after();
  if (ok) {
    const int qd = warp & 3, h = warp >> 2;
    const int rr = 32 * qd + lane, rg = r0 + rr;
    for (int g = 0; g < 2; ++g) {
      const int cb = 32 * h + 16 * g;
      uint32_t v[8][16];                           // the eight levels' loads in flight together
#pragma unroll
      for (int l = 0; l < 8; ++l) tmem_ld16_nowait(tmem + (uint32_t(32 * qd) << 16) + uint32_t(64 * l + cb), v[l]);
      tmem_wait_ld();
      float hi[16], lo[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) { hi[c] = ldexpf(__uint_as_float(v[7][c]), -49); lo[c] = 0.f; }
#pragma unroll
      for (int l = 6; l >= 0; --l) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const float2 sm = two_sum(hi[c], ldexpf(__uint_as_float(v[l][c]), -7 * l));
          hi[c] = sm.x;
          lo[c] = __fadd_rn(lo[c], sm.y);
        }
      }
      if (rg < n) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int cg = c0 + cb + c;
          if (cg < n && cg <= rg) {
            const int e = sEA[rr] + sEB[cb + c] - 14;
            const float2 pv = df_norm(make_float2(ldexpf(hi[c], e), ldexpf(lo[c], e)));
            float2* a = A + size_t(rg) * n + cg;
            *a = df_add(*a, df_neg(pv));
          }
        }
      }
    }
  } else if (threadIdx.x == 0) {
    atomicOr(d.flags, 1u);                         // a tensor-core wait expired
    mbar_drain(&done, 0u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
  if (ok && part <= 1 && pt == 0) {                // the same in every thread of the CTA
    __syncthreads();
    df_diag_block(A, d.L32 ? d.L32 + size_t(m) * n * n : nullptr, d.dinv + size_t(m) * n,
                  d.dinv32 ? d.dinv32 + size_t(m) * n : nullptr, d.status + m, n, t0, dg);
  }
}

// Both substitutions and the solution; the factor stays in double-float (its readers take
// the pairs).  Its high parts, the FP32 copy for the refinement's correction solves, were
// written by the diagonal-block and panel kernels as each element became final.
__global__ void __launch_bounds__(FTHREADS) cdf_final_kernel(Dev d) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int m = blockIdx.x, n = d.nz;
  const size_t go = size_t(m) * n * n, vo = size_t(m) * n;
  float2* sb = reinterpret_cast<float2*>(smraw);            // [n][2]
  float2* sInv = sb + 2 * n;                                // [n]
  float2* sL = sInv + n;                                    // solve scratch
  double* xo = d.x + vo * 2;
  if (!has_rows(d, m)) {
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) xo[i] = 0.0;
    if (threadIdx.x == 0) { d.status[m] = EDT_OK; d.trace[m] = 0.0; }
    return;
  }
  if (d.status[m] != EDT_OK) {
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) xo[i] = 0.0;
    return;
  }
  const float2* A = reinterpret_cast<const float2*>(d.G + go);
  float* L32 = d.L32 ? d.L32 + go : nullptr;
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) sb[i] = df_of(d.b[vo * 2 + i]);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double inv = d.dinv[vo + i];
    sInv[i] = df_of(inv);
    if (L32) d.dinv32[vo + i] = float(inv);
  }
  __syncthreads();
  blk_solve_2rhs<DfArith, FTHREADS>(A, sInv, n, sb, sL);
  bool bad = false;
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) {
    const double v = df_val(sb[i]);
    xo[i] = v;
    if (!isfinite(v)) bad = true;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0 && bad) d.status[m] = EDT_ENONFINITE;
}

// x = (L L^T)^-1 b with the double-float factor of the last factorisation (no refactorisation):
// the inversion adjoint's re-solve.
__global__ void __launch_bounds__(FTHREADS) cdf_resolve_kernel(Dev d) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int m = blockIdx.x, n = d.nz;
  const size_t vo = size_t(m) * n;
  float2* sb = reinterpret_cast<float2*>(smraw);
  float2* sInv = sb + 2 * n;
  float2* sL = sInv + n;
  double* xo = d.x + vo * 2;
  if (!has_rows(d, m) || d.status[m] != EDT_OK) {
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) xo[i] = 0.0;
    return;
  }
  const float2* A = reinterpret_cast<const float2*>(d.G + size_t(m) * n * n);
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) sb[i] = df_of(d.b[vo * 2 + i]);
  for (int i = threadIdx.x; i < n; i += blockDim.x) sInv[i] = df_of(d.dinv[vo + i]);
  __syncthreads();
  blk_solve_2rhs<DfArith, FTHREADS>(A, sInv, n, sb, sL);
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) xo[i] = df_val(sb[i]);
}

// The double-float factor as FP64 [nsub][n][n] (lower triangle) into out.
__global__ void cdf_export_kernel(Dev d, double* out) {
  const size_t total = size_t(d.nsub) * d.nz * d.nz;
  const float2* A = reinterpret_cast<const float2*>(d.G);
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += size_t(gridDim.x) * blockDim.x) {
    const size_t r = e % (size_t(d.nz) * d.nz);
    const int i = int(r / d.nz), j = int(r - size_t(i) * d.nz);
    out[e] = j <= i ? df_val(A[e]) : 0.0;
  }
}

size_t cdf_final_smem(int n) { return size_t(3 * n + blk_solve_scratch<DfArith, FTHREADS>()) * sizeof(float2); }

}  // namespace

int chol_dfloat_launches(int n) {
  int k = 2;                                        // the first diagonal block, the final solve
  for (int k0 = 0; k0 + FB < n; k0 += FB) {
    const int nt = (n - k0 - FB + UT - 1) / UT;
    k += 1 + (nt < 2 ? 1 : 2);                      // panel, update (one or two parts; the next
  }                                                 // diagonal block inside the first)
  return k;
}

cudaError_t prepare_chol_dfloat(const Dev& d) {
  cudaError_t e = cudaFuncSetAttribute(cdf_final_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(cdf_final_smem(d.nz)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(cdf_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TCU_SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(cdf_resolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(cdf_final_smem(d.nz)));
}

cudaError_t launch_chol_dfloat_resolve(const Dev& d, cudaStream_t s) {
  cdf_resolve_kernel<<<d.nsub, FTHREADS, cdf_final_smem(d.nz), s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_chol_dfloat_export(const Dev& d, double* out, cudaStream_t s) {
  cdf_export_kernel<<<4 * 152, 256, 0, s>>>(d, out);
  return cudaGetLastError();
}

cudaError_t launch_chol_dfloat(const Dev& d, int trace_mode, cudaStream_t s, const CholLookahead* la) {
  (void)trace_mode;                       // the Gram reduction has added lam = alpha * trace
  const int n = d.nz;
  const int nsteps = (n + FB - 1) / FB;
  const bool ahead = la && la->side && la->nev >= 2 * nsteps + 1;
  cudaError_t e;
  // Look-ahead on two streams: step k's update of the tile column J = 0 runs on s, followed by
  // the next diagonal block and panel (which read only that column); the update of the tiles
  // J >= 1 runs on the side stream meanwhile.  Step k + 1's updates wait for it.
  cudaEvent_t prev_rest = nullptr;
  // The diagonal block of step 0 has a launch of its own; every later one is factored by the
  // previous step's update (parts 0 and 1) as soon as its tile is final.
  cdf_diag_kernel<<<d.nsub, 256, 0, s>>>(d);
  for (int step = 0, k0 = 0; k0 + FB < n; ++step, k0 += FB) {
    const int t = n - k0 - FB, nt = (t + UT - 1) / UT;
    cdf_panel_kernel<<<dim3((t + 31) / 32, d.nsub), 128, 0, s>>>(d, k0);
    if (d.chol_tc) {                               // tensor-core updates: tiles of 128 x 64
      const int ct = (t + TCU_N - 1) / TCU_N;
      if (!ahead || ct < 2) {
        if (prev_rest && (e = cudaStreamWaitEvent(s, prev_rest, 0)) != cudaSuccess) return e;
        prev_rest = nullptr;
        cdf_update_tc_kernel<<<unsigned(tcu_count(t, 0) * d.nsub), 256, TCU_SMEM, s>>>(d, k0, 0);
        continue;
      }
      cudaEvent_t ev_panel = la->ev[2 * step], ev_rest = la->ev[2 * step + 1];
      if ((e = cudaEventRecord(ev_panel, s)) != cudaSuccess) return e;
      if (prev_rest && (e = cudaStreamWaitEvent(s, prev_rest, 0)) != cudaSuccess) return e;
      cdf_update_tc_kernel<<<unsigned(tcu_count(t, 1) * d.nsub), 256, TCU_SMEM, s>>>(d, k0, 1);
      if ((e = cudaStreamWaitEvent(la->side, ev_panel, 0)) != cudaSuccess) return e;
      cdf_update_tc_kernel<<<dim3(tcu_count(t, 2), d.nsub), 256, TCU_SMEM, la->side>>>(d, k0, 2);
      if ((e = cudaEventRecord(ev_rest, la->side)) != cudaSuccess) return e;
      prev_rest = ev_rest;
      continue;
    }
    if (!ahead || nt < 2) {
      if (prev_rest && (e = cudaStreamWaitEvent(s, prev_rest, 0)) != cudaSuccess) return e;
      prev_rest = nullptr;
      cdf_update_kernel<<<unsigned(nt * (nt + 1) / 2 * d.nsub), 256, 0, s>>>(d, k0, 0);
      continue;
    }
    cudaEvent_t ev_panel = la->ev[2 * step], ev_rest = la->ev[2 * step + 1];
    if ((e = cudaEventRecord(ev_panel, s)) != cudaSuccess) return e;
    if (prev_rest && (e = cudaStreamWaitEvent(s, prev_rest, 0)) != cudaSuccess) return e;
    cdf_update_kernel<<<unsigned(nt * d.nsub), 256, 0, s>>>(d, k0, 1);
    if ((e = cudaStreamWaitEvent(la->side, ev_panel, 0)) != cudaSuccess) return e;
    cdf_update_kernel<<<dim3(nt * (nt - 1) / 2, d.nsub), 256, 0, la->side>>>(d, k0, 2);
    if ((e = cudaEventRecord(ev_rest, la->side)) != cudaSuccess) return e;
    prev_rest = ev_rest;
  }
  if (prev_rest && (e = cudaStreamWaitEvent(s, prev_rest, 0)) != cudaSuccess) return e;
  cdf_final_kernel<<<d.nsub, FTHREADS, cdf_final_smem(n), s>>>(d);
  return cudaGetLastError();
}

}  // namespace edt
