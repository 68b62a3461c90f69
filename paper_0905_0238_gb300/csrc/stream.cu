// Streaming batches of independent 1D depth subproblems (one request = the split system of one
// midpoint wavenumber, eqs. DMV, M and Split of Section "Two dimensions", with its own layered
// reference, depth grid, frequencies and rows).  Request r solves, for real x_+ and x_- (nz),
//     min ||Ahat x_+- - dhat_+-||^2 + lam ||x_+-||^2,   lam = alpha trace(Ahat^T Ahat),
// Ahat = [Re a; Im a], a_i(z_j) = s_f g(k_p, z_j) g(k_q, z_j) for row i = (f, p, q).
//
// A batch of requests runs as eight stages, every launch covering all requests of the batch:
//   st_prep   per depth: layer index and the depth below its top as FP32 (hi, lo) pairs;
//   st_coef   per (request, f, k): vertical wavenumbers in FP64 (complex square root), the
//             reflectivity recursion of the depth march (upward for the reflection coefficients,
//             downward for the amplitudes) in FP32 with double-float phases;
//   st_eval   per (request, 8 (f, k) rows) x depth: the FP32 table sqrt|s_f| g(k, z);
//   st_tiles  per (request, 32 complex rows, 32 depths): the kernel rows |s_f| g_p g_q, split
//             into BF16 hi and lo and stored K-major in the 128-byte-swizzled layout the tensor
//             cores read (the unit phase of s_f moves onto the data, which leaves the
//             real-stacked problem unchanged); the data rows (d_+, d_-) follow the depth rows;
//             alpha trace(Ahat^T Ahat) accumulated from the unrounded FP32 rows;
//   st_gram   persistent tcgen05 kernel over (request, 128-depth tile pair) items: bulk copies
//             stage the hi/lo tiles, three BF16 MMAs per K step accumulate in tensor memory,
//             the epilogue writes the lower triangle of G (the FP32 accumulators as double-
//             float pairs (v, 0)) and b_+- = Ahat^T dhat_+- (FP64);
//   chol      double-float Cholesky of G + lam I in 32-column steps (a panel launch and a
//             64 x 64 tile update launch per step over every active request, so one large
//             factorisation spreads over many SMs), then the two solves (per-request size);
//   st_refine matrix-free residual Ahat^T (dhat - Ahat x), FP32 products, FP64 accumulation;
//   update    x += (LL^T)^-1 (r - lam x) with the FP32 copy of the factor.
// Every wait of the tensor-core kernel is bounded; on expiry it raises a device flag.
#include "edt_internal.h"
#include "cplx.cuh"
#include "tc_ptx.cuh"
#include "stream_internal.h"

namespace edt {

namespace {

using namespace tcx;

__device__ __forceinline__ int find_req(const long long* pre, int nreq, long long i) {
  int lo = 0, hi = nreq - 1;            // last request with pre[req] <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// unit phase of s_f = omega~^2 dz / dx (dz / dx > 0): omega~^2 / |omega~|^2
__device__ __forceinline__ float2 sf_phase(double f_hz, double eps) {
  const double wr = 2.0 * M_PI * f_hz;
  const double re = wr * wr - eps * eps, im = 2.0 * wr * eps;
  const double r = 1.0 / sqrt(re * re + im * im);
  return make_float2(float(re * r), float(im * r));
}

// ------------------------------------------------------------------------- depth tables
__global__ void st_prep_kernel(StBatch b) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.pre_z[b.nreq]) return;
  const int q = find_req(b.pre_z, b.nreq, i);
  const StSub S = b.sub[q];
  const int z = int(i - b.pre_z[q]);
  const double* tops = b.dbl + S.o_lay;
  const double zd = S.z0 + (z + 0.5) * S.dz;
  int l = 0;
  while (l + 1 < S.nl && tops[l + 1] <= zd) ++l;
  const double off = zd - tops[l];
  const double two = l + 1 < S.nl ? 2.0 * (tops[l + 1] - tops[l]) - off : 0.0;
  float4 t;
  split_ff(off, t.x, t.y);
  split_ff(two, t.z, t.w);
  b.zt[S.o_v + z] = t;
  b.zl[S.o_v + z] = l;
  if (z == 0) b.status[q] = EDT_OK;
}

// ------------------------------------------------------------------------- depth march
// coefficient slots per (f, k, layer): kappa.x (hi, lo), kappa.y (hi, lo), amplitude, rho
__global__ void __launch_bounds__(128) st_coef_kernel(StBatch b) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.pre_fk[b.nreq]) return;
  const int q = find_req(b.pre_fk, b.nreq, i);
  const StSub S = b.sub[q];
  const long long fk = i - b.pre_fk[q];
  const int f = int(fk / S.nk), k = int(fk % S.nk);
  const double* tops = b.dbl + S.o_lay;
  const double* vel = tops + S.nl;
  const double wr = 2.0 * M_PI * b.dbl[S.o_freq + f];
  const double kv = b.dbl[S.o_kval + k];
  const double om2r = wr * wr - S.eps * S.eps, om2i = 2.0 * wr * S.eps;
  const int J = S.nl;
  float* c = b.coef + S.o_coef + size_t(fk) * J * 8;
  float2 kap[ST_MAX_LAYERS], eh[ST_MAX_LAYERS], rho[ST_MAX_LAYERS], inv1r[ST_MAX_LAYERS];
  const double kv2 = kv * kv;
  for (int j = 0; j < J; ++j) {
    // kappa^2 = w = omega~^2 / c_j^2 - k^2 in FP64; kappa = sqrt(w) in FP32 on the branch
    // Im >= 0, then one Newton step kappa + (w - kappa^2) / (2 kappa): the square of the FP32
    // kappa is exact in FP64, so the residual is exact to FP64 rounding and the (hi, lo) pair
    // carries kappa to ~1e-14 relative with four FP64 products instead of a complex FP64 root
    const double ic2 = vel[J + j];                     // 1 / c_j^2, formed on the host
    const double wr2 = om2r * ic2 - kv2, wi2 = om2i * ic2;
    const float2 k32 = csqrt_upper32(make_float2(float(wr2), float(wi2)));
    const double rr = wr2 - (double(k32.x) * k32.x - double(k32.y) * k32.y);
    const double ri = wi2 - 2.0 * double(k32.x) * k32.y;
    const float2 dk = (k32.x == 0.f && k32.y == 0.f)
                          ? make_float2(0.f, 0.f)
                          : make_float2(float(rr), float(ri)) * cinv32(make_float2(2.f * k32.x, 2.f * k32.y));
    const float kxh = k32.x, kxl = dk.x, kyh = k32.y, kyl = dk.y;
    c[j * 8 + 0] = kxh; c[j * 8 + 1] = kxl; c[j * 8 + 2] = kyh; c[j * 8 + 3] = kyl;
    kap[j] = make_float2(kxh + kxl, kyh + kyl);
    if (j + 1 < J) {
      float hh, hl;
      split_ff(tops[j + 1] - tops[j], hh, hl);
      eh[j] = expi_ff(kxh, kxl, kyh, hh, hl);           // exp(i kappa_j h_j)
    } else {
      eh[j] = make_float2(1.f, 0.f);
    }
  }
  // upward: r_{J-1} = 0; y = kappa_{j+1}(1 - r_{j+1})/(1 + r_{j+1}); rho_j = (kappa_j - y)/(kappa_j + y)
  const float2 one = make_float2(1.f, 0.f);
  float2 r = make_float2(0.f, 0.f);
  rho[J - 1] = make_float2(0.f, 0.f);
  for (int j = J - 2; j >= 0; --j) {
    inv1r[j] = cinv32(one + r);
    const float2 y = kap[j + 1] * (one - r) * inv1r[j];
    rho[j] = (kap[j] - y) * cinv32(kap[j] + y);
    r = rho[j] * (eh[j] * eh[j]);
  }
  // downward: A_0 = i / (2 kappa_0), A_{j+1} = A_j exp(i kappa_j h_j)(1 + rho_j)/(1 + r_{j+1})
  float2 amp = make_float2(0.f, 0.5f) * cinv32(kap[0]);
  for (int j = 0; j < J; ++j) {
    c[j * 8 + 4] = amp.x; c[j * 8 + 5] = amp.y;
    c[j * 8 + 6] = rho[j].x; c[j * 8 + 7] = rho[j].y;
    if (j + 1 < J) amp = amp * eh[j] * (one + rho[j]) * inv1r[j];
  }
}

// g32 = sqrt|s_f| A_l [exp(i kappa_l off) + rho_l exp(i kappa_l (2 h_l - off))]: one CTA per
// (request, 8 consecutive (f, k) rows), threads over depth (the depth's layer and offsets are
// read once, the request found once per CTA)
constexpr int EV_ROWS = 8;

__global__ void __launch_bounds__(256) st_eval_kernel(StBatch b) {
  const int q = find_req(b.pre_eb, b.nreq, blockIdx.x);
  const StSub S = b.sub[q];
  const int fk0 = int(blockIdx.x - b.pre_eb[q]) * EV_ROWS;
  const int nfk = S.nf * S.nk;
  __shared__ float sq_row[EV_ROWS];                         // sqrt|s_f| of each row's frequency
  if (threadIdx.x < EV_ROWS && fk0 + int(threadIdx.x) < nfk) {
    const float wr = 6.283185307179586f * float(b.dbl[S.o_freq + (fk0 + threadIdx.x) / S.nk]);
    sq_row[threadIdx.x] = sqrtf((wr * wr + S.eps2) * S.dzdx);
  }
  __syncthreads();
  for (int z = threadIdx.x; z < S.nz; z += blockDim.x) {
    const int l = b.zl[S.o_v + z];
    const float4 zo = b.zt[S.o_v + z];
    const bool two = l + 1 < S.nl;
    for (int r = 0; r < EV_ROWS && fk0 + r < nfk; ++r) {
      const int fk = fk0 + r;
      const float4* c4 = reinterpret_cast<const float4*>(b.coef + S.o_coef + (size_t(fk) * S.nl + l) * 8);
      const float4 k4 = c4[0], ar = c4[1];
      float2 ex = expi_ff(k4.x, k4.y, k4.z, zo.x, zo.y);
      if (two) ex = ex + make_float2(ar.z, ar.w) * expi_ff(k4.x, k4.y, k4.z, zo.z, zo.w);
      const float sq = sq_row[r];
      const float2 g = make_float2(ar.x, ar.y) * ex;
      b.g32[S.o_g + size_t(fk) * S.nzs + z] = make_float2(sq * g.x, sq * g.y);
    }
  }
}

// ------------------------------------------------------------------------- operand tiles
// Byte offset of (row, 16-byte chunk c) of K stage s, half hl (0 hi, 1 lo) in a request's tiles.
__device__ __forceinline__ size_t tile_off(const StSub& S, int s, int hl, int row, int c) {
  const int TR = S.nzt * ST_TILE + ST_DROWS;
  return size_t(S.o_tile) + (size_t(s * 2 + hl) * TR + row) * 128 + size_t((c ^ (row & 7)) << 4);
}

__global__ void __launch_bounds__(256) st_tiles_kernel(StBatch b) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= b.pre_tw[b.nreq]) return;
  const int q = find_req(b.pre_tw, b.nreq, w);
  const StSub S = b.sub[q];
  const long long e = w - b.pre_tw[q];
  const int nunit = 4 * S.nzt + 1;
  const int s = int(e / nunit), u = int(e % nunit);
  const int r0 = s * ST_KC;
  if (u < 4 * S.nzt) {
    const int z = u * 32 + lane;
    const bool zv = z < S.nz;
    float tr = 0.f;
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
      float2 a[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int r = r0 + c * 4 + t;
        a[t] = make_float2(0.f, 0.f);
        if (r < S.nrow && zv) {
          const int4 row = b.rows[S.o_row + r];
          const size_t base = size_t(S.o_g) + size_t(row.x) * S.nk * S.nzs + z;
          a[t] = b.g32[base + size_t(row.y) * S.nzs] * b.g32[base + size_t(row.z) * S.nzs];
          tr = fmaf(a[t].x, a[t].x, fmaf(a[t].y, a[t].y, tr));
        }
      }
      uint4 h, l;
      h.x = pack_bf16(a[0].x, a[0].y); h.y = pack_bf16(a[1].x, a[1].y);
      h.z = pack_bf16(a[2].x, a[2].y); h.w = pack_bf16(a[3].x, a[3].y);
      const __nv_bfloat162* hb = reinterpret_cast<const __nv_bfloat162*>(&h);
      float2 h0 = __bfloat1622float2(hb[0]), h1 = __bfloat1622float2(hb[1]);
      float2 h2 = __bfloat1622float2(hb[2]), h3 = __bfloat1622float2(hb[3]);
      l.x = pack_bf16(a[0].x - h0.x, a[0].y - h0.y); l.y = pack_bf16(a[1].x - h1.x, a[1].y - h1.y);
      l.z = pack_bf16(a[2].x - h2.x, a[2].y - h2.y); l.w = pack_bf16(a[3].x - h3.x, a[3].y - h3.y);
      *reinterpret_cast<uint4*>(b.tiles + tile_off(S, s, 0, z, c)) = h;
      *reinterpret_cast<uint4*>(b.tiles + tile_off(S, s, 1, z, c)) = l;
    }
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (lane == 0) b.twtr[w] = S.alpha * double(tr);
  } else {
    if (lane == 0) b.twtr[w] = 0.0;
    const int drow0 = S.nzt * ST_TILE;
    if (lane < 8) {
      // chunk c = lane: complex rows 4c .. 4c + 3 of the stage, data d' = conj(u_f) d (u_f the
      // unit phase of s_f) for both right-hand sides; the rotated data are kept for the refinement
      const int c = lane;
      float v[2][8];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int r = r0 + c * 4 + t;
        float2 d0 = make_float2(0.f, 0.f), d1 = d0;
        if (r < S.nrow) {
          const float4 dd = b.data[S.o_row + r];
          const float2 ph = cconj(sf_phase(b.dbl[S.o_freq + b.rows[S.o_row + r].x], S.eps));
          d0 = ph * make_float2(dd.x, dd.y);
          d1 = ph * make_float2(dd.z, dd.w);
          b.drot[S.o_row + r] = make_float4(d0.x, d0.y, d1.x, d1.y);
        }
        v[0][2 * t] = d0.x; v[0][2 * t + 1] = d0.y;
        v[1][2 * t] = d1.x; v[1][2 * t + 1] = d1.y;
      }
#pragma unroll
      for (int which = 0; which < 2; ++which) {
        const float* vv = v[which];
        uint4 h, l;
        h.x = pack_bf16(vv[0], vv[1]); h.y = pack_bf16(vv[2], vv[3]);
        h.z = pack_bf16(vv[4], vv[5]); h.w = pack_bf16(vv[6], vv[7]);
        const __nv_bfloat162* hb = reinterpret_cast<const __nv_bfloat162*>(&h);
        float2 h0 = __bfloat1622float2(hb[0]), h1 = __bfloat1622float2(hb[1]);
        float2 h2 = __bfloat1622float2(hb[2]), h3 = __bfloat1622float2(hb[3]);
        l.x = pack_bf16(vv[0] - h0.x, vv[1] - h0.y); l.y = pack_bf16(vv[2] - h1.x, vv[3] - h1.y);
        l.z = pack_bf16(vv[4] - h2.x, vv[5] - h2.y); l.w = pack_bf16(vv[6] - h3.x, vv[7] - h3.y);
        *reinterpret_cast<uint4*>(b.tiles + tile_off(S, s, 0, drow0 + which, c)) = h;
        *reinterpret_cast<uint4*>(b.tiles + tile_off(S, s, 1, drow0 + which, c)) = l;
      }
    } else {
      const uint4 zero = make_uint4(0, 0, 0, 0);
      for (int e2 = lane - 8; e2 < 2 * 14 * 8; e2 += 24) {    // rows drow0 + 2 .. + 15, both halves
        const int hl = e2 / 112, rem = e2 % 112;
        *reinterpret_cast<uint4*>(b.tiles + tile_off(S, s, hl, drow0 + 2 + rem / 8, rem % 8)) = zero;
      }
    }
  }
}

// ------------------------------------------------------------------------- tensor-core Gram
constexpr int GS_STAGES = 3;
constexpr int GS_THREADS = 192;                  // warp 0 copies, warp 1 MMA, warps 2-5 epilogue
constexpr int GS_A = ST_TILE * 128;              // one 128-row operand (bytes)
constexpr int GS_B = (ST_TILE + ST_DROWS) * 128; // 128 depth rows + 16 data rows
constexpr int GS_STAGE = 2 * GS_A + 2 * GS_B;    // A hi, A lo, B hi, B lo
constexpr int GS_TMEM_COLS = 256;

__global__ void __launch_bounds__(GS_THREADS, 1) st_gram_kernel(StBatch b) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023);
  unsigned char* ops = reinterpret_cast<unsigned char*>(base);
  uint64_t* bars = reinterpret_cast<uint64_t*>(ops + size_t(GS_STAGES) * GS_STAGE);
  uint64_t* full = bars;                       // [GS_STAGES] copies landed
  uint64_t* empty = bars + GS_STAGES;          // [GS_STAGES] MMAs done with the stage
  uint64_t* acc_full = bars + 2 * GS_STAGES;   // accumulator complete
  uint64_t* acc_empty = acc_full + 1;          // epilogue done reading it
  uint64_t* drain = acc_empty + 1;
  uint64_t* never = drain + 1;                 // never completed: the wait-test stall
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k0 = b.cta_item0[blockIdx.x], k1 = b.cta_item0[blockIdx.x + 1];
  const long long budget = b.wait_cycles > 0 ? b.wait_cycles : WAIT_CYCLES;
  if (threadIdx.x == 0) {
    for (int s = 0; s < GS_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 128);
    mbar_init(drain, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, GS_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      for (int k = k0; k < k1 && ok; ++k) {
        const StItem itm = b.items[k];
        const StSub S = b.sub[itm.req];
        const int TR = S.nzt * ST_TILE + ST_DROWS;
        const bool last = itm.tj == S.nzt - 1, diag = itm.ti == itm.tj;
        const uint32_t nb = uint32_t(last ? GS_B : GS_A);
        const uint32_t bytes = 2 * nb + (diag ? 0u : 2u * GS_A);
        for (int s = 0; s < S.kst; ++s, ++it) {
          const int st = int(it % GS_STAGES);
          if (it >= GS_STAGES &&
              !mbar_wait(&empty[st], unsigned(((it / GS_STAGES) - 1) & 1), abort_flag, budget)) {
            ok = false;
            break;
          }
          unsigned char* sb = ops + size_t(st) * GS_STAGE;
          const unsigned char* hi = b.tiles + size_t(S.o_tile) + size_t(s) * 2 * TR * 128;
          const unsigned char* lo = hi + size_t(TR) * 128;
          mbar_expect_tx(&full[st], bytes);
          bulk_g2s(sb + 2 * GS_A, hi + size_t(itm.tj) * GS_A, nb, &full[st]);
          bulk_g2s(sb + 2 * GS_A + GS_B, lo + size_t(itm.tj) * GS_A, nb, &full[st]);
          if (!diag) {
            bulk_g2s(sb, hi + size_t(itm.ti) * GS_A, GS_A, &full[st]);
            bulk_g2s(sb + GS_A, lo + size_t(itm.ti) * GS_A, GS_A, &full[st]);
          }
        }
      }
      // copies of the last GS_STAGES stages may still be in flight after an early exit:
      // each must land before the CTA leaves
      for (long long j = it > GS_STAGES ? it - GS_STAGES : 0; j < it; ++j)
        mbar_drain(&full[j % GS_STAGES], unsigned((j / GS_STAGES) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t ops_s = smem_u32(ops);
      long long it = 0;
      // wait test: a barrier nothing completes, so the kernel takes its timeout path
      bool ok = !(b.wait_stall && !mbar_wait(never, 0u, abort_flag, budget));
      for (int k = k0; k < k1 && ok; ++k) {
        const StItem itm = b.items[k];
        const StSub S = b.sub[itm.req];
        const bool last = itm.tj == S.nzt - 1, diag = itm.ti == itm.tj;
        const uint32_t idesc = idesc_bf16(ST_TILE, last ? ST_TILE + ST_DROWS : ST_TILE);
        if (k > k0) {
          if (!mbar_wait(acc_empty, unsigned((k - k0 - 1) & 1), abort_flag, budget)) { ok = false; break; }
          tc_fence_after();
        }
        for (int s = 0; s < S.kst; ++s, ++it) {
          const int st = int(it % GS_STAGES);
          if (!mbar_wait(&full[st], unsigned((it / GS_STAGES) & 1), abort_flag, budget)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sb = ops_s + uint32_t(st) * GS_STAGE;
          const uint32_t bh = sb + 2 * GS_A, bl = bh + GS_B;
          const uint32_t ah = diag ? bh : sb, al = diag ? bl : sb + GS_A;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t o = kk * 32;
            mma_bf16(tmem, sw128_desc(ah + o), sw128_desc(bh + o), idesc, (s > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(tmem, sw128_desc(ah + o), sw128_desc(bl + o), idesc, 1u);
            mma_bf16(tmem, sw128_desc(al + o), sw128_desc(bh + o), idesc, 1u);
          }
          mma_commit(&empty[st]);
        }
        if (!ok) break;
        mma_commit(acc_full);
      }
      // drain: every issued MMA has completed before tensor memory is released
      mma_commit(drain);
      mbar_drain(drain, 0u);
    }
    __syncwarp();
  } else {
    // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 = rows of the 128-row tile
    const int qd = warp & 3;
    for (int k = k0; k < k1; ++k) {
      if (!mbar_wait(acc_full, unsigned((k - k0) & 1), abort_flag, budget)) break;
      tc_fence_after();
      const StItem itm = b.items[k];
      const StSub S = b.sub[itm.req];
      const bool last = itm.tj == S.nzt - 1;
      const int ncol = last ? ST_TILE + ST_DROWS : ST_TILE;
      const int a = itm.ti * ST_TILE + qd * 32 + lane;
      float2* G = reinterpret_cast<float2*>(b.G) + S.o_G;
      for (int c0 = 0; c0 < ncol; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + (uint32_t(qd * 32) << 16) + uint32_t(c0), v);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int col = c0 + c;
          if (col < ST_TILE) {
            const int bc = itm.tj * ST_TILE + col;
            if (a < S.nz && bc < S.nz) G[size_t(bc) * S.nz + a] = make_float2(v[c], 0.f);   // lower triangle
          } else if (col < ST_TILE + 2 && a < S.nz) {
            b.b[(S.o_v + a) * 2 + (col - ST_TILE)] = double(v[c]);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(acc_empty);
    }
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(b.flags, 1u);
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, GS_TMEM_COLS);
  }
}

// alpha trace(Ahat^T Ahat) of each request: the parts of its tile-writer warps in a fixed order
// (lane l takes parts l, l + 32, ...; then a butterfly over the lanes), one warp per request.
__global__ void __launch_bounds__(256) st_trace_kernel(StBatch b) {
  const int q = int(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (q >= b.nreq) return;
  double t = 0.0;
  for (long long w = b.pre_tw[q] + lane; w < b.pre_tw[q + 1]; w += 32) t += b.twtr[w];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) b.trace[q] = t;
}

// ------------------------------------------------------------------------- refinement residual
// Ahat^T (dhat - Ahat x) over 256 rows per CTA (one warp per 32 rows, lanes over depth); FP32
// products, warp partials summed in FP64 into the CTA's partial; st_rsum adds a request's
// partials in CTA order.
__global__ void __launch_bounds__(256) st_refine_kernel(StBatch b) {
  constexpr int NZL = ST_MAX_NZ / 32;
  __shared__ float xs[2][ST_MAX_NZ];
  __shared__ float red[8][2][ST_MAX_NZ];
  const int q = find_req(b.pre_rc, b.nreq, blockIdx.x);
  const StSub S = b.sub[q];
  if (b.status[q] != EDT_OK) return;
  const int chunk = int(blockIdx.x - b.pre_rc[q]);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < S.nz; i += blockDim.x) {
    xs[0][i] = float(b.x[(S.o_v + i) * 2 + 0]);
    xs[1][i] = float(b.x[(S.o_v + i) * 2 + 1]);
  }
  __syncthreads();
  float acc0[NZL], acc1[NZL];
#pragma unroll
  for (int i = 0; i < NZL; ++i) { acc0[i] = 0.f; acc1[i] = 0.f; }
  const int rbeg = chunk * ST_REFINE_ROWS + warp * 32;
  for (int rr = 0; rr < 32; ++rr) {
    const int r = rbeg + rr;
    if (r >= S.nrow) break;
    const int4 row = b.rows[S.o_row + r];
    const float4 dd = b.drot[S.o_row + r];
    const float2* gp = b.g32 + S.o_g + (size_t(row.x) * S.nk + row.y) * S.nzs;
    const float2* gq = b.g32 + S.o_g + (size_t(row.x) * S.nk + row.z) * S.nzs;
    float2 a[NZL];
    float s0r = 0.f, s0i = 0.f, s1r = 0.f, s1i = 0.f;
#pragma unroll
    for (int i = 0; i < NZL; ++i) {
      const int z = lane + 32 * i;
      a[i] = make_float2(0.f, 0.f);
      if (z < S.nz) {
        a[i] = gp[z] * gq[z];
        s0r = fmaf(a[i].x, xs[0][z], s0r); s0i = fmaf(a[i].y, xs[0][z], s0i);
        s1r = fmaf(a[i].x, xs[1][z], s1r); s1i = fmaf(a[i].y, xs[1][z], s1i);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      s0r += __shfl_xor_sync(0xffffffffu, s0r, o); s0i += __shfl_xor_sync(0xffffffffu, s0i, o);
      s1r += __shfl_xor_sync(0xffffffffu, s1r, o); s1i += __shfl_xor_sync(0xffffffffu, s1i, o);
    }
    const float t0r = dd.x - s0r, t0i = dd.y - s0i, t1r = dd.z - s1r, t1i = dd.w - s1i;
#pragma unroll
    for (int i = 0; i < NZL; ++i) {
      acc0[i] = fmaf(a[i].x, t0r, fmaf(a[i].y, t0i, acc0[i]));
      acc1[i] = fmaf(a[i].x, t1r, fmaf(a[i].y, t1i, acc1[i]));
    }
  }
#pragma unroll
  for (int i = 0; i < NZL; ++i) {
    const int z = lane + 32 * i;
    if (z < S.nz) { red[warp][0][z] = acc0[i]; red[warp][1][z] = acc1[i]; }
  }
  __syncthreads();
  double* part = b.rcp + 2 * (b.pre_rz[q] + (long long)chunk * S.nz);
  for (int e = threadIdx.x; e < 2 * S.nz; e += blockDim.x) {
    const int side = e / S.nz, z = e - side * S.nz;
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += double(red[w][side][z]);
    part[e] = t;
  }
}

// r of request blockIdx.x: its refinement CTAs' partials in CTA order (zero after a failure,
// when they stored nothing)
__global__ void __launch_bounds__(256) st_rsum_kernel(StBatch b) {
  const int q = blockIdx.x;
  const StSub S = b.sub[q];
  const int ncta = b.status[q] == EDT_OK ? int(b.pre_rc[q + 1] - b.pre_rc[q]) : 0;
  const double* part = b.rcp + 2 * b.pre_rz[q];
  for (int e = threadIdx.x; e < 2 * S.nz; e += blockDim.x) {
    const int side = e / S.nz, z = e - side * S.nz;
    double t = 0.0;
    for (int c = 0; c < ncta; ++c) t += part[size_t(c) * 2 * S.nz + e];
    b.r[(S.o_v + z) * 2 + side] = t;
  }
}

}  // namespace

int st_gram_smem_bytes() { return GS_STAGES * GS_STAGE + 1024 + 128; }

cudaError_t prepare_stream() {
  cudaError_t e = cudaFuncSetAttribute(st_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       st_gram_smem_bytes());
  if (e != cudaSuccess) return e;
  return prepare_chol_var(ST_MAX_NZ);
}

static unsigned blocks_for(long long n, int per) { return unsigned((n + per - 1) / per); }

const char* const kStreamKernels[ST_NKERNEL] = {"st_prep", "st_coef", "st_eval", "st_tiles", "st_gram",
                                                "chol", "st_refine", "update"};

cudaError_t launch_stream_batch(const StBatch& b, int nmax, cudaStream_t s, cudaEvent_t* ev) {
  if (b.nreq <= 0) return cudaSuccess;
  auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], s); };
  mark(0);
  if (b.tot_z > 0) st_prep_kernel<<<blocks_for(b.tot_z, 256), 256, 0, s>>>(b);
  mark(1);
  if (b.tot_fk > 0) st_coef_kernel<<<blocks_for(b.tot_fk, 128), 128, 0, s>>>(b);
  mark(2);
  if (b.tot_eb > 0) st_eval_kernel<<<unsigned(b.tot_eb), 256, 0, s>>>(b);
  mark(3);
  if (b.tot_tw > 0) {
    st_tiles_kernel<<<blocks_for(b.tot_tw * 32, 256), 256, 0, s>>>(b);
    st_trace_kernel<<<blocks_for((long long)b.nreq * 32, 256), 256, 0, s>>>(b);
  }
  mark(4);
  if (b.ncta > 0) st_gram_kernel<<<b.ncta, GS_THREADS, st_gram_smem_bytes(), s>>>(b);
  mark(5);
  Dev d{};
  d.nz = nmax;
  d.nsub = b.nreq;
  d.alpha = 1.0;                 // trace[] already holds alpha trace(Ahat^T Ahat)
  d.G = b.G; d.L32 = b.L32; d.dinv = b.dinv; d.dinv32 = b.dinv32;
  d.b = b.b; d.x = b.x; d.r = b.r; d.trace = b.trace; d.status = b.status;
  d.row_off = b.row_off;
  d.sub_n = b.sub_n; d.sub_goff = b.sub_goff; d.sub_voff = b.sub_voff; d.sub_order = b.sub_order;
  cudaError_t e = launch_chol_blocked(d, true, nmax, b.cb_nstep, b.cb_act, b.cb_nact_host, b.cb_tpre,
                                      b.cb_ntile_host, b.cb_cpre, b.cb_nchunk_host, 1, s);
  if (e != cudaSuccess) return e;
  mark(6);
  if (b.tot_rc > 0) {
    st_refine_kernel<<<unsigned(b.tot_rc), 256, 0, s>>>(b);
    st_rsum_kernel<<<unsigned(b.nreq), 256, 0, s>>>(b);
  }
  mark(7);
  e = launch_refine_update_var(d, nmax, s);
  mark(8);
  return e;
}

}  // namespace edt
