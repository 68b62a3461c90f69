// Tensor-core (tcgen05, sm_103a) augmented Gram of the split systems, mixed precision.
//
// For every midpoint index m the split least-squares problem of eq. Split has the
// real-stacked matrix Ahat = [Re A; Im A] (rows: frequencies x receiver wavenumbers, one
// complex row giving two real rows) and right-hand sides dhat_+-.  This kernel forms
//     [Ahat | dhat_+ | dhat_-]^T [Ahat | dhat_+ | dhat_-]  restricted to the rows z < nz,
// i.e. G = Ahat^T W Ahat and b_+- = Ahat^T W dhat_+-, with BF16 operands (optionally the
// split hi + lo pair, three MMAs per product) and FP32 accumulation in tensor memory.
//
// Structure (one persistent CTA per SM, all subproblems in one launch):
//   * rows of all subproblems are concatenated and split evenly over the CTAs; a CTA's
//     range falls into 1..few "segments" (its part of one subproblem), each accumulated
//     in TMEM and written out as an FP32 partial tile, summed per subproblem afterwards;
//   * warps 0-15 are producers: for 32 complex rows per pipeline stage they rebuild the
//     kernel rows a(z) = |s_f| g(k_p, z) g(k_q, z) from the L2-resident FP32 table of
//     sqrt|s_f| g (unpredicated loads at byte offsets kept in the row table; padding rows
//     and depths take weight 0), scale weight-2 rows by sqrt 2, split into hi (and lo)
//     16-bit halves, and
//     store them K-major with the 128-byte swizzle; (Re a, Im a) of one complex row are two
//     adjacent K elements.  The data rows d_+, d_- occupy two extra operand rows;
//   * operand type: FP16 (line geometry) or BF16 (window geometry).  FP16's 11-bit
//     significand makes the hi + lo pair a 22-bit row (BF16: 16 bits), at the same MMA rate,
//     but its range is narrow, so each segment's kernel rows and data rows are multiplied
//     by powers of two (chosen by gram_scale_kernel from per-row maxima of the table) that
//     put the segment's largest value just under 2^14; the reduction divides them out
//     exactly.  The Gram's representation error sets the contraction rate of the iterative
//     refinement (it is amplified by 1 / lam in the null space of Ahat), so the FP16 pair
//     lets one refinement step reach 1e-5 at damping two orders of magnitude weaker;
//   * warp 16 issues tcgen05.mma (M = 128, K = 16) from one thread: both operands are
//     views of the same stage tile (A = depth rows of one 128-row half, B = all depth rows
//     plus the data rows), so one generated tile feeds the whole upper block row;
//   * after the last stage of a segment the producers read the accumulator with
//     tcgen05.ld and write the partial tile; they also accumulate trace(G) in FP64 from the
//     unrounded FP32 rows (the damping lam = alpha * trace(G) must not inherit BF16 error).
// Every wait is bounded; on expiry the CTA raises a device flag and leaves cleanly.
#include "edt_internal.h"
#include "cplx.cuh"
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include "tc_ptx.cuh"

namespace edt {

namespace {

constexpr int PRODUCER_WARPS = 16;
constexpr int NTHREADS = (PRODUCER_WARPS + 1) * 32;
constexpr int ROWB = 128;                       // bytes per operand row per stage (64 bf16)

__host__ __device__ inline int nzp_of(int nz) { return (nz + 31) / 32 * 32; }
__host__ __device__ inline int zrows_of(int nzp) {
  int need = nzp + 16;
  int mrows = nzp > TC_M ? 2 * TC_M : TC_M;
  return need > mrows ? need : mrows;
}
__host__ __device__ inline int cols_of(int nzp) { return (nzp + 16) + (nzp > TC_M ? nzp - TC_M + 16 : 0); }
__host__ __device__ inline int stages_of(int passes) { return passes == 1 ? 4 : 3; }

// Row table of one stage in shared memory: TC_KC GramRow entries (offsets, sqrt weight),
// then the rows' data (d_+, d_-) as TC_KC float4; both arrive by bulk copy.
constexpr int TAB_BYTES = TC_KC * int(sizeof(GramRow) + sizeof(float4));

using namespace tcx;


// Exponent k of the scale 2^k for a positive bound v in [2^(e-1), 2^e): k = 14 - e puts the
// scaled bound in [2^13, 2^14); clamped so that 2^k stays a normal float.
__device__ __forceinline__ int pow2_exp(float v) {
  if (!(v > 0.f) || !isfinite(v)) return 0;
  int e;
  frexpf(v, &e);
  return max(-120, min(120, 14 - e));
}

// 2^k as a double, exactly (|k| <= 1000)
__device__ __forceinline__ double pow2d(int k) {
  return __longlong_as_double((long long)(1023 + k) << 52);
}

// (lo_k, hi_k) as two 16-bit values in one word, .x at the lower address (smaller K)
template <bool F16>
__device__ __forceinline__ uint32_t pack16(float lo_k, float hi_k) {
  if (F16) {
    __half2 v = __floats2half2_rn(lo_k, hi_k);
    return *reinterpret_cast<uint32_t*>(&v);
  }
  return pack_bf16(lo_k, hi_k);
}
template <bool F16>
__device__ __forceinline__ float2 unpack16(uint32_t w) {
  if (F16) return __half22float2(*reinterpret_cast<const __half2*>(&w));
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
}
// hi and lo words of four complex values (eight K elements)
template <bool F16>
__device__ __forceinline__ void split16(const float2 (&v)[4], uint4& h, uint4& l) {
  h.x = pack16<F16>(v[0].x, v[0].y); h.y = pack16<F16>(v[1].x, v[1].y);
  h.z = pack16<F16>(v[2].x, v[2].y); h.w = pack16<F16>(v[3].x, v[3].y);
  const float2 h0 = unpack16<F16>(h.x), h1 = unpack16<F16>(h.y);
  const float2 h2 = unpack16<F16>(h.z), h3 = unpack16<F16>(h.w);
  l.x = pack16<F16>(v[0].x - h0.x, v[0].y - h0.y); l.y = pack16<F16>(v[1].x - h1.x, v[1].y - h1.y);
  l.z = pack16<F16>(v[2].x - h2.x, v[2].y - h2.y); l.w = pack16<F16>(v[3].x - h3.x, v[3].y - h3.y);
}

template <int PASSES, bool F16>
__global__ void __launch_bounds__(NTHREADS, 1) gram_tc_kernel(Dev d) {
  constexpr int STAGES = PASSES == 1 ? 4 : 3;
  constexpr int NCOMP = PASSES == 1 ? 1 : 2;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int nz = d.nz, nzp = nzp_of(nz), zr = zrows_of(nzp), ncols = cols_of(nzp);
  const uint32_t stage_bytes = uint32_t(zr) * ROWB;

  // carve shared memory: operand stages (1024-aligned), row tables, barriers
  uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023);
  unsigned char* ops = reinterpret_cast<unsigned char*>(base);
  unsigned char* rowtab = ops + size_t(STAGES) * NCOMP * stage_bytes;   // [2][TAB_BYTES]
  uint64_t* bars = reinterpret_cast<uint64_t*>(rowtab + 2 * TAB_BYTES);
  uint64_t* full = bars;                   // [STAGES] producers -> MMA
  uint64_t* empty = bars + STAGES;         // [STAGES] MMA commit -> producers
  uint64_t* acc_full = bars + 2 * STAGES;  // MMA commit -> epilogue
  uint64_t* acc_empty = acc_full + 1;      // epilogue -> MMA
  uint64_t* drain = acc_empty + 1;         // final commit: every issued MMA has completed
  uint64_t* tbar = drain + 1;              // [2] row-table bulk copies
  uint64_t* never = tbar + 2;              // never completed: the wait-test stall
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cta = blockIdx.x;
  const int s0 = d.cta_seg0[cta], s1 = d.cta_seg0[cta + 1];
  const long long budget = d.wait_cycles > 0 ? d.wait_cycles : WAIT_CYCLES;
  const int* slots = d.cta_seg0 + d.ncta_gram + 1;

  // zero every operand stage once: padding rows stay zero for the whole kernel
  {
    uint4* z4 = reinterpret_cast<uint4*>(ops);
    const size_t n16 = size_t(STAGES) * NCOMP * stage_bytes / 16;
    for (size_t i = threadIdx.x; i < n16; i += NTHREADS) z4[i] = make_uint4(0, 0, 0, 0);
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], PRODUCER_WARPS * 32); mbar_init(&empty[s], 1); }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, PRODUCER_WARPS * 32);
    mbar_init(drain, 1);
    mbar_init(&tbar[0], 1);
    mbar_init(&tbar[1], 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  uint32_t alloc_cols = 32;
  while (alloc_cols < uint32_t(ncols)) alloc_cols <<= 1;
  if (warp == PRODUCER_WARPS) tmem_alloc(tmem_slot, alloc_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == PRODUCER_WARPS) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t ops_s = smem_u32(ops);
    long long it = 0;
    // wait test: a barrier nothing completes, so this wait runs out and the kernel takes its
    // timeout path (flag raised, producers released through the abort flag, TMEM freed)
    bool ok = !(d.wait_stall && !mbar_wait(never, 0u, abort_flag, budget));
    for (int si = s0; si < s1 && ok; ++si) {
      const int slot = slots[si];
      const long long nrow = d.seg_nrow[slot];
      const long long nst = (nrow + TC_KC - 1) / TC_KC;
      const int k = si - s0;
      if (k > 0) {
        if (!mbar_wait(acc_empty, unsigned((k - 1) & 1), abort_flag, budget)) { ok = false; break; }
        tc_fence_after();
      }
      for (long long st = 0; st < nst; ++st, ++it) {
        const int s = int(it % STAGES);
        if (!mbar_wait(&full[s], unsigned((it / STAGES) & 1), abort_flag, budget)) { ok = false; break; }
        tc_fence_after();
        if (lane == 0) {
          const uint32_t hi = ops_s + uint32_t(s) * NCOMP * stage_bytes;
          const uint32_t lo = hi + stage_bytes;
          const int n0 = nzp + 16;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              int ar, br, n, col;
              if (i == 0) { ar = 0; br = 0; n = n0 > 256 ? 256 : n0; col = 0; }
              else if (i == 1) { if (n0 <= 256) continue; ar = 0; br = 256; n = n0 - 256; col = 256; }
              else { if (nzp <= TC_M) continue; ar = TC_M; br = TC_M; n = nzp - TC_M + 16; col = n0; }
              const uint32_t ao = uint32_t(ar) * ROWB + kk * 32, bo = uint32_t(br) * ROWB + kk * 32;
              const uint32_t idesc = F16 ? idesc_f16(TC_M, n) : idesc_bf16(TC_M, n);
              const uint32_t dt = tmem + uint32_t(col);
              const uint32_t acc0 = (st > 0 || kk > 0) ? 1u : 0u;
              mma_bf16(dt, sw128_desc(hi + ao), sw128_desc(hi + bo), idesc, acc0);
              if (PASSES == 3) {
                mma_bf16(dt, sw128_desc(hi + ao), sw128_desc(lo + bo), idesc, 1u);
                mma_bf16(dt, sw128_desc(lo + ao), sw128_desc(hi + bo), idesc, 1u);
              }
            }
          }
          mma_commit(&empty[s]);
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) mma_commit(acc_full);
      __syncwarp();
    }
    // drain: wait (bounded, independent of the abort flag) until every issued MMA is done
    if (lane == 0) {
      mma_commit(drain);
      mbar_drain(drain, 0u);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ producers + epilogue
    const int ptid = threadIdx.x;                 // 0..255
    const int nunits = (nzp / 32) * 8;            // (32-depth group, 16-byte K chunk)
    const float2* g32 = d.rowtab32;
    const size_t nzs = size_t(d.nzs);
    long long it = 0;
    bool ok = true;
    // The row table of each stage (32 GramRow entries, 1 KB) arrives by a bulk copy issued
    // one stage ahead into a double buffer, so it is off the producers' critical path.
    int nsi = s0;                        // (segment, stage) of the next table copy to issue
    long long nst_next = 0;
    long long tb_issued = 0, tb_done = 0;   // table copies issued (thread 0) and waited for
    auto issue_table = [&](long long it_next) {
      while (nsi < s1) {
        const int sl = slots[nsi];
        const long long n = (d.seg_nrow[sl] + TC_KC - 1) / TC_KC;
        if (nst_next < n) {
          const int b = int(it_next & 1);
          const long long r = d.seg_row0[sl] + nst_next * TC_KC;
          unsigned char* tb = rowtab + b * TAB_BYTES;
          mbar_expect_tx(&tbar[b], TAB_BYTES);
          bulk_g2s(tb, d.gent + r, TC_KC * sizeof(GramRow), &tbar[b]);
          bulk_g2s(tb + TC_KC * sizeof(GramRow), reinterpret_cast<const float4*>(d.rhs) + r,
                   TC_KC * sizeof(float4), &tbar[b]);
          ++nst_next;
          ++tb_issued;
          return;
        }
        ++nsi;
        nst_next = 0;
      }
    };
    if (ptid == 0) issue_table(0);
    float tr_hi = 0.f, tr_lo = 0.f;      // Kahan-compensated FP32 trace of the segment
    for (int si = s0; si < s1 && ok; ++si) {
      const int slot = slots[si];
      const long long nrow = d.seg_nrow[slot];
      const long long nst = (nrow + TC_KC - 1) / TC_KC;
      // power-of-two scales of this segment's kernel rows and data rows (FP16 operands)
      const int2 se = F16 ? d.gscale[slot] : make_int2(0, 0);
      const float2 sc = make_float2(ldexpf(1.f, se.x), ldexpf(1.f, se.y));
      tr_hi = 0.f; tr_lo = 0.f;
      for (long long st = 0; st < nst; ++st, ++it) {
        const int s = int(it % STAGES);
        if (it >= STAGES) {
          if (!mbar_wait(&empty[s], unsigned(((it / STAGES) - 1) & 1), abort_flag, budget)) { ok = false; break; }
        }
        if (!mbar_wait(&tbar[it & 1], unsigned((it >> 1) & 1), abort_flag, budget)) { ok = false; break; }
        tb_done = it + 1;
        const GramRow* rt = reinterpret_cast<const GramRow*>(rowtab + (it & 1) * TAB_BYTES);
        const float4* rdat = reinterpret_cast<const float4*>(rt + TC_KC);
        const int nvalid = int(min((long long)TC_KC, nrow - st * TC_KC));   // rows past it: padding
        asm volatile("bar.sync 1, %0;" ::"n"(PRODUCER_WARPS * 32) : "memory");
        if (ptid == 0) issue_table(it + 1);
        unsigned char* hi = ops + size_t(s) * NCOMP * stage_bytes;
        unsigned char* lo = hi + stage_bytes;
        float trs = 0.f;
        // two (32-depth, 16-byte chunk) units per warp at a time: all 16 table loads of
        // both are issued before either is converted, to keep enough L2 reads in flight
        for (int u0 = warp; u0 < nunits; u0 += 2 * PRODUCER_WARPS) {
          float2 gpv[2][4], gqv[2][4];
          float swv[2][4];
          int zz[2], cc[2];
          const char* gz[2];
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const int u = u0 + h2 * PRODUCER_WARPS;
            const bool uv = u < nunits;
            zz[h2] = uv ? (u >> 3) * 32 + lane : nzp;     // nzp: marks an absent unit
            cc[h2] = u & 7;
            // this lane's depth in every table row (a padding depth reads depth 0, weight 0)
            gz[h2] = reinterpret_cast<const char*>(g32 + (uv && zz[h2] < nz ? zz[h2] : 0));
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
              const GramRow e = rt[cc[h2] * 4 + rr];
              // entries past the segment's last row belong to the next segment: padding here
              const bool ok2 = uv && zz[h2] < nz && (cc[h2] * 4 + rr) < nvalid;
              swv[h2][rr] = ok2 ? e.sw * sc.x : 0.f;
              gpv[h2][rr] = __ldg(reinterpret_cast<const float2*>(gz[h2] + e.bp));
              gqv[h2][rr] = __ldg(reinterpret_cast<const float2*>(gz[h2] + e.bq));
            }
          }
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            if (zz[h2] >= nzp) continue;
            float2 a[4];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
              const float2 v = gpv[h2][rr] * gqv[h2][rr];
              a[rr] = make_float2(swv[h2][rr] * v.x, swv[h2][rr] * v.y);
              trs = fmaf(a[rr].x, a[rr].x, fmaf(a[rr].y, a[rr].y, trs));
            }
            const uint32_t off = sw_off(zz[h2], cc[h2]);
            if (PASSES == 3) {
              uint4 h, l;
              split16<F16>(a, h, l);
              *reinterpret_cast<uint4*>(hi + off) = h;
              *reinterpret_cast<uint4*>(lo + off) = l;
            } else {
              uint4 h;
              h.x = pack16<F16>(a[0].x, a[0].y); h.y = pack16<F16>(a[1].x, a[1].y);
              h.z = pack16<F16>(a[2].x, a[2].y); h.w = pack16<F16>(a[3].x, a[3].y);
              *reinterpret_cast<uint4*>(hi + off) = h;
            }
          }
        }
        // data rows: operand rows nzp (d_+) and nzp + 1 (d_-), 8 chunks each
        if (warp == PRODUCER_WARPS - 1 && lane < 16) {
          const int which = lane >> 3, c = lane & 7;
          float2 v[4];
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) {
            const float4 dd = rdat[c * 4 + rr];
            const float sw = rt[c * 4 + rr].sw * sc.y;
            v[rr] = which ? make_float2(sw * dd.z, sw * dd.w) : make_float2(sw * dd.x, sw * dd.y);
            if (c * 4 + rr >= nvalid) v[rr] = make_float2(0.f, 0.f);
          }
          const uint32_t off = sw_off(nzp + which, c);
          if (PASSES == 3) {
            uint4 h, l;
            split16<F16>(v, h, l);
            *reinterpret_cast<uint4*>(hi + off) = h;
            *reinterpret_cast<uint4*>(lo + off) = l;
          } else {
            uint4 h;
            h.x = pack16<F16>(v[0].x, v[0].y); h.y = pack16<F16>(v[1].x, v[1].y);
            h.z = pack16<F16>(v[2].x, v[2].y); h.w = pack16<F16>(v[3].x, v[3].y);
            *reinterpret_cast<uint4*>(hi + off) = h;
          }
        }
        {   // Kahan: tr_hi + tr_lo carries the segment's trace without FP64 arithmetic
          const float yk = trs - tr_lo, tk = tr_hi + yk;
          tr_lo = (tk - tr_hi) - yk;
          tr_hi = tk;
        }
        fence_proxy_async();
        mbar_arrive(&full[s]);
      }
      if (!ok) break;
      // epilogue: accumulator -> FP32 partial tile [col][128 lanes]
      if (!mbar_wait(acc_full, unsigned((si - s0) & 1), abort_flag, budget)) { ok = false; break; }
      tc_fence_after();
      float* out = d.gpart + size_t(slot) * size_t(ncols) * TC_M;
      const int quarter = warp & 3, group = warp >> 2;   // TMEM lanes 32*quarter..+31
      constexpr int NGROUP = PRODUCER_WARPS / 4;
      const uint32_t lane_base = uint32_t(quarter * 32) << 16;
      for (int c0 = group * 16; c0 < ncols; c0 += 16 * NGROUP) {
        float v[16];
        tmem_ld16(tmem + lane_base + uint32_t(c0), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) out[size_t(c0 + j) * TC_M + quarter * 32 + lane] = v[j];
      }
      tc_fence_before();
      mbar_arrive(acc_empty);
      // trace(G) of this warp's rows of the segment, summed over the warp in FP64 (the
      // kernel-row scale divided out exactly: it is a power of two); the reduction adds the
      // partials of all warps and segments of a subproblem in a fixed order
      double tr = (double(tr_hi) - double(tr_lo)) * pow2d(-2 * se.x);
      for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
      if (lane == 0) d.tpart[size_t(slot) * PRODUCER_WARPS + warp] = tr;
    }
    // a table copy still in flight after an early exit must land before the CTA leaves
    if (ptid == 0)
      for (long long k = tb_done; k < tb_issued; ++k) mbar_drain(&tbar[k & 1], unsigned((k >> 1) & 1));
  }

  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(&d.flags[0], 1u);
  if (warp == PRODUCER_WARPS) {
    tc_fence_after();
    tmem_dealloc(tmem, alloc_cols);
  }
}

// Largest modulus over depth of every row of the FP32 table (one warp per row).
__global__ void table_rowmax_kernel(Dev d, long long nrows) {
  const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  const float2* t = d.rowtab32 + size_t(r) * d.nzs;
  float mx = 0.f;
  for (int z = lane; z < d.nz; z += 32) {
    const float2 v = t[z];
    mx = fmaxf(mx, sqrtf(v.x * v.x + v.y * v.y));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) d.rowmax[r] = mx;
}

// Per segment: bounds of its kernel rows (sqrt(w) |g_p| |g_q| over depth, from the row
// maxima) and of its data rows, turned into power-of-two scales for the FP16 operands.
__global__ void gram_scale_kernel(Dev d) {
  __shared__ float red[2][32];
  const int slot = blockIdx.x;
  const long long r0 = d.seg_row0[slot], n = d.seg_nrow[slot];
  const float4* rhs = reinterpret_cast<const float4*>(d.rhs);
  float ma = 0.f, md = 0.f;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const GramRow e = d.gent[r0 + i];
    ma = fmaxf(ma, e.sw * d.rowmax[e.rp] * d.rowmax[e.rq]);
    const float4 v = rhs[r0 + i];
    md = fmaxf(md, e.sw * fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  for (int o = 16; o > 0; o >>= 1) {
    ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
    md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { red[0][warp] = ma; red[1][warp] = md; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < int(blockDim.x >> 5); ++w) { ma = fmaxf(ma, red[0][w]); md = fmaxf(md, red[1][w]); }
    d.gscale[slot] = make_int2(pow2_exp(ma), pow2_exp(md));
  }
}

// Sum the partial tiles of each subproblem into the FP64 Gram (both triangles) and b.  With
// df_out (the double-float factorisation follows) the lower triangle of G + lam I is written
// instead, lam = alpha * trace, each value as a double-float pair (float2) in the same 8 bytes.
// trace(G) of subproblem m: the per-warp partials of its segments, in slot and warp order.
__device__ __forceinline__ double trace_of(const Dev& d, int sl0, int sl1) {
  double t = 0.0;
  for (int i = sl0 * PRODUCER_WARPS; i < sl1 * PRODUCER_WARPS; ++i) t += d.tpart[i];
  return t;
}

// One CTA per 32 x 32 tile of G (the lower triangle with df_out, else the whole matrix),
// 32 x 8 threads: the partial tiles are read with consecutive threads on consecutive TMEM
// lanes (coalesced; a tile below the diagonal block TC_M x TC_M in its left part reads the
// transposed tile, whose lanes run along its columns), summed over the subproblem's slots in
// slot order, staged in shared memory and written as rows of G (coalesced).  CTA ntile of each
// subproblem forms b and the trace.
__global__ void __launch_bounds__(256) gram_reduce_kernel(Dev d, int df_out) {
  __shared__ double s64[32][33];
  float2* sdf = reinterpret_cast<float2*>(&s64[0][0]);   // [32][33] pairs, same storage
  const int m = blockIdx.y;
  const int nz = d.nz, nzp = nzp_of(nz), ncols = cols_of(nzp);
  const int c1 = nzp + 16;
  const int sl0 = d.m_slot0[m], sl1 = d.m_slot0[m + 1];
  const int T = (nz + 31) / 32;
  const int ntile = df_out ? T * (T + 1) / 2 : T * T;
  const long long nG = (long long)nz * nz;
  if (int(blockIdx.x) == ntile) {                      // right-hand sides and the trace
    if (threadIdx.x == 0) d.trace[m] = trace_of(d, sl0, sl1);
    for (int e = threadIdx.x; e < 2 * nz; e += blockDim.x) {
      const int zi = e >> 1, k = e & 1;
      int lanei, col;
      if (zi < TC_M) { lanei = zi; col = nzp + k; }
      else { lanei = zi - TC_M; col = c1 + (nzp - TC_M) + k; }
      double sacc = 0.0;
      for (int sl = sl0; sl < sl1; ++sl) {
        const double v = double(d.gpart[(size_t(sl) * ncols + col) * TC_M + lanei]);
        sacc += d.gscale ? v * pow2d(-d.gscale[sl].x - d.gscale[sl].y) : v;
      }
      d.b[(size_t(m) * nz + zi) * 2 + k] = sacc;
    }
    return;
  }
  int ti, tj;
  if (df_out) {
    const int t = blockIdx.x;
    ti = int((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    tj = t - ti * (ti + 1) / 2;
  } else {
    ti = blockIdx.x / T;
    tj = blockIdx.x - ti * T;
  }
  const int i0 = 32 * ti, j0 = 32 * tj;
  const bool lane_on_j = i0 >= TC_M && j0 < TC_M;     // TC_M is a multiple of 32: no tile straddles it
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  __shared__ double s_lam;
  if (df_out && ti == tj) {                           // lam for the diagonal, formed once per CTA
    if (threadIdx.x == 0) s_lam = d.alpha * trace_of(d, sl0, sl1);
    __syncthreads();
  }
  for (int k = 0; k < 4; ++k) {
    const int r = ty + 8 * k;
    const int zi = lane_on_j ? i0 + r : i0 + tx, zj = lane_on_j ? j0 + tx : j0 + r;
    if (zi >= nz || zj >= nz || (df_out && zj > zi)) continue;
    int lanei, col;
    if (zi < TC_M) { lanei = zi; col = zj; }
    else if (zj < TC_M) { lanei = zj; col = zi; }
    else { lanei = zi - TC_M; col = c1 + (zj - TC_M); }
    if (df_out) {
      // the partial tiles (FP32, exact power-of-two scales) summed as a double-float pair by
      // TwoSum on the FP32 pipes, then lam added on the diagonal
      float sh = 0.f, sl_ = 0.f;
      for (int sl = sl0; sl < sl1; ++sl) {
        float v = d.gpart[(size_t(sl) * ncols + col) * TC_M + lanei];
        if (d.gscale) v = ldexpf(v, -2 * d.gscale[sl].x);
        const float t = __fadd_rn(sh, v), bb = __fsub_rn(t, sh);
        sl_ = __fadd_rn(sl_, __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(v, bb)));
        sh = t;
      }
      if (zi == zj) {
        const double lam = s_lam;
        const float lh = __double2float_rn(lam), ll = __double2float_rn(lam - double(lh));
        const float t = __fadd_rn(sh, lh), bb = __fsub_rn(t, sh);
        sl_ = __fadd_rn(sl_, __fadd_rn(__fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(lh, bb)), ll));
        sh = t;
      }
      const float hs = __fadd_rn(sh, sl_);
      sdf[(zi - i0) * 33 + (zj - j0)] = make_float2(hs, __fsub_rn(sl_, __fsub_rn(hs, sh)));
    } else {
      double sacc = 0.0;
      for (int sl = sl0; sl < sl1; ++sl) {
        const double v = double(d.gpart[(size_t(sl) * ncols + col) * TC_M + lanei]);
        sacc += d.gscale ? v * pow2d(-2 * d.gscale[sl].x) : v;
      }
      s64[zi - i0][zj - j0] = sacc;
    }
  }
  __syncthreads();
  for (int k = 0; k < 4; ++k) {
    const int r = ty + 8 * k, zi = i0 + r, zj = j0 + tx;
    if (zi >= nz || zj >= nz || (df_out && zj > zi)) continue;
    if (df_out) reinterpret_cast<float2*>(d.G + size_t(m) * nG)[size_t(zi) * nz + zj] = sdf[r * 33 + tx];
    else d.G[size_t(m) * nG + size_t(zi) * nz + zj] = s64[r][tx];
  }
}

}  // namespace

int tc_cols(int nz) { return cols_of(nzp_of(nz)); }

int gram_trace_parts() { return PRODUCER_WARPS; }

int tc_smem_bytes(int nz, int passes) {
  const int zr = zrows_of(nzp_of(nz));
  const int stages = stages_of(passes), ncomp = passes == 1 ? 1 : 2;
  return 1024 + stages * ncomp * zr * ROWB + 2 * TAB_BYTES + (2 * stages + 6) * 8 + 16;
}

cudaError_t prepare_gram_tc(const Dev& d) {
  const int smem = tc_smem_bytes(d.nz, d.passes);
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (d.f16)
    return d.passes == 3 ? cudaFuncSetAttribute(gram_tc_kernel<3, true>, attr, smem)
                         : cudaFuncSetAttribute(gram_tc_kernel<1, true>, attr, smem);
  return d.passes == 3 ? cudaFuncSetAttribute(gram_tc_kernel<3, false>, attr, smem)
                       : cudaFuncSetAttribute(gram_tc_kernel<1, false>, attr, smem);
}

int gram_scale_launches(const Dev& d, bool rowmax_ready) {
  return d.f16 && d.ncta_gram > 0 ? (rowmax_ready ? 1 : 2) : 0;
}

cudaError_t launch_gram_scale(const Dev& d, cudaStream_t s, bool rowmax_ready) {
  if (!d.f16 || d.ncta_gram <= 0) return cudaSuccess;
  const long long nrows = (long long)d.nf * d.nk;
  if (!rowmax_ready) table_rowmax_kernel<<<unsigned((nrows + 7) / 8), 256, 0, s>>>(d, nrows);
  gram_scale_kernel<<<d.nseg, 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_gram_tc(const Dev& d, cudaStream_t s) {
  const int smem = tc_smem_bytes(d.nz, d.passes);
  cudaError_t e;
  if (d.ncta_gram > 0) {
    if (d.f16) {
      if (d.passes == 3) gram_tc_kernel<3, true><<<d.ncta_gram, NTHREADS, smem, s>>>(d);
      else gram_tc_kernel<1, true><<<d.ncta_gram, NTHREADS, smem, s>>>(d);
    } else {
      if (d.passes == 3) gram_tc_kernel<3, false><<<d.ncta_gram, NTHREADS, smem, s>>>(d);
      else gram_tc_kernel<1, false><<<d.ncta_gram, NTHREADS, smem, s>>>(d);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_gram_reduce(const Dev& d, cudaStream_t s, int df_out) {
  const int T = (d.nz + 31) / 32;
  dim3 g(unsigned((df_out ? T * (T + 1) / 2 : T * T) + 1), d.nsub);
  gram_reduce_kernel<<<g, 256, 0, s>>>(d, df_out);
  return cudaGetLastError();
}

}  // namespace edt
