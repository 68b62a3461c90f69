// Internal layout of a streaming batch (not installed): one descriptor per request, the batch's
// device view, and the launchers of csrc/stream.cu.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "edt_internal.h"

namespace edt {

constexpr int ST_MAX_NZ = 512;          // unknowns per request (shared memory of the substitutions)
constexpr int ST_MAX_LAYERS = 64;       // layers of a request's reference
constexpr int ST_TILE = 128;            // depth rows per tensor-core tile
constexpr int ST_DROWS = 16;            // data rows after the depth rows (d_+, d_-, zeros)
constexpr int ST_KC = 32;               // complex rows per K stage (64 real rows = 128 B of BF16)
constexpr int ST_REFINE_ROWS = 256;     // rows per refinement CTA

// One request of a batch.  Offsets index the batch arrays of StBatch (element units).
struct StSub {
  int nz, nl, nf, nk, nrow;
  int nzs;                // row stride of the FP32 Green's table (nz rounded up to 32)
  int nzt;                // 128-depth tiles
  int kst;                // K stages of 32 complex rows
  double dz, z0, eps, dx, alpha;
  float eps2, dzdx;       // eps^2 and dz / dx as FP32
  long long o_lay;        // dbl: layer tops [nl], velocities [nl], 1 / velocity^2 [nl]
  long long o_freq;       // dbl: frequencies [nf] (Hz)
  long long o_kval;       // dbl: wavenumbers [nk] (rad/m)
  long long o_row;        // rows / data [nrow]
  long long o_v;          // depth vectors: zt, zl, dinv, dinv32 [nz]; b, x, r [nz][2]
  long long o_coef;       // coef: [nf][nk][nl][8]
  long long o_g;          // g32: [nf][nk][nzs]
  long long o_tile;       // tiles (bytes): [kst][hi, lo][nzt * 128 + 16][128]
  long long o_G;          // G (double-float pairs), L32 (float): [nz][nz]
};

// Tensor-core Gram work item: request, depth tile of the rows (ti) and of the columns (tj >= ti).
struct StItem { int req, ti, tj, pad; };

// Device view of one batch (every pointer into the batch's arena).
struct StBatch {
  int nreq, ncta;
  const StSub* sub;              // [nreq]
  const long long* pre_z;        // [nreq + 1] prefix sums of nz
  const long long* pre_fk;       //            of nf * nk
  const long long* pre_eb;       //            of ceil(nf * nk / 8)  (table-evaluation CTAs)
  const long long* pre_tw;       //            of kst * (4 nzt + 1)  (tile-writer warps)
  const long long* pre_rc;       //            of ceil(nrow / 256)   (refinement CTAs)
  const long long* pre_rz;       //            of ceil(nrow / 256) * nz (refinement partials / 2)
  const StItem* items;           // Gram items grouped by CTA
  const int* cta_item0;          // [ncta + 1]
  const double* dbl;             // layer tables, frequencies, wavenumbers
  const int4* rows;              // (f, p, q, 0)
  const float4* data;            // (d_+ re, d_+ im, d_- re, d_- im)
  float4* drot;                  // data times conj of the unit phase of s_f (the rows' phase)
  float4* zt;                    // (off hi, off lo, 2h - off hi, 2h - off lo)
  int* zl;                       // layer of each depth
  float* coef;
  float2* g32;
  unsigned char* tiles;
  double* G;                     // [sum nz^2] double-float pairs (float2 per 8-byte slot)
  float* L32;
  double* dinv;
  float* dinv32;
  double* b;
  double* x;
  double* r;
  double* trace;                 // alpha trace(Ahat^T Ahat), then lam
  double* twtr;                  // [tot_tw] alpha * trace part of each tile-writer warp
  double* rcp;                   // [pre_rz[nreq]][2] each refinement CTA's partial residual
  int* status;
  long long* row_off;            // [nreq + 1] prefix sums of nrow
  int* sub_n;                    // [nreq]
  long long* sub_goff;           // [nreq]
  long long* sub_voff;           // [nreq]
  int* sub_order;                // [nreq] requests by decreasing nz (Cholesky launch order)
  unsigned int* flags;           // [1] tensor-core wait expired
  long long wait_cycles;         // budget of the Gram's bounded waits (0: about 2 s)
  int wait_stall;                // wait test: the Gram issuer waits on a barrier nothing completes
  // launch extents (host side)
  long long tot_z, tot_fk, tot_eb, tot_tw, tot_rc;
  // blocked Cholesky: per 32-column step k the active requests (device, [nstep][nreq]), their
  // prefix sums of update tiles (device, [nstep][nreq + 1]); counts on the host
  int cb_nstep;
  const int* cb_act;
  const long long* cb_tpre;
  const int* cb_nact_host;
  const long long* cb_ntile_host;
  const long long* cb_cpre;      // [nstep][nreq + 1] prefix sums of the active requests' panel chunks
  const long long* cb_nchunk_host;
};

constexpr int ST_NKERNEL = 8;
extern const char* const kStreamKernels[ST_NKERNEL];   // names of the eight stages

int st_gram_smem_bytes();
cudaError_t prepare_stream();
// The eight stages of one batch on stream s (nmax: largest nz of the batch); with ev
// non-null, ev[0..8] are recorded before the first, between consecutive and after the last.
cudaError_t launch_stream_batch(const StBatch& b, int nmax, cudaStream_t s, cudaEvent_t* ev);

}  // namespace edt
