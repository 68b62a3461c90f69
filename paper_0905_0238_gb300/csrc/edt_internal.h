// Internal declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <vector>
#include <string>

#include "../../include/edt.h"

namespace edt {

// Packed row of a midpoint-wavenumber system: (frequency index f, receiver wavenumber
// index p, weight flag).  Weight 2 marks a row that stands for itself and its reciprocal
// partner (-q, -p), which carries the same kernel row.
__host__ __device__ inline uint32_t row_pack(int f, int p, int w2) {
  return (uint32_t(f) << 16) | (uint32_t(w2 & 1) << 15) | uint32_t(p);
}
__host__ __device__ inline int row_f(uint32_t r) { return int(r >> 16); }
__host__ __device__ inline int row_p(uint32_t r) { return int(r & 0x7fffu); }
__host__ __device__ inline int row_w2(uint32_t r) { return int((r >> 15) & 1u); }

// Per-row operand metadata of the tensor-core Gram (fixed by the row plan, written once per
// workspace): the two rows p, q of the FP32 row table whose elementwise product is the
// kernel row (row r of the table starts at element r * nzs), as byte offsets and as row
// indices, and sqrt(weight).  The data
// of a row, (d_+, d_-) as a float4 in the right-hand-side array, are scaled by sw on use.
// Line geometry: the table is sqrt|s_f| g and the rows are g(|k_p|), g(|k_q|); window
// geometry: the table holds the assembled kernel rows and q is a row of ones.
struct GramRow {
  unsigned long long bp, bq;     // byte offsets of the two table rows (row * nzs * 8)
  float sw;                      // sqrt(weight)
  unsigned rp, rq;               // the two rows' indices
  float pad;
};

// Wavenumber band of one frequency kept by the evanescent cut: signed indices
// [lo, lo + w), and the offsets (in complex elements, within the chunk buffers) of the
// band-limited row spectrum Y_f [N][w] and transformed plane Xc_f [w][w].
struct BandInfo {
  int lo, w;
  long long yoff, xoff;
};

// One chunk of frequency planes of the band-limited transform: planes [f0, f1), column-pass
// blocks [bcol0, bcol0 + nbcol) of the block table, nrow rows of all subproblems at these
// frequencies, ci = index of its row-count prefix array.
struct BandChunk {
  int f0, f1, bcol0, nbcol;
  long long nrow;
  int ci;
};

// Per-frequency constants: omega~ = omega + i eps, |s_f| with s_f = omega~^2 dz/dx, and
// the unit phase conj(s_f)/|s_f| that moves the complex prefactor onto the data.
struct FreqConst {
  double om_re, om_im;
  double s_abs;
  double rot_re, rot_im;
  double lim;        // (cutoff * f) * L
};

// Device-side view of the workspace and constant tables of one context.
struct Dev {
  int N, nk, nz, nf, nsub, nlayer;
  int nzs;                      // row stride of the FP32 table: nz rounded up to even
  int precision, passes, fold, chol_df;
  int chol_tc;                  // double-float factorisation with the sliced tensor-core updates
  // window geometry (geom == EDT_GEOM_WINDOW): ny x nx midpoints (nx == N), wy x wx
  // half-offsets, W = wx * wy, nxy = nx * ny
  int geom, ny, wx, wy, W, nxy;
  double dy;
  double alpha, dx, dz;
  // constant tables
  const FreqConst* fc;          // [nf]
  const double* layer_top;      // [nlayer]
  const double* layer_vel;      // [nlayer]
  const int* z_layer;           // [nz] layer of each sample depth
  const double* z_off;          // [nz] depth below that layer's top
  const float* z_off32;         // [nz][4] (off hi, off lo, 2h - off hi, 2h - off lo) as floats
  const float* fc32_sqrt_s;     // [nf] sqrt|s_f| as float
  const uint32_t* rows;         // [rows_solved], grouped by m
  const long long* row_off;     // [nsub + 1]
  long long rows_max_sub;       // most rows of any subproblem
  const long long* row_off_mf;  // [nsub][nf + 1]: first row of frequency f within subproblem m
  int fchunk;                   // frequency planes per chunk of the full-plane transform
  // launch shapes picked by the autotuner (edt_autotune): band-column block width (4, 8,
  // 16), refinement CTA shape (0: 4 warps x 32 rows, 1: 8 x 32, 2: 4 x 64, 3: 8 x 16),
  // depths per kernel-row cluster of the window geometry (2, 4, 8)
  int tune_bc, tune_rf, tune_zc;
  // band-limited transform (mixed path)
  const BandInfo* band;         // [nf]
  const int2* bcol;             // column-pass block table: (f, first band column)
  const long long* cpre;        // [nchunk][nsub + 1] chunk rows of subproblems < m
  float2* Yc;                   // band row spectra of one chunk
  float2* Xc;                   // band planes of one chunk
  const double2* tw64;          // [N/2] exp(-2 pi i k / N)
  const float2* tw32;           // [N/2]
  const double* kval;           // [nk] |k| of each table row (window geometry), else null
  const float2* rowtab32;       // row table the tensor-core Gram and the refinement read
  // window geometry
  const int* pair_m;            // [nsub] midpoint index my * nx + mx of each pair's k_m
  const int* fj_off;            // [nf * W + 1] entry ranges of the (f, j) lists
  const int2* fj_ent;           // (midpoint index, row) of every row, grouped by (f, j)
  const int* jact;              // [nf][W] active offset wavenumbers of each frequency (those
                                //   with kept rows), compacted; then -1
  const int* jmap;              // [nf][W] position of j among the active ones, or -1
  float2* Gs;                   // [nz][ny][nx] G(y, z) of one frequency
  float2* U;                    // [W][nz][ny/2 + 1][nx] window products of one frequency
                                //   (centrosymmetric in y: rows 0..ny/2 stored)
  float2* Dw;                   // [nf][W][ny][nx] window-transformed data
  float2* A32;                  // [rows + 1][nzs] kernel rows, then a row of ones
  long long ones_row;           // index of the ones row in A32
  const int* seg_m;             // tensor-core Gram: per segment its m      [nseg]
  const long long* seg_row0;    //                   first row, row count    [nseg], [nseg]
  const long long* seg_nrow;
  const int* cta_seg0;          //                   per CTA first segment   [ncta + 1]
  const int* m_slot0;           //                   per m first partial slot [nsub + 1]
  int nseg, ncta_gram;
  // scratch
  double2* coef;                // [nf][nk][nlayer][7] recursion coefficients (FP64)
  float* coef32;                // [nf][nk][nlayer][8] FP32 copies for the fast evaluation
  double2* g64;                 // [nf][nk][nz]
  float2* g32;                  // [nf][nk][nzs] sqrt|s_f| g, mixed path (padding zero)
  float2* g32lo;                // [nf][nk][nzs] its FP32 remainder: g32 + g32lo carries the
                                //   FP64 table to ~1e-14 (line geometry, mixed path)
  float* rowmax;                // [nf * nk] max over depth of |g32| per table row
  int2* gscale;                 // [nseg] tensor-core Gram: exponents k of the power-of-two
                                //   scales 2^k of each segment's kernel rows and data rows
                                //   (FP16 operands)
  int f16;                      // tensor-core Gram operands: 1 = FP16 with per-segment
                                //   scales (line geometry), 0 = BF16 (window geometry)
  int resid_df;                 // refinement residual: 1 = double-float accumulation from
                                //   the double-float table, 0 = FP32 products
  void* X;                      // [fchunk][N][N] complex, path precision (one chunk of planes)
  void* Dstage;                 // host-call staging of D (complex128-sized)
  void* Vstage;                 // host-call staging of V (double-sized)
  void* rhs;                    // [rows_solved][2] complex, path precision
  GramRow* gent;                // [rows_solved + 32] tensor-core Gram row metadata (mixed)
  float* gpart;                 // tensor-core Gram partial tiles [nslot][TM_COLS * 128]
  double* G;                    // [nsub][nz][nz]  Gram, then its Cholesky factor
  double* dinv;                 // [nsub][nz]      1 / diagonal of the factor
  float* L32;                   // [nsub][nz][nz]  FP32 copy of the factor (mixed path: the
                                //                 refinement's correction solves)
  float* dinv32;                // [nsub][nz]
  double* b;                    // [nsub][nz][2]
  double* trace;                // [nsub]
  double* tpart;                // [nslot][gram_trace_parts()] tensor-core Gram: trace of each
                                //   segment per producer warp, summed in order by the reduction
  double* x;                    // [nsub][nz][2]
  double* r;                    // [nsub][nz][2]
  double* rpart;                // [nsub][rf_stride][nz][2] refinement: each CTA's partial
  int rf_stride;                //   residual, summed in CTA order into r (deterministic)
  double2* vhat;                // [nsub][nz]
  double2* vfull;               // [N][nz] scratch for the forward model (Vhat of V)
  // misfit gradients (line geometry, mixed path)
  double2* gscr;                // [nf][nlayer][8][nk] depth-march states and cotangents
  double2* adj;                 // [N][nz] Ahat = F^H R2 summed over frequencies
  double* gacc;                 // [1 + nlayer] sum |R2|^2
  double* gcpart;               // [warps of the reverse march][nlayer] partial dJ/dc_l
  float2* gbar;                 // [nf][N][nz] dJ/dg per full lateral index (aliases g64)
  // dL/dc through the damped solve (line geometry, mixed path)
  float4* rowc;                 // [rows_solved][2] per row (u_+, u_-) = d - A x, (v_+, v_-) = -A mu
  float4* xmu;                  // [nsub][nz] (x_+, x_-, mu_+, mu_-) in FP32
  double* gam;                  // [nsub] -2 alpha sum_k mu_k . x_k
  const int2* tref;             // [2 rows_solved] (row, m << 1 | side), grouped by table row
  const long long* tref_off;    // [nf * nk + 1] the groups' offsets
  int refine_nodata;            // refinement residual without the data term (adjoint solves)
  int* status;                  // [nsub]
  unsigned int* flags;          // [8] device-side error flags; [0]: a tensor-core Gram wait expired
  long long wait_cycles;        // budget of the tensor-core Gram's bounded waits (0: about 2 s)
  int wait_stall;               // wait test: the Gram's MMA issuer waits on a barrier that
                                //   nothing completes, so the kernel takes its timeout path
  // streaming batches (per-subproblem sizes; null for a context's own subproblems)
  const int* sub_n;             // [nsub] unknowns of subproblem m
  const long long* sub_goff;    // [nsub] element offset of its matrix in G and L32
  const long long* sub_voff;    // [nsub] element offset of its vectors (dinv; b, x, r x 2)
  const int* sub_order;         // [nsub] launch order of the factorisations (largest first), or null
  // solver variants (FP64 line path): vertical-wavenumber basis and restricted systems
  int solver;                   // EDT_SOLVE_DAMPED or EDT_SOLVE_TSVD
  double tsvd_tol;
  const double* kz_P;           // [nz][nz] orthonormal real depth basis, columns by |k_z|
  const int* kz_p;              // [nsub] kept columns p(m) (null: no disk)
  const long long* kz_goff;     // [nsub] m * nz * nz
  const long long* kz_voff;     // [nsub] m * nz
  double* kz_G;                 // [nsub][p][p] restricted normal matrices (stride nz * nz)
  double* kz_T;                 // [nsub][nz][p] scratch G P_p
  double* kz_b;                 // [nsub][nz][2] restricted right-hand sides
  double* kz_x;                 // [nsub][nz][2] restricted solutions
};

// Record a CUDA error for edt_last_cuda_error; returns EDT_ECUDA.
int record_cuda_error(cudaError_t e);

// ---- launchers (each returns cudaGetLastError()) ---------------------------------------
constexpr int GREEN_G64 = 1, GREEN_G32 = 2, GREEN_G32DF = 4;   // tables launch_green writes
constexpr int GREEN_G32F = 8;
// GREEN_G32 alone: the fast FP32 evaluation for the mixed path (no FP64 table);
// GREEN_G32F: the same table from coefficients formed in FP32 (green_coef32; about the number
// of layers times FP32 rounding, for the line inversion with the FP32 residual);
// GREEN_G32DF: the FP64 evaluation written as the double-float pair g32 + g32lo (no g64)
cudaError_t launch_green(const Dev& d, cudaStream_t s, int tables);

// Data transform of frequency planes [f0, f0 + nfc) into X, then the split right-hand
// sides of every subproblem's rows at those frequencies (X holds only the chunk).
template <typename T>
cudaError_t launch_transform(const Dev& d, const void* D, int D_dtype, int f0, int nfc, cudaStream_t s);
template <typename T>
cudaError_t launch_rhs(const Dev& d, int f0, int nfc, cudaStream_t s);
// Tensor-core Gram row metadata from the row plan (once per workspace, mixed path).
cudaError_t launch_gent_static(const Dev& d, cudaStream_t s);
// Band-limited transform and right-hand sides of one chunk (FP32, mixed path, 32 <= N <= 1024).
bool band_supported(int N);
cudaError_t launch_band_chunk(const Dev& d, const BandChunk& ch, const void* D, int D_dtype, cudaStream_t s);
cudaError_t prepare_band(const Dev& d);

// Window geometry (csrc/fa.cu): kernel rows of frequency f into A32, data transform and
// right-hand sides, the inverse transform to V[ny][nx][nz]; supported grids and windows.
bool fa_supported(int nx, int ny, int wx, int wy);
cudaError_t launch_fa_rows(const Dev& d, int f, int nact, double2 cf, cudaStream_t s);
cudaError_t launch_fa_data(const Dev& d, const void* D, int D_dtype, cudaStream_t s);
cudaError_t launch_fa_inverse(const Dev& d, void* V, int V_dtype, cudaStream_t s);
cudaError_t launch_fa_setup(const Dev& d, long long nrows, cudaStream_t s);
cudaError_t prepare_fa(const Dev& d);
// FP64 2D transform of [planes][ny][N] in place (ny == N or 1), sign +-1, times scale.
cudaError_t fft2_f64(const Dev& d, double2* X, int planes, int ny, int sign, double scale, cudaStream_t s);

cudaError_t launch_gram_f64(const Dev& d, cudaStream_t s);
cudaError_t launch_gram_tc(const Dev& d, cudaStream_t s);       // partial tiles + trace
int gram_scale_launches(const Dev& d, bool rowmax_ready);       // FP16 operand scales: 0, 1 or 2 kernels
int gram_trace_parts();                                         // trace partials per Gram segment
// per-segment FP16 operand scales; rowmax_ready: the FP32 table's evaluation (green_eval32)
// has already written the row maxima
cudaError_t launch_gram_scale(const Dev& d, cudaStream_t s, bool rowmax_ready);
// partials -> G, b (FP64); df_out: the lower triangle of G + lam I as double-float pairs
cudaError_t launch_gram_reduce(const Dev& d, cudaStream_t s, int df_out = 0);
cudaError_t launch_trace_diag(const Dev& d, cudaStream_t s);   // trace[m] = sum_z G[m][z][z]
int chol_launches(int nz);                                      // kernels of launch_chol_solve
// The double-float factorisation (csrc/chol_df.cu) runs its updates with a one-step look-ahead
// on two streams when given a side stream and 2 * ceil(nz / 32) + 1 events (joined back into s
// before it returns).
struct CholLookahead {
  cudaStream_t side;
  const cudaEvent_t* ev;
  int nev;
};
cudaError_t launch_chol_solve(const Dev& d, int trace_mode, cudaStream_t s, const CholLookahead* la = nullptr);
// The double-float factorisation and solve (csrc/chol_df.cu), used when d.chol_df is set.
cudaError_t prepare_chol_dfloat(const Dev& d);
int chol_dfloat_launches(int nz);
cudaError_t launch_chol_dfloat_resolve(const Dev& d, cudaStream_t s);           // x = (LL^T)^-1 b
cudaError_t launch_chol_dfloat_export(const Dev& d, double* out, cudaStream_t s); // factor as FP64
cudaError_t launch_chol_dfloat(const Dev& d, int trace_mode, cudaStream_t s, const CholLookahead* la = nullptr);
// r = Ahat^T (dhat - Ahat x): per-CTA partials, then their sum in CTA order (2 launches)
cudaError_t launch_refine(const Dev& d, cudaStream_t s);
int refine_stride(long long rows_max_sub);                      // refinement CTAs per subproblem, at most
cudaError_t launch_refine_update(const Dev& d, cudaStream_t s);   // x += (LL^T)^-1 (r - lam x)
cudaError_t launch_inverse(const Dev& d, void* V, int V_dtype, cudaStream_t s);
cudaError_t launch_forward(const Dev& d, const void* V, int V_dtype, void* D, int D_dtype,
                           cudaStream_t s);
// vfull[m][z] = sum_x V[x][z] e^{-i k_m x} (FP64)
cudaError_t launch_lateral_dft(const Dev& d, const void* V, int V_dtype, cudaStream_t s);
// out[x][z] = scale Re sum_m in[m][z] e^{+i k_m x} over every m (FP64 transform)
cudaError_t launch_lateral_idft_real(const Dev& d, const double2* in, double scale, void* out,
                                     int out_dtype, cudaStream_t s);

// Adjoint of the data transform on the chunk's planes X (FP32) into D[f0 .. f0 + nfc).
cudaError_t launch_transform_adjoint(const Dev& d, void* D, int D_dtype, int f0, int nfc, cudaStream_t s);
// x = (LL^T)^-1 b with the factors of the last factorisation (no refactorisation).
cudaError_t launch_chol_resolve(const Dev& d, cudaStream_t s);
// The vector-Jacobian products of the last edt_invert (mixed line path) for Vbar = dL/dV:
// Dbar = S^T Vbar (S: D -> V, linear) when Dbar is set, and gc[l] = dL/dc_l through the damped
// solve (the kernel rows and lam depend on the reference) when gc is set (needs
// grad_supported and the row groups).  mu = (G + lam I)^-1 xbar with `refine` refinement
// steps like the forward solve.
cudaError_t launch_invert_vjp(const Dev& d, const void* Vbar, int Vbar_dtype, void* Dbar, int Dbar_dtype,
                              double* gc, int refine, cudaStream_t s);

// Misfit J = ||F V - D||^2 and its gradients (csrc/grad.cu); layers the reverse-mode depth
// march supports (its per-(f, k) scratch is sized by it).
constexpr int GRAD_MAX_LAYERS = 64;
bool grad_supported(const Dev& d);
cudaError_t launch_misfit_grad(const Dev& d, const void* V, int V_dtype, const void* D, int D_dtype,
                               double* J, void* gV, double* gc, cudaStream_t s);
// V = F^T D, the adjoint Born operator (line geometry; the mixed path needs grad_supported).
cudaError_t launch_adjoint(const Dev& d, const void* D, int D_dtype, void* V, int V_dtype, cudaStream_t s);
// FP64 data transform of frequency planes [f0, f0 + nfc) and their adjoint-Born contraction,
// accumulated into vfull.
cudaError_t launch_adjoint64_chunk(const Dev& d, const void* D, int D_dtype, int f0, int nfc, cudaStream_t s);

// Streaming batches: Cholesky and refinement update with per-subproblem sizes (<= nmax).
cudaError_t prepare_chol_var(int nmax);
cudaError_t launch_chol_var(const Dev& d, int nmax, cudaStream_t s);
cudaError_t launch_refine_update_var(const Dev& d, int nmax, cudaStream_t s);
// Blocked Cholesky over several launches (panel + tile update per 32-column step, then the
// solves), in double-float: d.G holds a float2 (hi, lo) pair in each 8-byte slot; see chol.cu
// for the step lists.  chol_blocked_tiles: update tiles of step k0 of an
// n-unknown subproblem; chol_block_cols: the panel width.
cudaError_t launch_chol_blocked(const Dev& d, bool var, int nmax, int nstep, const int* act_dev,
                                const int* nact_host, const long long* tpre_dev,
                                const long long* ntile_host, const long long* cpre_dev,
                                const long long* nchunk_host, int trace_mode, cudaStream_t s);
int chol_blocked_tiles(int n, int k0);
int chol_blocked_chunks(int n, int k0);   // 32-row panel chunks below the diagonal block
int chol_block_cols();

// Solver variants (csrc/variants.cu): the truncated SVD (nz <= TSVD_MAX_NZ) and the
// vertical-wavenumber disk, in place of the Cholesky stage of the FP64 line path.
constexpr int TSVD_MAX_NZ = 96;
size_t tsvd_smem_bytes(int p);
cudaError_t prepare_variants(int nz);
cudaError_t launch_solve_variant(const Dev& d, cudaStream_t s);

// One-time kernel attribute setup (opt-in shared memory), done outside any stream capture.
cudaError_t prepare_fft(const Dev& d);
cudaError_t prepare_chol(const Dev& d);
cudaError_t prepare_gram_tc(const Dev& d);
cudaError_t prepare_grad(const Dev& d);

// Tensor-core Gram tiling (shared by host planning and the kernel).
constexpr int TC_M = 128;              // MMA rows (depth unknowns per M tile)
constexpr int TC_KC = 32;              // complex rows per pipeline stage (K = 64 real rows)
int tc_cols(int nz);                   // TMEM columns of one subproblem's accumulator
int tc_smem_bytes(int nz, int passes); // dynamic shared memory of the Gram kernel

}  // namespace edt
