/*
 * edt.h - C ABI of the GB300 (sm_103a) extended-diffraction-tomography library.
 *
 * The library solves the linear (first-order Born) seismic inverse problem of
 * R. B. Schlottmann, "Extended diffraction tomography": surface data D(omega, xs, xr)
 * over a laterally invariant reference c0(z) are mapped to the scattering potential
 * V(x, z) = 1/c^2 - 1/c0^2 (Section "Two dimensions", eq. Born and the definition of V
 * after it).  The 2D problem decouples into one independent 1D depth problem per
 * midpoint wavenumber k_m (eqs. DMV and M); each is split into real systems for
 * Re Vhat and Im Vhat (eq. Split) and solved by damped least squares; the negative
 * wavenumbers follow from Vhat(-k_m) = conj Vhat(k_m) (eq. VSym).
 *
 * Discrete model (shared by every entry point):
 *   - lateral grid x_i = i dx, i < nx, periodic with L = nx dx; one source and one
 *     receiver at every grid point on z = 0; k_n = 2 pi n'/L, n' = n (n <= nx/2) or n - nx;
 *   - depths z_j = z0 + (j + 1/2) dz, j < nz;
 *   - complex frequency omega~_f = 2 pi freq_hz[f] + i eps (the paper's omega -> omega + i eps);
 *   - g(k, z) solves g'' + (omega~^2/c0(z)^2 - k^2) g = -delta(z) (the reference
 *     Green's-function equation after a lateral Fourier transform), radiating away from
 *     the surface source, with the top layer continued above z = 0 (no free surface);
 *   - kernel rows M[(f, p), j] = (omega~_f^2 dz/dx) g(k_p, z_j) g(k_{p-m}, z_j)
 *     (eq. M with every offset recorded, so the aperture sinc is a delta);
 *   - data transform D2(p, q) = sum_is sum_ir D(is, ir) exp(-i k_p x_ir) exp(+i k_q x_is);
 *   - per 0 <= m <= nx/2: minimise ||Ahat x - dhat||^2 + lam ||x||^2 with
 *     Ahat = [Re M; Im M], lam = alpha * trace(Ahat^T Ahat), dhat from d_+ and d_- of
 *     eq. Split; Vhat(k_m) = x_+ + i x_- (x_- = 0 at m = 0 and m = nx/2);
 *   - V(x, z) = (1/nx) sum_m Vhat(k_m, z) exp(+i k_m x).
 *   Rows with a leg evanescent in the slowest layer are dropped when cutoff > 0:
 *   row (f, p) of m is kept iff |p'| c_min < (cutoff f) L and |q'| c_min < (cutoff f) L,
 *   q = (p - m) mod nx, evaluated in IEEE double exactly in that order.
 *
 * Finite-aperture geometry (geometry = EDT_GEOM_WINDOW; Section "A practical 3D geometry"
 * with the aperture sinc of eq. M kept): a periodic nx x ny midpoint grid (spacings dx, dy;
 * ny = 1 is a 2D line), data recorded for every half-offset w of the window
 * [-wx/2, wx/2) x [-wy/2, wy/2) grid steps, source at m - w and receiver at m + w:
 *   - G(y, z) = (1/(L_x L_y)) sum_a exp(i k_a.y) g(|k_a|, z), k_a on the 2D grid;
 *   - Born data D(f, m, w) = omega~^2 dx dy dz sum_j sum_x G(m + w - x, z_j) V(x, z_j) G(x - m + w, z_j);
 *   - d(k_m; f, j) = sum_w exp(-2 pi i j.w/W) sum_m exp(-i k_m.m) D(f, m, w) (j, w signed);
 *   - rows M(k_m; f, j, z) = sum_w exp(-2 pi i j.w/W) omega~^2 dx dy dz
 *                            sum_y exp(i k_m.(y - w)) G(2w - y, z) G(y, z);
 *   - M(-k_m) = M(k_m) row by row, so one real damped least-squares problem per pair
 *     {k_m, -k_m} (eq. Split), lam = alpha trace(Gram);
 *   - cut: row (f, j) of k_m is kept iff c_min^2 ((m_x'/L_x +- j_x/(wx dx))^2 +
 *     (m_y'/L_y +- j_y/(wy dy))^2) < (2 cutoff f)^2 for both signs (cutoff <= 0: all rows);
 *   - V(x, z) = (1/(nx ny)) sum_m Vhat(k_m, z) exp(i k_m.x), Vhat(-k_m) = conj Vhat(k_m).
 *   Pairs are numbered my = 0..ny/2 and, within, mx = 0..nx-1 (mx = 0..nx/2 on the rows
 *   my = 0 and my = ny/2, whose other half is the conjugate); layouts D
 *   [nfreq][ny][nx][wy][wx], V [ny][nx][nz].  Mixed precision only.
 *
 * Conventions for every call:
 *   - Pointers named *_dev are CUDA device pointers of the current device; *_host are
 *     host pointers (pinned memory recommended).  Complex data are interleaved (re, im).
 *   - Layouts are row-major: D is [nfreq][nx (source)][nx (receiver)], V is [nx][nz],
 *     Vhat is [nx/2 + 1][nz], g is [nfreq][nx/2 + 1][nz].
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Every
 *     device call is asynchronous on that stream; results are valid after it syncs.
 *   - The caller owns every input/output buffer and the device workspace; nothing is
 *     allocated on the device after edt_create (edt_invert is safe to capture in a graph
 *     once edt_set_workspace has run).  edt_create allocates host memory only.
 *   - edt_invert forks one internal stream (created by edt_set_workspace) from `stream` for
 *     the depth march, which overlaps the data transform, and joins it back before the
 *     Gram; to the caller the call is ordered on `stream` as a whole.
 *   - Errors are negative return codes (below); no exception crosses the ABI.  A context
 *     must not be used by two threads at once.
 */
#ifndef EDT_H
#define EDT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define EDT_OK            0
#define EDT_EINVAL       -1   /* invalid argument or configuration                        */
#define EDT_ENOMEM_WS    -2   /* workspace not set or smaller than edt_create reported     */
#define EDT_ENOTPD       -3   /* a damped normal matrix was not positive definite          */
#define EDT_ETIMEOUT     -4   /* a bounded device-side wait expired                        */
#define EDT_ENONFINITE   -5   /* non-finite value met in the data or a factorisation       */
#define EDT_ECUDA        -6   /* a CUDA runtime call failed (see edt_last_cuda_error)      */
#define EDT_EUNSUPPORTED -7   /* valid request outside what this build implements          */

/* ---- enumerations ---------------------------------------------------------------- */
#define EDT_FP64   0   /* every stage in IEEE double                                          */
#define EDT_MIXED  1   /* FP32 transforms, tensor-core Gram from 16-bit hi/lo operand pairs
                          (FP16 with power-of-two scales on the line geometry, BF16 on the
                          window geometry) with FP32 accumulation, a Cholesky of FP64-class
                          accuracy (double-float on the FP32 pipes by default, native FP64
                          with chol_df = 2) and iterative refinement with an FP64-summed
                          residual                                                         */

#define EDT_GEOM_LINE    0   /* 2D line, every source/receiver pair recorded (default)  */
#define EDT_GEOM_WINDOW  1   /* finite half-offset window on an nx x ny midpoint grid   */

#define EDT_C64    0   /* complex64 data (interleaved float)   */
#define EDT_C128   1   /* complex128 data (interleaved double) */
#define EDT_F32    2   /* real float32 model                   */
#define EDT_F64    3   /* real float64 model                   */

typedef struct edt_ctx edt_ctx;   /* opaque; owned by the library */

/* Problem description.  Lengths in metres, velocities in m/s, frequencies in Hz.
 * Arrays are read during edt_create only and may be freed afterwards. */
typedef struct {
  int nx;                       /* lateral samples (power of two, 4..1024)               */
  double dx;                    /* lateral spacing (> 0)                                 */
  int nz;                       /* depth unknowns (1..512; the mixed path: 1..256)       */
  double dz;                    /* depth spacing (> 0)                                   */
  double z0;                    /* depth of the top of the first depth cell (>= 0)       */
  int nfreq;                    /* number of frequencies (1..32767)                      */
  const double* freq_hz;        /* [nfreq], > 0                                          */
  double eps;                   /* imaginary part of the complex frequency (1/s, >= 0)    */
  int nlayer;                   /* layers of the reference c0(z) (1..4096)               */
  const double* layer_top_m;    /* [nlayer], layer_top_m[0] == 0, strictly increasing    */
  const double* layer_vel_mps;  /* [nlayer], > 0; the last layer is a half-space         */
  int precision;                /* EDT_FP64 or EDT_MIXED                                 */
  int passes;                   /* mixed: 1 = BF16 Gram, 3 = split BF16x3 Gram           */
  int refine;                   /* mixed: refinement steps (0..8, default 1)             */
  double alpha;                 /* damping: lam = alpha * trace(Gram) (>= 0)             */
  double cutoff;                /* evanescent cut factor; <= 0 keeps every row           */
  int fold;                     /* 1: merge the identical reciprocal rows (p,q),(-q,-p)
                                   into one row of weight 2 (same normal equations);
                                   0: keep every row as the paper writes them           */
  int chol_df;                  /* mixed path only: the damped Cholesky factorisation and
                                   solves in double-float (FP32 hi/lo pairs, ~48-bit,
                                   error-free products and sums) on the FP32 pipes with
                                   FP64 pivots (1, and 0 = automatic, the default), or
                                   native FP64 throughout (2), or double-float with the
                                   trailing updates on the tensor cores (3: each panel
                                   value cut into eight 7-bit BF16 slices, every level of
                                   slice products summed exactly in FP32 tensor memory;
                                   the same factor to FP64 class, slower as built); the
                                   FP64 path always factors in native FP64              */
  int freq_chunk;               /* frequency planes per chunk of the data transform and
                                   the forward model (the spectrum buffer holds one
                                   chunk); 0 = automatic: as many planes as fit in
                                   256 MB.  Smaller chunks trade speed for workspace.   */
  int geometry;                 /* EDT_GEOM_LINE (0) or EDT_GEOM_WINDOW (1)              */
  int ny;                       /* window geometry: midpoints along y (1, or == nx with
                                   nx <= 128); nx in 32..512 (ny == 1) or 32..128       */
  double dy;                    /* window geometry: y spacing (> 0)                      */
  int wx, wy;                   /* window geometry: half-offsets per axis (powers of
                                   two, 1..16; wx <= nx, wy <= ny); the half-offset
                                   spacing equals the midpoint spacing                  */
  /* Solver variants of Section "Numerical Examples" (line geometry, EDT_FP64 only; else
   * EDT_EUNSUPPORTED):                                                                  */
  int solver;                   /* EDT_SOLVE_DAMPED (0, default) or EDT_SOLVE_TSVD (1):
                                   x = V S~^-1 U^T dhat, 1/s_j kept for s_j >= sigma, from
                                   the eigenpairs of the FP64 normal matrix; nz <= 96    */
  double tsvd_tol;              /* sigma: > 0 absolute, < 0 relative (|tol| * s_max),
                                   0: every positive singular value                      */
  double kz_disk;               /* > 0: restrict the unknowns of k_m to the vertical
                                   wavenumbers k_z = 2 pi l / (nz dz) (orthonormal real
                                   depth basis: constant, cos/sin of 2 pi l j / nz, and
                                   (-1)^j) with k_m^2 + k_z^2 <= (kz_disk omega_max /
                                   c_min)^2, c_min the slowest layer; 0: off             */
  int gram_seg_rows;            /* mixed path: most complex rows one FP32 tensor-memory
                                   accumulation of the Gram covers before it is flushed
                                   to a partial tile that is summed in FP64 (rounded up
                                   to a multiple of 32; shorter runs lose less to FP32
                                   accumulation); 0 = automatic                          */
  int resid;                    /* mixed: arithmetic of the refinement residual
                                   r = Ahat^T (dhat - Ahat x): 1 = FP32 rows and products,
                                   FP64 sums across warps and blocks; 2 = FP64-accurate:
                                   rows from a double-float table (FP32 hi + lo of the
                                   FP64 depth march), the accumulation Ahat^T u by exact
                                   products and compensated sums (line geometry only);
                                   0 = automatic: 2 on the line geometry when
                                   alpha < 1e-3, else 1                                 */
  int sub_begin, sub_end;       /* line geometry: plan and solve only the subproblems
                                   m in [sub_begin, sub_end) (0 <= sub_begin <= sub_end
                                   <= nx/2 + 1); the others get no rows and Vhat = 0.
                                   0, 0 = every subproblem.  The partitioned solve gives
                                   each rank such a range (see edt_import_rhs).         */
} edt_config;

#define EDT_SOLVE_DAMPED 0
#define EDT_SOLVE_TSVD   1

/* Host-side statistics of a context; the device-side fields are refreshed by
 * edt_get_stats, which synchronises the context's last stream. */
typedef struct {
  int n_sub;                    /* subproblems solved: nx/2 + 1 (line geometry) or the
                                   number of pairs {k_m, -k_m} (window geometry)        */
  long long rows_total;         /* complex rows over all subproblems after the cut       */
  long long rows_solved;        /* rows actually processed (after folding)               */
  int rows_min, rows_max;       /* per-subproblem complex rows after the cut             */
  size_t workspace_bytes;       /* device workspace required                             */
  double gram_flop;             /* algorithmic Gram flops per invert (2 * rows_solved'
                                   * 2 * nz * (nz + 2), real rows, full square)          */
  int n_notpd;                  /* subproblems whose factorisation failed (last invert)  */
  int n_nonfinite;              /* subproblems with a non-finite solution (last invert)  */
  int last_status;              /* status of the last device call                        */
  int launches_per_invert;      /* CUDA kernels one edt_invert launches                  */
  long long gram_rows_padded;   /* complex rows the tensor-core Gram processes per call,
                                   each CTA segment padded to a multiple of 32           */
  int freq_chunk;               /* frequency planes the data transform and the
                                   right-hand-side gather process per chunk (the
                                   spectrum buffer holds one chunk, about 32 MB)         */
  int launches_per_grad;        /* CUDA kernels one edt_misfit_grad launches (0 where it
                                   is unsupported)                                       */
  int gram_timeouts;            /* 1 if a bounded wait of the tensor-core Gram expired in
                                   the last edt_invert / edt_gram (its result is then
                                   invalid and last_status is EDT_ETIMEOUT), else 0      */
} edt_stats;

/* Launch shapes the autotuner chooses among (candidates in brackets; all give the same
 * results up to FP32 summation order). */
typedef struct {
  int band_budget_mb;           /* line geometry, mixed: bytes of band spectra per transform
                                   chunk, in MB [16, 32, 48, 96]; default 48                */
  int band_cols;                /* line geometry, mixed: band columns per column-FFT block
                                   [4, 8, 16]; default 8                                    */
  int refine_shape;             /* mixed: refinement CTA shape, 0 = 4 warps x 32 rows,
                                   1 = 8 x 32, 2 = 4 x 64, 3 = 8 x 16; default 0           */
  int window_ztile;             /* window geometry: depths per kernel-row cluster [2, 4, 8];
                                   default 4                                                */
  int overlap;                  /* 1: depth march (and window kernel rows) on the internal
                                   stream, concurrent with the data transform; 0: in
                                   sequence on the caller's stream [0, 1]; default 1        */
  double invert_ms;             /* edt_invert time with these shapes when the autotuner
                                   chose them (0 if never tuned)                           */
} edt_tuning;

/* Create a context for `cfg` and report the device workspace it needs.
 * Returns EDT_OK, EDT_EINVAL or EDT_EUNSUPPORTED.  *out is NULL on failure. */
int edt_create(edt_ctx** out, const edt_config* cfg, size_t* workspace_bytes);

/* Attach a caller-owned device workspace of at least the reported size (256-byte
 * aligned) and upload the context's constant tables into it (synchronous copies on the
 * legacy stream).  The workspace must stay valid until edt_destroy or the next call. */
int edt_set_workspace(edt_ctx* ctx, void* ws_dev, size_t bytes);

/* Invert data D -> model V (the whole method above).  D_dtype is EDT_C64 or EDT_C128,
 * V_dtype EDT_F32 or EDT_F64.  Per-subproblem failures (EDT_ENOTPD) zero that
 * subproblem and are counted in edt_get_stats; they do not fail the call. */
int edt_invert(edt_ctx* ctx, const void* D_dev, int D_dtype, void* V_dev, int V_dtype,
               void* stream);

/* CUDA-graph mode: with on != 0, edt_invert captures all of its stages into one CUDA graph
 * on the first call and replays it while the data and model pointers, their dtypes and the
 * stream stay the same (a change re-captures).  Requires a non-default stream; calls on the
 * legacy default stream, and calls made while profiling is on, run uncaptured. */
int edt_set_graph(edt_ctx* ctx, int on);

/* Autotuner: for each tunable launch shape in turn, time `reps` (>= 1) edt_invert calls on
 * the caller's data with every candidate (the others at their current best) and keep the
 * fastest (coordinate descent, CUDA events on `stream`; one warm-up call, then the reps back
 * to back, their mean time per call).  The tuned
 * shapes stay with the context; V_dev receives the last inversion.  Synchronises `stream`.
 * Must not run while the stream is being captured. */
int edt_autotune(edt_ctx* ctx, const void* D_dev, int D_dtype, void* V_dev, int V_dtype,
                 void* stream, int reps);
/* The current launch shapes; setting them validates every field (EDT_EINVAL). */
int edt_get_tuning(const edt_ctx* ctx, edt_tuning* out);
int edt_set_tuning(edt_ctx* ctx, const edt_tuning* in);

/* edt_invert from host buffers: copies D to the device, inverts, copies V back, all on
 * `stream` (asynchronous; the host buffers must stay valid until the stream syncs).
 * Uses the staging areas inside the workspace.  With the host pipeline on (below) the copy
 * of D runs on an internal stream into one of two staging buffers, so consecutive calls
 * overlap one call's input copy with the previous call's stages. */
int edt_invert_host(edt_ctx* ctx, const void* D_host, int D_dtype, void* V_host,
                    int V_dtype, void* stream);

/* on = 1: edt_invert_host copies D_host on the context's internal copy stream, waiting only
 * for the call before last (which used the same staging buffer), not for earlier work on
 * `stream`; the inversion then waits for the copy on `stream`, and V is copied back on
 * `stream`.  D_host must therefore be complete when the call is made (written by the host,
 * not by device work still pending on `stream`).  on = 0 (default): every step on
 * `stream` in order. */
int edt_set_host_pipeline(edt_ctx* ctx, int on);

/* Born forward model V -> D in the same discrete model (eq. Born with omega~^2):
 * D(is, ir) = omega~^2 dx dz sum_x sum_j G(x_ir - x, z_j) V(x, z_j) G(x - x_is, z_j),
 * evaluated spectrally.  Precision follows cfg.precision (FP32 for EDT_MIXED). */
int edt_forward(edt_ctx* ctx, const void* V_dev, int V_dtype, void* D_dev, int D_dtype,
                void* stream);

/* Adjoint Born operator (Section "Two dimensions", eq. Born and its decoupled form eq. DMV):
 * V = F^T D, the adjoint of edt_forward's map V -> D for the inner products
 * <D1, D2> = Re sum conj(D1) D2 and <V1, V2> = sum V1 V2, i.e. with D2 = T(D) / nx^2 (T the
 * data transform of the header, whose adjoint inverse is T / nx^2),
 *   Vbar_hat(k_m, z_j) = sum_f sum_p conj(s_f g(k_p, z_j) g(k_{p-m}, z_j)) D2_f(p, p - m),
 *   V(x_i, z_j) = Re sum_m Vbar_hat(k_m, z_j) exp(+i k_m x_i),   s_f = omega~_f^2 dz / dx.
 * D_dev: complex [nfreq][nx][nx] (EDT_C64 or EDT_C128), caller-owned; V_dev: real [nx][nz]
 * (EDT_F32 or EDT_F64), overwritten.  EDT_FP64: FP64 transform and contraction; EDT_MIXED:
 * FP32 transform and table, FP32 products with FP64 sums across frequencies (needs nx >= 64
 * and at most 64 layers, as edt_misfit_grad).  Line geometry only (else EDT_EUNSUPPORTED).
 * Asynchronous on `stream`; uses the workspace (not the factors of the last edt_invert). */
int edt_adjoint(edt_ctx* ctx, const void* D_dev, int D_dtype, void* V_dev, int V_dtype, void* stream);

/* Misfit of a model against data and its gradients (line geometry, EDT_MIXED; FP32
 * arithmetic with FP64 accumulation across frequencies):
 *   J = || F(c0) V - D ||^2 = sum_f sum_is sum_ir |(F V - D)(f, is, ir)|^2,
 * F the Born operator of edt_forward with every row (no evanescent cut), and
 *   gV[x][z]  = dJ/dV(x, z)  (adjoint Born: 2 F^T (F V - D)),
 *   gc[l]     = dJ/dc_l, the derivative with respect to the velocity of layer l of the
 *               reference, through the depth march of g (reverse-mode differentiation of
 *               the reflectivity recursion, recomputed, not stored).
 * V_dev: [nx][nz] (EDT_F32 or EDT_F64), D_dev: [nfreq][nx][nx] (EDT_C64 or EDT_C128);
 * outputs are device pointers: J_dev one double, gV_dev [nx][nz] of V_dtype, gc_dev
 * double[nlayer].  Requires nx >= 64 and nlayer <= 64 (else EDT_EUNSUPPORTED).  The
 * evaluation is in the (p, q) spectral domain, where the data transform is nx times a
 * unitary map per axis, so J = (1/nx^2) sum |D2-domain residual|^2 exactly. */
int edt_misfit_grad(edt_ctx* ctx, const void* V_dev, int V_dtype, const void* D_dev,
                    int D_dtype, double* J_dev, void* gV_dev, double* gc_dev, void* stream);

/* Adjoint of the inversion (line geometry, EDT_MIXED).  edt_invert maps D linearly to V
 * (the normal matrices and the damping depend on the reference only), V = S D; this call
 * computes Dbar = S^T Vbar for the real inner products <V1, V2> = sum V1 V2 and
 * <D1, D2> = Re sum conj(D1) D2 -- the gradient of any loss L(V) with respect to D, given
 * Vbar = dL/dV.  It reuses the factors of the last successful edt_invert on this context
 * (EDT_EINVAL if there is none, or if edt_gram, edt_set_workspace or edt_set_reference ran
 * since): xbar from the lateral DFT of Vbar, bbar = (G + lam I)^-1 xbar with the same
 * refinement steps as the forward solve (the transpose of the forward's own linear map),
 * and for every kept row the split and the data transform reversed.  Vbar_dev: [nx][nz]
 * (EDT_F32/EDT_F64); Dbar_dev: [nfreq][nx][nx] (EDT_C64/EDT_C128), fully written.  The
 * solve's scratch (b, x, the residual) is overwritten; the factors, the right-hand sides and
 * edt_get_vhat's result are not, so the call may be repeated for other Vbar. */
int edt_invert_adjoint(edt_ctx* ctx, const void* Vbar_dev, int Vbar_dtype, void* Dbar_dev,
                       int Dbar_dtype, void* stream);

/* The inversion's vector-Jacobian products with respect to the data and to the reference
 * (line geometry, EDT_MIXED), for Vbar = dL/dV after a successful edt_invert (same
 * preconditions as edt_invert_adjoint):
 *   Dbar_dev (may be null): as edt_invert_adjoint;
 *   gc_dev   (may be null): double[nlayer], gc[l] = dL/dc_l through the damped solve.  Per
 *     midpoint index m the solution of (Ahat^T Ahat + lam I) x = Ahat^T dhat, lam = alpha
 *     tr(Ahat^T Ahat), depends on the layer velocities through the kernel rows (eq. M, the
 *     depth march of g) and through lam; with mu = (Ahat^T Ahat + lam I)^-1 xbar,
 *       dL/dc_l = sum_m [ mu^T dAhat^T (dhat - Ahat x) - mu^T Ahat^T dAhat x - dlam mu^T x ],
 *     dlam = 2 alpha <Ahat, dAhat>, the rows' derivatives taken by reverse-mode
 *     differentiation of the depth march (as edt_misfit_grad).  The set of kept rows is held
 *     fixed (the evanescent cut does not move with the velocities).  Needs nx >= 64,
 *     nlayer <= 64 and nz <= 512 (else EDT_EUNSUPPORTED).
 * At least one output must be given (else EDT_EINVAL).  The factors, the tables and the
 * right-hand sides of the forward call are kept, so the call may be repeated for other Vbar;
 * edt_get_vhat still returns the forward's Vhat.  Asynchronous on `stream`. */
int edt_invert_vjp(edt_ctx* ctx, const void* Vbar_dev, int Vbar_dtype, void* Dbar_dev, int Dbar_dtype,
                   double* gc_dev, void* stream);

/* Replace the layer velocities of the reference (same layer tops); every later call uses
 * them (the depth march runs in every call).  With cutoff > 0 the row plan depends on the
 * slowest velocity, so that minimum must stay the same (else EDT_EINVAL: create a new
 * context).  The host array is copied before the call returns. */
int edt_set_reference(edt_ctx* ctx, const double* layer_vel_mps, void* stream);

/* Reference Green's function table g(k_n, z_j; omega~_f), n = 0..nx/2, as complex128
 * [nfreq][nx/2+1][nz] (computed in FP64 by the depth march). */
int edt_green(edt_ctx* ctx, void* g_dev, void* stream);

/* ---- partitioned solve (the subproblems are independent: Section "Two dimensions", the
 * decoupling of eqs. DMV and M; Discussion) -----------------------------------------------
 * A job sharded over ranks runs: on each rank, a context for its frequencies (a contiguous
 * range of the job's frequency list, cfg.freq_hz restricted to it) produces the split
 * right-hand sides of every subproblem (edt_export_rhs); the rows of each subproblem go to the
 * rank owning it (an all-to-all; row blocks are contiguous per destination because the rows
 * are ordered by subproblem, then frequency); each rank's context restricted to its
 * subproblems (sub_begin, sub_end; all frequencies) places the received blocks
 * (edt_import_rhs, one call per source) and solves (edt_solve_imported); the Vhat of all ranks
 * are summed (disjoint supports) and edt_inverse_vhat returns V.  The result equals
 * edt_invert's up to the summation order of the tensor-core Gram (FP64 path: bitwise the
 * same arithmetic). */

/* Offsets of each subproblem's solved rows (after the reciprocal folding) in the context's row
 * order: off[nx/2 + 2].  Host only.  Returns nx/2 + 2 or EDT_EINVAL. */
int edt_row_offsets(const edt_ctx* ctx, long long* off);

/* Data transform and split right-hand sides of D (this context's frequencies, on the device)
 * copied out to rhs_dev: off[nx/2 + 1] rows (edt_row_offsets) in the context's order
 * (subproblem, then frequency, then receiver index), two complex values (d_+, d_-) each,
 * rotated by the unit phase conj(s_f)/|s_f| (the kernel rows carry |s_f|): complex64 on the
 * mixed path, complex128 on the FP64 path.  rhs_dev is the caller's.  Line geometry.
 * Asynchronous on `stream`.  Returns EDT_OK, EDT_EINVAL (null pointer, bad dtype),
 * EDT_ENOMEM_WS (no workspace), EDT_EUNSUPPORTED (window geometry, solver variants). */
int edt_export_rhs(edt_ctx* ctx, const void* D_dev, int D_dtype, void* rhs_dev, void* stream);

/* Place the rows of frequencies [f_begin, f_end) of every subproblem of this context into the
 * workspace: block_dev holds nrows rows, ordered by subproblem, then frequency, as exported by
 * a context holding exactly those frequencies (same grid, layers and cut; its rows of the
 * subproblems outside this context's range are left out).  nrows must equal this context's row
 * count at those frequencies, else EDT_EINVAL (block_dev may be null when it is 0).  Every
 * frequency must be imported before edt_solve_imported.  Asynchronous on `stream`. */
int edt_import_rhs(edt_ctx* ctx, const void* block_dev, long long nrows, int f_begin, int f_end,
                   void* stream);

/* The stages of edt_invert after the data transform (depth march, Gram, Cholesky, refinement)
 * on the imported right-hand sides; writes Vhat(k_m, z_j) = x_+ + i x_- as complex128
 * [nx/2 + 1][nz] (zero outside the context's subproblem range and for failed subproblems).
 * Asynchronous on `stream`; edt_get_stats reports as after edt_invert. */
int edt_solve_imported(edt_ctx* ctx, void* vhat_dev, void* stream);

/* V from Vhat (complex128 [nx/2 + 1][nz]): the completion Vhat(-k_m) = conj Vhat(k_m)
 * (eq. VSym) and the inverse lateral DFT, as edt_invert's last stage.  Line geometry. */
int edt_inverse_vhat(edt_ctx* ctx, const void* vhat_dev, void* V_dev, int V_dtype, void* stream);

/* Copy the Cholesky factors of the last edt_invert on this context, G + lam I = L L^T per
 * subproblem, as double [n_sub][nz][nz] into caller device memory: the lower triangle and
 * the diagonal hold L (row-major), the strict upper triangle is unspecified.  EDT_EINVAL if
 * no factorisation is held (no edt_invert since the workspace, reference or a stage call
 * changed it, or a solver variant without a Cholesky ran). */
int edt_get_factor(edt_ctx* ctx, void* L_dev, void* stream);

/* Copy Vhat(k_m, z_j) of the last edt_invert on this context, m = 0..nx/2, as
 * complex128 [nx/2+1][nz], into caller device memory. */
int edt_get_vhat(edt_ctx* ctx, void* vhat_dev, void* stream);

/* Stages up to the normal matrices only (depth march, data transform, split right-hand
 * sides, Gram): writes G = Ahat^T W Ahat as double [nx/2+1][nz][nz], b = Ahat^T W dhat as
 * double [nx/2+1][nz][2] (columns d_+, d_-) and trace(G) as double [nx/2+1], where W holds
 * the row weights (2 for merged reciprocal rows).  For EDT_MIXED these are the tensor-core
 * results (BF16 operands, FP32 accumulation) and the FP64 trace used for the damping. */
int edt_gram(edt_ctx* ctx, const void* D_dev, int D_dtype, void* G_dev, void* b_dev,
             void* trace_dev, void* stream);

/* Allocation-free depth march (no counterpart in the paper: a library service).
 * For callers that may not allocate device memory at all, e.g. a component running
 * inside a host application that owns the device allocator, or one that is handed only
 * its input and output buffers.  It computes the same table as edt_green,
 * g(k_n, z_j; omega~_f) as complex128 [nfreq][nx/2+1][nz] into the caller's g_dev, from
 * host arrays, without a context and without any device allocation: all scratch (the
 * layer stack, per-frequency constants and the recursion coefficients) lives in one
 * fixed 8 MiB device array inside the library, which every GPU that loads the library
 * keeps until the process exits.  Frequencies are processed in chunks that fit it.
 * Limits: nx a power of two >= 2; one frequency's coefficients, (nx/2+1) * nlayer * 112
 * bytes, must fit in the 8 MiB (else EDT_EUNSUPPORTED).  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device current and keeps
 * it for the life of the process: the call is not valid on a device after a
 * cudaDeviceReset of it.  The call copies its host arrays through pageable memory, so it
 * must never run while `stream` is being captured into a CUDA graph (nor, on the legacy
 * stream, while any thread captures in global mode): it checks and returns EDT_EINVAL
 * then.  Every call reuses the same array, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race on it; each call fully writes the scratch it reads,
 * so nothing carries over between calls.  Host arrays may be freed when the call returns;
 * the computation is asynchronous on `stream`.  Returns EDT_OK, EDT_EINVAL,
 * EDT_EUNSUPPORTED or EDT_ECUDA. */
int edt_green_noalloc(int nx, double dx, int nz, double dz, double z0, int nfreq,
                      const double* freq_hz, double eps, int nlayer, const double* layer_top_m,
                      const double* layer_vel_mps, void* g_dev, void* stream);

/* Vertical-wavenumber disk (kz_disk > 0): p[m] = the depth-basis columns kept for midpoint index
 * m = 0..nx/2 (host only).  Returns nx/2 + 1, or EDT_EINVAL without the disk. */
int edt_kz_disk_columns(const edt_ctx* ctx, int* p);

/* Measured FP64 and FP32 fused multiply-add rates of the current device, in TFLOP/s (2 flops
 * per multiply-add; the best of three timed launches of independent multiply-add chains over
 * every SM).  A utility for stating rooflines (the library's double-float kernels trade FP64
 * work for FP32 work); no counterpart in the paper.  Synchronous; allocates and frees a small
 * device buffer, so not for use during stream capture.  Returns EDT_OK or EDT_ECUDA. */
int edt_measure_fma_rates(double* fp64_tflops, double* fp32_tflops);

/* Per-subproblem complex row counts after the cut (before folding): counts[nx/2+1]. */
int edt_row_counts(const edt_ctx* ctx, long long* counts);

/* Fill *out; synchronises the stream of the last device call on this context.  A device
 * wait that expired in the last edt_invert (every wait of the tensor-core Gram is bounded,
 * about 2 s) shows here as gram_timeouts = 1 and last_status = EDT_ETIMEOUT: edt_invert
 * itself returns before the device work ends, so this is where the failure surfaces. */
int edt_get_stats(edt_ctx* ctx, edt_stats* out);

/* Test hook for the failure path of the bounded device waits (failure detection exercised
 * without a GPU fault; not for production use).  wait_cycles > 0 replaces the
 * ~2 s budget of every bounded wait of the tensor-core Gram by that many SM clock cycles;
 * stall = 1 (requires wait_cycles > 0) makes the Gram's MMA issuer wait on an mbarrier that
 * nothing completes, so the wait runs out, the kernel raises its flag, releases the
 * producers through its abort flag, drains its MMAs and copies, frees its tensor memory
 * and returns; edt_get_stats then reports EDT_ETIMEOUT.  stall = 0, wait_cycles = 0 restore
 * normal operation; the context stays usable throughout.  Host-only; returns EDT_OK or
 * EDT_EINVAL. */
int edt_set_wait_test(edt_ctx* ctx, long long wait_cycles, int stall);

/* Per-stage device timing.  With profiling on, every edt_invert (up to 256 calls between
 * reads) records CUDA events at the beginning and end of each stage on the stream the stage
 * runs on (the depth march overlaps the data transform, so the stage times may add up to
 * more than the call); edt_read_profile synchronises and returns the summed milliseconds
 * per stage since the last reset (names[i] static strings), then resets.
 * Returns the number of stages written (<= max_stages), or a negative code. */
int edt_set_profiling(edt_ctx* ctx, int on);
int edt_read_profile(edt_ctx* ctx, double* ms, const char** names, int max_stages,
                     int* n_calls);

/* ---------------------------------------------------------------- streaming 1D solves
 * A stream of independent 1D depth subproblems.  Each request is the split system of one
 * midpoint wavenumber (eqs. DMV, M and Split of Section "Two dimensions") standing on its own,
 * with its own layered reference, depth grid, frequencies and rows.  Request r solves, for
 * real x_+ and x_- (nz unknowns each),
 *     min ||Ahat x_+- - dhat_+-||^2 + lam ||x_+-||^2,     lam = alpha trace(Ahat^T Ahat),
 * Ahat = [Re a; Im a], dhat_+- = [Re d_+-; Im d_+-], a_i(z_j) = s_f g(kval[p], z_j) g(kval[q], z_j)
 * for row i = (f, p, q), s_f = omega~_f^2 dz / dx, omega~_f = 2 pi freq_hz[f] + i eps,
 * z_j = z0 + (j + 1/2) dz, g the Green's function of the layered reference (the depth march of
 * edt_green); the result is Vhat(z_j) = x_+(z_j) + i x_-(z_j).  Arithmetic follows EDT_MIXED:
 * FP32 Green's table (FP64 vertical wavenumbers), split BF16 tensor-core Gram with FP32
 * accumulation, double-float Cholesky (FP64-class, on the FP32 pipes), one refinement step
 * (FP32 residual accumulated in FP64, FP32 correction solve).
 *
 * Requests are admitted by device memory: the caller's workspace is split into two arenas, a
 * submitted list is cut in order into batches whose summed edt_stream_request_bytes fit one
 * arena (and at most max_batch requests), and each batch runs as eight stages whose launches
 * cover all its requests (the Cholesky as a panel-row and a tile-update launch per 32-column
 * step, so that a large factorisation spreads over many SMs).  The two arenas have a CUDA stream each, so one batch's launches
 * overlap the next batch's copies and launches while the host packs the batch after into
 * pinned staging.  All state stays on the device until the results of a batch are copied
 * back. */
typedef struct {
  int nz;                       /* unknowns (depths), 1..512                                */
  double dz, z0;                /* depth step > 0 (m) and offset: z_j = z0 + (j + 1/2) dz     */
  double eps;                   /* omega~ = omega + i eps (1/s), >= 0                        */
  double alpha;                 /* damping factor, >= 0                                      */
  double dx;                    /* lateral spacing (m) in s_f, > 0                           */
  int nlayer;                   /* 1..64 layers; top of layer 0 at 0, tops increasing;       */
  const double* layer_top_m;    /*   the last layer is a half-space                          */
  const double* layer_vel_mps;  /*   velocities > 0                                          */
  int nfreq;                    /* >= 1 */
  const double* freq_hz;        /* [nfreq], > 0                                              */
  int nk;                       /* >= 1 */
  const double* kval;           /* [nk] lateral wavenumbers |k| (rad/m), >= 0                */
  int nrow;                     /* >= 0 rows                                                 */
  const int* rows;              /* [nrow][3] (f, p, q): f < nfreq, p, q < nk                 */
  const float* data;            /* [nrow][4] complex64 pairs: d_+ (re, im), d_- (re, im)     */
} edt_sub1d;

typedef struct edt_stream edt_stream;   /* opaque; owned by the library */

typedef struct {
  long long requests;           /* requests solved since creation                            */
  long long batches;            /* batches launched                                          */
  double compute_ms;            /* summed device time of the batches' launches (CUDA events,
                                   host-device copies excluded)                             */
  double busy_ms;               /* since the last edt_stream_epoch: union over the delivered
                                   batches of the intervals in which their launches ran
                                   (overlapping batches counted once)                       */
  long long bytes_in, bytes_out;/* host-to-device and device-to-host bytes copied            */
  long long launches;           /* CUDA kernels launched (all batches)                       */
  int launches_per_batch;       /* most kernels one batch launched: 7 + 2 per 32-column step of
                                   its blocked Cholesky, at most 39                          */
  size_t arena_bytes;           /* device bytes of one arena (half the workspace)            */
  int max_batch;
} edt_stream_stats;

/* Device bytes a request occupies in an arena (>= 0), or EDT_EINVAL for an invalid one. */
long long edt_stream_request_bytes(const edt_sub1d* sub);

/* Admission plan (host only): requests 0..n-1, of request_bytes[i] device bytes, are cut in
 * order into batches of at most max_batch requests whose summed bytes plus the fixed per-batch
 * overhead fit arena_bytes; batch_of[i] receives the batch index of request i.  Returns the
 * number of batches, EDT_ENOMEM_WS if a request alone does not fit, or EDT_EINVAL. */
int edt_stream_plan(int n, const long long* request_bytes, long long arena_bytes, int max_batch,
                    int* batch_of);

/* Create a stream solver on the current device.  max_batch: 1..4096 requests per batch.
 * stream: NULL, or a CUDA stream (cudaStream_t) whose work submitted before each
 * edt_stream_submit the batches of that call wait for (they run on the solver's own two
 * streams).  *workspace_min receives the smallest workspace that admits the largest possible
 * request (nz = 512, nrow = 4096) in each arena. */
int edt_stream_create(edt_stream** out, int max_batch, void* stream, size_t* workspace_min);

/* Hand the solver its device workspace (caller-owned, >= 256-byte aligned, kept until
 * edt_stream_destroy).  Waits for any batch in flight.  EDT_ENOMEM_WS if too small. */
int edt_stream_set_workspace(edt_stream* s, void* ws_dev, size_t bytes);

/* Submit n requests.  Their host arrays may be freed when the call returns (they are packed
 * into pinned staging).  Results arrive in vhat_host (complex128 interleaved, the requests'
 * nz values one after another, sum of nz entries) and status_host (EDT_OK, EDT_ENOTPD,
 * EDT_ENONFINITE or EDT_ETIMEOUT per request); both must stay valid until edt_stream_wait on
 * *ticket returns.  A request larger than an arena fails the call with EDT_ENOMEM_WS before
 * anything is launched.  Returns EDT_OK, EDT_EINVAL, EDT_ENOMEM_WS or EDT_ECUDA. */
int edt_stream_submit(edt_stream* s, int n, const edt_sub1d* subs, double* vhat_host,
                      int* status_host, long long* ticket);

/* Block until every batch of the ticket is done and its results are in the caller's arrays.
 * done_ms (may be NULL) receives the completion time of its last batch in milliseconds after
 * the last edt_stream_epoch (CUDA events; -1 if no epoch was set). */
int edt_stream_wait(edt_stream* s, long long ticket, double* done_ms);

/* Non-blocking: *done = 1 if every batch of the ticket has completed on the device. */
int edt_stream_query(edt_stream* s, long long ticket, int* done);

/* Synchronise the stream and record the time origin of edt_stream_wait's done_ms. */
int edt_stream_epoch(edt_stream* s);

int edt_stream_get_stats(const edt_stream* s, edt_stream_stats* out);

/* Per-stage device timing: with profiling on, batches run one at a time (no overlap between
 * the two arenas' streams) and CUDA events are recorded between the eight stages of every batch; edt_stream_read_profile delivers the batches in flight, returns the
 * summed milliseconds per launch (names[i] static strings) since the last read, the number of
 * batches they cover in *n_batches, and resets.  Returns the number of entries written. */
int edt_stream_set_profiling(edt_stream* s, int on);
/* Test hook for the streaming Gram's bounded waits, as edt_set_wait_test: batches submitted
 * while stall = 1 take the timeout path and report EDT_ETIMEOUT for each of their requests;
 * later batches (stall = 0) run normally. */
int edt_stream_set_wait_test(edt_stream* s, long long wait_cycles, int stall);
int edt_stream_read_profile(edt_stream* s, double* ms, const char** names, int max_kernels,
                            long long* n_batches);

/* Wait for the batches in flight and release the solver (not the caller's workspace). */
void edt_stream_destroy(edt_stream* s);

/* Message for a status code; message of the last CUDA error seen by the library. */
const char* edt_strerror(int code);
const char* edt_last_cuda_error(void);

/* Release the context (does not free the caller's workspace). */
void edt_destroy(edt_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* EDT_H */
