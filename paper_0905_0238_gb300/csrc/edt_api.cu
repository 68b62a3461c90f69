// C ABI: context creation, host-side planning (row lists, tables, workspace layout) and
// the orchestration of the device stages.  See include/edt.h for the contract.
#include "edt_internal.h"
#include "cplx.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

namespace edt {

namespace {

thread_local std::string g_last_cuda;

int cuda_fail(cudaError_t e) {
  g_last_cuda = cudaGetErrorString(e);
  return EDT_ECUDA;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

struct Region { size_t off = 0, bytes = 0; };

}  // namespace

int record_cuda_error(cudaError_t e) { return cuda_fail(e); }

// Most complex rows one FP32 tensor-memory accumulation of the Gram covers (a segment);
// longer runs are split into several segments, each flushed to its own partial tile.
// Damping below which the automatic residual mode switches to double-float: with FP32
// products the residual's rounding reaches x amplified by up to 1 / lam, which at alpha
// ~1e-5 approaches the 1e-5 parity bar.
constexpr double kResidDfAlpha = 1e-3;

static long long gram_seg_cap(const edt_config& g) {
  if (g.gram_seg_rows > 0) return (long long)(g.gram_seg_rows + TC_KC - 1) / TC_KC * TC_KC;
  return 1LL << 40;
}

}  // namespace edt

using namespace edt;

struct edt_ctx {
  edt_config cfg{};
  std::vector<double> freq, tops, vel;
  // plan
  int N = 0, nk = 0, nz = 0, nf = 0, nsub = 0, nlayer = 0;
  std::vector<FreqConst> fc;
  std::vector<int> z_layer;
  std::vector<double> z_off;
  std::vector<float> z_off32;      // [nz][4]
  std::vector<float> fc32;         // [nf] sqrt|s_f|
  std::vector<uint32_t> rows;
  std::vector<long long> row_off;
  std::vector<long long> row_off_mf;   // [nsub][nf + 1]
  int fchunk = 1;
  // window geometry
  bool win = false;
  int ny = 1, wx = 1, wy = 1, W = 1, nxy = 0;
  std::vector<double> kval;            // [nk] |k| of each table row
  std::vector<int> pair_m;             // [nsub] midpoint index of each pair
  std::vector<int> fj_off;             // [nf * W + 1]
  std::vector<int2> fj_ent;            // [rows] (midpoint index, row) grouped by (f, j)
  std::vector<double2> cf;             // [nf] omega~^2 dx dy dz
  std::vector<int> jact, jmap, nact;   // active offset wavenumbers per frequency
  long long rows_max_sub = 0;
  // band-limited transform of the mixed path
  bool band_mode = false;
  bool have_factor = false;            // the workspace holds the factors of the last edt_invert
  bool resid_df = false;               // double-float refinement residual (line geometry, mixed)
  std::vector<BandInfo> band;
  std::vector<int2> bcol;
  std::vector<long long> cpre;
  std::vector<BandChunk> bchunks;
  size_t band_ymax = 0, band_xmax = 0;   // complex elements of the largest chunk's Y and Xc
  int band_maxplanes = 0;
  // launch shapes (autotuned) and the workspace maxima over their candidates
  int band_budget_mb = 48, tune_bc = 8, tune_rf = 0, tune_zc = 4, tune_ov = 1;
  size_t ws_band_elems = 0, ws_bcol = 0, ws_cpre = 0;
  double tuned_ms = 0.0;
  std::vector<long long> counts_cut;
  std::vector<double2> tw64;
  std::vector<float2> tw32;
  // tensor-core Gram schedule
  std::vector<int> seg_m, cta_seg0, m_slot0;
  // solver variants: kept vertical-wavenumber columns per subproblem and the depth basis
  bool variant = false;
  std::vector<int> kz_p;
  std::vector<long long> kz_goff, kz_voff;
  std::vector<double> kz_P;
  std::vector<long long> seg_row0, seg_nrow;
  int ncta_gram = 0, nslot = 0;
  // reference gradient through the solve: the rows reading each table row (f, |n|)
  std::vector<int2> tref;
  std::vector<long long> tref_off;
  // workspace
  size_t ws_bytes = 0;
  void* ws = nullptr;
  Region r_fc, r_ltop, r_lvel, r_zl, r_zo, r_rows, r_roff, r_roffmf, r_band, r_bcol, r_cpre, r_kval, r_pairm, r_fjoff, r_fjent, r_jact, r_jmap, r_Gs, r_U, r_Dw, r_A32, r_tw64, r_tw32, r_segm, r_segr0,
      r_segn, r_ctas, r_mslot, r_zo32, r_fc32, r_coef, r_coef32, r_g64, r_g32, r_g32lo, r_rowmax, r_gscale, r_X, r_Dst, r_Vst, r_rhs, r_gent, r_gpart, r_G,
      r_dinv, r_L32, r_dinv32, r_b, r_tr, r_tpart, r_x, r_r, r_rpart, r_rowc, r_xmu, r_gam, r_tref, r_treoff, r_vhat, r_vfull, r_gscr, r_adj, r_gacc, r_gcpart, r_status, r_flags,
      r_kzP, r_kzp, r_kzgoff, r_kzvoff, r_kzG, r_kzT, r_kzb, r_kzx;
  Dev dev{};
  cudaStream_t last_stream = nullptr;
  int last_status = EDT_OK;
  // CUDA-graph replay of edt_invert (keyed on the call's pointers, dtypes and stream)
  bool use_graph = false;
  cudaGraphExec_t gexec = nullptr;
  const void* g_D = nullptr;
  void* g_V = nullptr;
  int g_Dt = -1, g_Vt = -1;
  cudaStream_t g_s = nullptr;
  // profiling
  bool prof = false;
  static constexpr int NSTAGE = 9;        // timed stages
  std::vector<cudaEvent_t> ev;   // [calls][NSTAGE][begin, end]
  // auxiliary stream of edt_invert: the depth march (and the window geometry's kernel rows)
  // runs there concurrently with the data transform on the caller's stream
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::vector<cudaEvent_t> ev_la;      // look-ahead of the double-float Cholesky (on aux)
  // host-buffer calls: the input copy on its own stream into one of two staging buffers, so
  // one call's copy overlaps the previous call's stages (edt_set_host_pipeline)
  bool host_pipe = false;
  int host_buf = 0;
  size_t dst_half = 0;
  cudaStream_t cpy = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  int prof_calls = 0;
  int prof_used[NSTAGE] = {};
};

namespace {

constexpr int kProfCalls = 256;   // calls whose stage events are kept between reads

const char* kStageNames[edt_ctx::NSTAGE] = {"green", "kernel_rows", "transform_rhs", "gram_prep",
                                            "gram", "gram_reduce", "cholesky", "refine",
                                            "inverse"};

int validate(const edt_config* c) {
  if (!c) return EDT_EINVAL;
  if (!is_pow2(c->nx) || c->nx < 16 || c->nx > 1024) return EDT_EUNSUPPORTED;
  if (!(c->dx > 0) || !(c->dz > 0) || !(c->z0 >= 0) || !(c->eps >= 0)) return EDT_EINVAL;
  if (c->nz < 1 || c->nz > 512) return EDT_EUNSUPPORTED;
  if (c->nfreq < 1 || c->nfreq > 32767 || !c->freq_hz) return EDT_EINVAL;
  if (c->nlayer < 1 || c->nlayer > 4096 || !c->layer_top_m || !c->layer_vel_mps) return EDT_EINVAL;
  if (c->layer_top_m[0] != 0.0) return EDT_EINVAL;
  for (int j = 0; j < c->nlayer; ++j) {
    if (!(c->layer_vel_mps[j] > 0) || !std::isfinite(c->layer_vel_mps[j])) return EDT_EINVAL;
    if (j > 0 && !(c->layer_top_m[j] > c->layer_top_m[j - 1])) return EDT_EINVAL;
  }
  for (int f = 0; f < c->nfreq; ++f)
    if (!(c->freq_hz[f] > 0) || !std::isfinite(c->freq_hz[f])) return EDT_EINVAL;
  if (c->precision != EDT_FP64 && c->precision != EDT_MIXED) return EDT_EINVAL;
  if (c->precision == EDT_MIXED) {
    if (c->passes != 1 && c->passes != 3) return EDT_EINVAL;
    if (c->refine < 0 || c->refine > 8) return EDT_EINVAL;
    if (c->nz > 256) return EDT_EUNSUPPORTED;
    // the tensor-core producer addresses the FP32 table with 32-bit element offsets
    if (double(c->nfreq) * (c->nx / 2 + 1) * c->nz >= 4294967295.0) return EDT_EUNSUPPORTED;
  }
  if (!(c->alpha >= 0) || !std::isfinite(c->alpha)) return EDT_EINVAL;
  if (!std::isfinite(c->cutoff)) return EDT_EINVAL;
  if (c->fold != 0 && c->fold != 1) return EDT_EINVAL;
  if (c->chol_df < 0 || c->chol_df > 3) return EDT_EINVAL;
  if (c->freq_chunk < 0 || c->gram_seg_rows < 0) return EDT_EINVAL;
  if (c->resid < 0 || c->resid > 2) return EDT_EINVAL;
  if (c->sub_begin < 0 || c->sub_end < 0 || c->sub_begin > c->sub_end) return EDT_EINVAL;
  if (c->sub_end > c->nx / 2 + 1) return EDT_EINVAL;
  if (c->sub_end > c->sub_begin && c->geometry == EDT_GEOM_WINDOW) return EDT_EUNSUPPORTED;
  if (c->resid == 2 && (c->geometry == EDT_GEOM_WINDOW || c->precision != EDT_MIXED)) return EDT_EUNSUPPORTED;
  if (c->geometry != EDT_GEOM_LINE && c->geometry != EDT_GEOM_WINDOW) return EDT_EINVAL;
  if (c->solver != EDT_SOLVE_DAMPED && c->solver != EDT_SOLVE_TSVD) return EDT_EINVAL;
  if (!std::isfinite(c->tsvd_tol) || !(c->kz_disk >= 0) || !std::isfinite(c->kz_disk)) return EDT_EINVAL;
  if (c->solver == EDT_SOLVE_TSVD || c->kz_disk > 0) {
    if (c->precision != EDT_FP64 || c->geometry != EDT_GEOM_LINE) return EDT_EUNSUPPORTED;
    if (c->solver == EDT_SOLVE_TSVD && c->nz > TSVD_MAX_NZ) return EDT_EUNSUPPORTED;
  }
  if (c->geometry == EDT_GEOM_WINDOW) {
    if (c->ny < 1 || c->wx < 1 || c->wy < 1 || !(c->dy > 0)) return EDT_EINVAL;
    if (c->precision != EDT_MIXED) return EDT_EUNSUPPORTED;
    if (!fa_supported(c->nx, c->ny, c->wx, c->wy)) return EDT_EUNSUPPORTED;
  }
  return EDT_OK;
}

// Window geometry: pairs {k_m, -k_m}, their rows (f, j) kept by the cut, the (f, j) lists
// the assembly and data kernels walk, and |k| of every table row (the quadrant
// |a_x| <= nx/2, |a_y| <= ny/2 of the wavenumber grid).  Same order and same IEEE double
// cut test as the finite-aperture oracle.
void plan_window(edt_ctx* c, double cmin) {
  const edt_config& g = c->cfg;
  const int nx = c->N, ny = c->ny, wx = c->wx, wy = c->wy, W = c->W, nf = c->nf;
  const int hx = nx / 2 + 1, hy = ny / 2 + 1;
  c->kval.resize(size_t(hx) * hy);
  for (int qy = 0; qy < hy; ++qy)
    for (int qx = 0; qx < hx; ++qx) {
      const double kx = 2.0 * M_PI * qx / (nx * g.dx), ky = 2.0 * M_PI * qy / (ny * g.dy);
      c->kval[size_t(qy) * hx + qx] = std::sqrt(kx * kx + ky * ky);
    }
  c->pair_m.clear();
  for (int my = 0; my <= ny / 2; ++my) {
    const bool half = my == 0 || 2 * my == ny;
    for (int mx = 0; mx < (half ? nx / 2 + 1 : nx); ++mx) c->pair_m.push_back(my * nx + mx);
  }
  c->nsub = int(c->pair_m.size());
  auto sgn = [](int n, int N) { return n <= N / 2 ? n : n - N; };
  std::vector<double> lim(nf);
  for (int f = 0; f < nf; ++f) lim[f] = (2.0 * g.cutoff * c->freq[f]) * (2.0 * g.cutoff * c->freq[f]);
  std::vector<std::vector<int2>> lists(size_t(nf) * W);
  c->rows.clear();
  c->row_off.assign(c->nsub + 1, 0);
  c->counts_cut.assign(c->nsub, 0);
  for (int p = 0; p < c->nsub; ++p) {
    c->row_off[p] = (long long)c->rows.size();
    const int m = c->pair_m[p], my = m / nx, mx = m - my * nx;
    const double mxs = double(sgn(mx, nx)) / (nx * g.dx), mys = double(sgn(my, ny)) / (ny * g.dy);
    for (int f = 0; f < nf; ++f)
      for (int jy = 0; jy < wy; ++jy)
        for (int jx = 0; jx < wx; ++jx) {
          bool keep = true;
          if (g.cutoff > 0) {
            const double jxs = double(jx - wx / 2) / (wx * g.dx), jys = double(jy - wy / 2) / (wy * g.dy);
            for (int sg = 0; sg < 2 && keep; ++sg) {
              const double vx = sg == 0 ? mxs + jxs : mxs + (-1.0) * jxs;
              const double vy = sg == 0 ? mys + jys : mys + (-1.0) * jys;
              keep = (cmin * cmin) * (vy * vy + vx * vx) < lim[f];
            }
          }
          if (!keep) continue;
          const int j = jy * wx + jx;
          lists[size_t(f) * W + j].push_back(make_int2(m, int(c->rows.size())));
          c->rows.push_back(uint32_t(f) << 16 | uint32_t(j));
          c->counts_cut[p] += 1;
        }
  }
  c->row_off[c->nsub] = (long long)c->rows.size();
  c->fj_off.assign(size_t(nf) * W + 1, 0);
  c->fj_ent.clear();
  c->fj_ent.reserve(c->rows.size());
  for (size_t i = 0; i < lists.size(); ++i) {
    c->fj_off[i] = int(c->fj_ent.size());
    c->fj_ent.insert(c->fj_ent.end(), lists[i].begin(), lists[i].end());
  }
  c->fj_off[lists.size()] = int(c->fj_ent.size());
  c->jact.assign(size_t(nf) * W, -1);
  c->jmap.assign(size_t(nf) * W, -1);
  c->nact.assign(nf, 0);
  for (int f = 0; f < nf; ++f)
    for (int j = 0; j < W; ++j)
      if (!lists[size_t(f) * W + j].empty()) {
        c->jmap[size_t(f) * W + j] = c->nact[f];
        c->jact[size_t(f) * W + c->nact[f]] = j;
        c->nact[f]++;
      }
  c->cf.resize(nf);
  for (int f = 0; f < nf; ++f) {
    const double2 om = make_double2(c->fc[f].om_re, c->fc[f].om_im);
    const double2 o2 = om * om;
    const double sc = g.dx * g.dy * g.dz;
    c->cf[f] = make_double2(o2.x * sc, o2.y * sc);
  }
}

// Band-limited transform of the mixed path: per frequency the band of signed wavenumber
// indices that the cut keeps (the same strict test as the row plan), then chunks of planes
// whose band spectra fit in L2 together (or freq_chunk planes each), the column-pass block
// table and, per chunk, the prefix counts of its rows over the subproblems.
void plan_band(edt_ctx* c, double cmin) {
  const edt_config& g = c->cfg;
  const int N = c->N, nf = c->nf, ns = c->nsub;
  c->band_mode = g.precision == EDT_MIXED && band_supported(N);
  c->band.assign(nf, BandInfo{0, 0, 0, 0});
  c->bcol.clear(); c->cpre.clear(); c->bchunks.clear();
  c->band_ymax = c->band_xmax = 0; c->band_maxplanes = 0;
  if (!c->band_mode) return;
  for (int f = 0; f < nf; ++f) {
    BandInfo& b = c->band[f];
    if (g.cutoff > 0) {
      const double lim = c->fc[f].lim;
      if (!(0.0 < lim)) { b.lo = 0; b.w = 0; continue; }       // even n' = 0 is cut
      int P = 0;
      while (P < N / 2 && double(P + 1) * cmin < lim) ++P;
      if (P >= N / 2) { b.lo = -N / 2 + 1; b.w = N; }
      else { b.lo = -P; b.w = 2 * P + 1; }
    } else {
      b.lo = -N / 2 + 1; b.w = N;
    }
  }
  const size_t budget = size_t(c->band_budget_mb) << 20;   // bytes of Y + Xc per chunk
  const int bc = c->tune_bc;
  int f0 = 0;
  while (f0 < nf) {
    BandChunk ch{f0, f0, int(c->bcol.size()), 0, 0, int(c->bchunks.size())};
    size_t ysz = 0, xsz = 0;
    while (ch.f1 < nf) {
      const BandInfo& b = c->band[ch.f1];
      const size_t yb = size_t(N) * b.w, xb = size_t(b.w) * b.w;
      if (g.freq_chunk > 0 ? ch.f1 - f0 >= g.freq_chunk
                           : (ch.f1 > f0 && (ysz + yb + xsz + xb) * sizeof(float2) > budget))
        break;
      c->band[ch.f1].yoff = (long long)ysz;
      c->band[ch.f1].xoff = (long long)xsz;
      ysz += yb; xsz += xb;
      for (int pb = 0; pb < b.w; pb += bc) c->bcol.push_back(make_int2(ch.f1, pb));
      ch.f1++;
    }
    ch.nbcol = int(c->bcol.size()) - ch.bcol0;
    const size_t base = c->cpre.size();
    c->cpre.resize(base + ns + 1, 0);
    for (int m = 0; m < ns; ++m) {
      const long long* mo = &c->row_off_mf[size_t(m) * (nf + 1)];
      c->cpre[base + m + 1] = c->cpre[base + m] + (mo[ch.f1] - mo[ch.f0]);
    }
    ch.nrow = c->cpre[base + ns];
    c->band_ymax = std::max(c->band_ymax, ysz);
    c->band_xmax = std::max(c->band_xmax, xsz);
    c->band_maxplanes = std::max(c->band_maxplanes, ch.f1 - ch.f0);
    c->bchunks.push_back(ch);
    f0 = ch.f1;
  }
}

// Solver variants: the depth basis (columns in order of |k_z|: constant, then cos and sin of
// 2 pi l j / nz for l = 1, 2, ..., then (-1)^j for even nz, each normalised) and, for the disk
// |(k_m, k_z)| <= kz_disk omega_max / c_min, the number of leading columns kept per k_m.
void plan_variant(edt_ctx* c) {
  const edt_config& g = c->cfg;
  c->variant = g.solver == EDT_SOLVE_TSVD || g.kz_disk > 0;
  c->kz_p.clear(); c->kz_goff.clear(); c->kz_voff.clear(); c->kz_P.clear();
  if (!(g.kz_disk > 0)) return;
  const int nz = c->nz;
  std::vector<int> lcol(nz);
  c->kz_P.assign(size_t(nz) * nz, 0.0);
  int col = 0;
  for (int l = 0; l <= nz / 2; ++l) {
    const bool pair = l > 0 && 2 * l < nz;
    for (int part = 0; part < (pair ? 2 : 1); ++part) {
      for (int j = 0; j < nz; ++j) {
        double v;
        if (l == 0) v = 1.0 / std::sqrt(double(nz));
        else if (!pair) v = (j % 2 == 0 ? 1.0 : -1.0) / std::sqrt(double(nz));
        else v = std::sqrt(2.0 / nz) * (part == 0 ? std::cos(2.0 * M_PI * l * j / nz) : std::sin(2.0 * M_PI * l * j / nz));
        c->kz_P[size_t(j) * nz + col] = v;
      }
      lcol[col++] = l;
    }
  }
  double fmax = 0.0, cmin = 1e300;
  for (double f : c->freq) fmax = std::max(fmax, f);
  for (double v : c->vel) cmin = std::min(cmin, v);
  const double K = g.kz_disk * 2.0 * M_PI * fmax / cmin;
  c->kz_p.resize(c->nsub);
  c->kz_goff.resize(c->nsub);
  c->kz_voff.resize(c->nsub);
  for (int m = 0; m < c->nsub; ++m) {
    const double km = 2.0 * M_PI * m / (c->N * g.dx);
    int p = 0;
    for (int k = 0; k < nz; ++k) {
      const double kz = 2.0 * M_PI * lcol[k] / (nz * g.dz);
      if (km * km + kz * kz <= K * K) p = k + 1; else break;
    }
    c->kz_p[m] = p;
    c->kz_goff[m] = (long long)m * nz * nz;
    c->kz_voff[m] = (long long)m * nz;
  }
}

// the reference gradient through the solve: line geometry, mixed path, the depth march's
// reverse-mode limits (misfit gradient) and at most 512 depths (the row products' vectors)
bool ref_grad_planned(const edt_ctx* c) {
  return c->cfg.precision == EDT_MIXED && !c->win && c->nlayer <= GRAD_MAX_LAYERS && c->N >= 64 &&
         c->nz <= 512;
}

void plan(edt_ctx* c) {
  const edt_config& g = c->cfg;
  c->N = g.nx; c->nk = g.nx / 2 + 1; c->nz = g.nz; c->nf = g.nfreq; c->nsub = g.nx / 2 + 1;
  c->nlayer = g.nlayer;
  c->win = g.geometry == EDT_GEOM_WINDOW;
  c->ny = c->win ? g.ny : 1;
  c->wx = c->win ? g.wx : 1;
  c->wy = c->win ? g.wy : 1;
  c->W = c->wx * c->wy;
  c->nxy = c->N * c->ny;
  if (c->win) c->nk = (g.nx / 2 + 1) * (c->ny / 2 + 1);
  const int N = c->N;
  const double L = double(N) * g.dx;
  // frequencies
  c->fc.resize(c->nf);
  for (int f = 0; f < c->nf; ++f) {
    FreqConst& q = c->fc[f];
    q.om_re = 2.0 * M_PI * c->freq[f];
    q.om_im = g.eps;
    double2 om = make_double2(q.om_re, q.om_im);
    double2 s = om * om;
    s = make_double2(s.x * g.dz / g.dx, s.y * g.dz / g.dx);
    q.s_abs = std::hypot(s.x, s.y);
    q.rot_re = s.x / q.s_abs;
    q.rot_im = -s.y / q.s_abs;
    q.lim = (g.cutoff * c->freq[f]) * L;
  }
  // depth samples -> layer and offset below its top (an interface belongs to the layer below)
  c->z_layer.resize(c->nz);
  c->z_off.resize(c->nz);
  for (int j = 0; j < c->nz; ++j) {
    double z = g.z0 + (j + 0.5) * g.dz;
    int l = int(std::upper_bound(c->tops.begin(), c->tops.end(), z) - c->tops.begin()) - 1;
    l = std::max(0, std::min(l, c->nlayer - 1));
    c->z_layer[j] = l;
    c->z_off[j] = z - c->tops[l];
  }
  // FP32 (hi, lo) pairs of the offset below the layer top and of 2 h_l - offset
  c->z_off32.assign(size_t(c->nz) * 4, 0.f);
  for (int j = 0; j < c->nz; ++j) {
    const int l = c->z_layer[j];
    const double off = c->z_off[j];
    const double o2 = l < c->nlayer - 1 ? 2.0 * (c->tops[l + 1] - c->tops[l]) - off : 0.0;
    const float oh = float(off), o2h = float(o2);
    c->z_off32[4 * j + 0] = oh; c->z_off32[4 * j + 1] = float(off - double(oh));
    c->z_off32[4 * j + 2] = o2h; c->z_off32[4 * j + 3] = float(o2 - double(o2h));
  }
  c->fc32.resize(c->nf);
  // line geometry: the FP32 table carries sqrt|s_f| (rows are products of two table rows);
  // window geometry: plain g (the assembly applies the prefactor)
  for (int f = 0; f < c->nf; ++f) c->fc32[f] = c->win ? 1.f : float(std::sqrt(c->fc[f].s_abs));
  const double cmin = *std::min_element(c->vel.begin(), c->vel.end());
  if (c->win) {
    plan_window(c, cmin);
    c->row_off_mf.assign(size_t(c->nsub) * (c->nf + 1), 0);
    c->fchunk = 0;
    c->band_mode = false;
  } else {
  // rows of every subproblem, in (f, p) order, evanescent cut and optional folding
  c->rows.clear();
  c->row_off.assign(c->nsub + 1, 0);
  c->row_off_mf.assign(size_t(c->nsub) * (c->nf + 1), 0);
  c->counts_cut.assign(c->nsub, 0);
  auto sidx = [N](int n) { return n <= N / 2 ? n : n - N; };
  const bool ranged = g.sub_end > g.sub_begin;
  std::vector<uint32_t> kept;
  std::vector<int> idx_of(size_t(N), -1);
  std::vector<char> done;
  for (int m = 0; m < c->nsub; ++m) {
    c->row_off[m] = (long long)c->rows.size();
    // a context restricted to subproblems [sub_begin, sub_end) plans no rows for the others
    const bool inrange = !ranged || (m >= g.sub_begin && m < g.sub_end);
    for (int f = 0; f < c->nf; ++f) {
      c->row_off_mf[size_t(m) * (c->nf + 1) + f] = (long long)c->rows.size();
      if (!inrange) continue;
      const double lim = c->fc[f].lim;
      // kept rows of (m, f), first in the order p = 0, N/2, 1, N-1, 2, N-2, ...
      kept.clear();
      for (int pi = 0; pi < N; ++pi) {
        int p;
        if (pi == 0) p = 0;
        else if (pi == 1) p = N / 2;
        else p = (pi & 1) ? N - (pi / 2) : pi / 2;
        const int q = (p - m + N) % N;
        bool keep = true;
        if (g.cutoff > 0) {
          keep = double(std::abs(sidx(p))) * cmin < lim && double(std::abs(sidx(q))) * cmin < lim;
        }
        if (!keep) continue;
        c->counts_cut[m] += 1;
        if (g.fold) {
          const int pp = (N - q) % N;          // first index of the reciprocal partner (-q, -p)
          if (pp == p) kept.push_back(row_pack(f, p, 0));
          else if (p < pp) kept.push_back(row_pack(f, p, 1));
        } else {
          kept.push_back(row_pack(f, p, 0));
        }
      }
      // then in chains p, p - m, p - 2m, ...: row (p, q = p - m) and the next row (q, q - m)
      // read the same table row g(|q|), so side by side the second read is served from L1.
      // A chain starts at a row whose p + m is not kept (every row is in exactly one chain;
      // rows left on a cycle are walked from the first of them).
      if (m == 0 || kept.size() < 2) {
        c->rows.insert(c->rows.end(), kept.begin(), kept.end());
      } else {
        for (size_t i = 0; i < kept.size(); ++i) idx_of[row_p(kept[i])] = int(i);
        done.assign(kept.size(), 0);
        auto walk = [&](size_t i0) {
          for (int j = int(i0); j >= 0 && !done[size_t(j)];
               j = idx_of[(row_p(kept[size_t(j)]) - m + N) % N]) {
            done[size_t(j)] = 1;
            c->rows.push_back(kept[size_t(j)]);
          }
        };
        for (size_t i = 0; i < kept.size(); ++i)
          if (idx_of[(row_p(kept[i]) + m) % N] < 0) walk(i);
        for (size_t i = 0; i < kept.size(); ++i)
          if (!done[i]) walk(i);
        for (uint32_t r : kept) idx_of[row_p(r)] = -1;
      }
    }
  }
  c->row_off[c->nsub] = (long long)c->rows.size();
  for (int m = 0; m < c->nsub; ++m) c->row_off_mf[size_t(m) * (c->nf + 1) + c->nf] = c->row_off[m + 1];
  // frequency planes per transform chunk: bounds the spectrum buffer (each chunk costs a
  // few partly filled waves of three launches, so the automatic size is large)
  {
    const size_t plane = size_t(N) * N * (g.precision == EDT_MIXED ? sizeof(float2) : sizeof(double2));
    const size_t want = g.freq_chunk > 0 ? size_t(g.freq_chunk) : (size_t(256) << 20) / plane;
    c->fchunk = int(std::max<size_t>(1, std::min<size_t>(c->nf, want)));
  }
  // the workspace holds the band buffers and tables of every autotuning candidate
  for (int mb : {16, 32, 48, 96})
    for (int bc : {4, 8, 16}) {
      const int mb0 = c->band_budget_mb, bc0 = c->tune_bc;
      c->band_budget_mb = mb; c->tune_bc = bc;
      plan_band(c, cmin);
      c->ws_band_elems = std::max(c->ws_band_elems, ((c->band_ymax * sizeof(float2) + 255) / 256 * 256) / sizeof(float2) + c->band_xmax);
      c->ws_bcol = std::max(c->ws_bcol, c->bcol.size());
      c->ws_cpre = std::max(c->ws_cpre, c->cpre.size());
      c->band_budget_mb = mb0; c->tune_bc = bc0;
    }
  plan_band(c, cmin);
  }
  c->rows_max_sub = 0;
  for (int m = 0; m < c->nsub; ++m) c->rows_max_sub = std::max(c->rows_max_sub, c->row_off[m + 1] - c->row_off[m]);
  // reference gradient through the solve (line geometry, mixed path): group the rows by the
  // table rows (f, |p|) and (f, |q|) they read, each group in row order
  c->tref.clear();
  c->tref_off.clear();
  if (ref_grad_planned(c)) {
    const size_t nte = size_t(c->nf) * c->nk;
    auto tab = [N](int n) { return n <= N / 2 ? n : N - n; };
    std::vector<long long> cnt(nte + 1, 0);
    for (int m = 0; m < c->nsub; ++m)
      for (long long r = c->row_off[m]; r < c->row_off[m + 1]; ++r) {
        const uint32_t row = c->rows[r];
        const int f = row_f(row), p = row_p(row), q = (p - m + N) % N;
        cnt[size_t(f) * c->nk + tab(p) + 1]++;
        cnt[size_t(f) * c->nk + tab(q) + 1]++;
      }
    for (size_t i = 0; i < nte; ++i) cnt[i + 1] += cnt[i];
    c->tref_off = cnt;
    c->tref.resize(size_t(cnt[nte]));
    for (int m = 0; m < c->nsub; ++m)
      for (long long r = c->row_off[m]; r < c->row_off[m + 1]; ++r) {
        const uint32_t row = c->rows[r];
        const int f = row_f(row), p = row_p(row), q = (p - m + N) % N;
        c->tref[size_t(cnt[size_t(f) * c->nk + tab(p)]++)] = make_int2(int(r), m << 1);
        c->tref[size_t(cnt[size_t(f) * c->nk + tab(q)]++)] = make_int2(int(r), (m << 1) | 1);
      }
  }
  // twiddles e^{-2 pi i k / N}
  c->tw64.resize(N / 2);
  c->tw32.resize(N / 2);
  for (int k = 0; k < N / 2; ++k) {
    double a = 2.0 * M_PI * double(k) / double(N);
    c->tw64[k] = make_double2(std::cos(a), -std::sin(a));
    c->tw32[k] = make_float2(float(std::cos(a)), float(-std::sin(a)));
  }
  // tensor-core Gram: split the concatenated rows evenly over the CTAs; a segment is the
  // part of one subproblem's rows that one CTA covers, each with its own partial slot
  c->seg_m.clear(); c->seg_row0.clear(); c->seg_nrow.clear(); c->cta_seg0.clear();
  c->m_slot0.assign(c->nsub + 1, 0);
  if (g.precision == EDT_MIXED) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long total = c->row_off[c->nsub];
    int ncta = int(std::max<long long>(1, std::min<long long>(sms, (total + TC_KC - 1) / TC_KC)));
    c->ncta_gram = ncta;
    // segments per CTA, slots ordered by m so each m's slots are contiguous
    std::vector<std::vector<std::pair<int, std::pair<long long, long long>>>> per_m(c->nsub);
    std::vector<std::vector<int>> cta_segs(ncta);
    struct Seg { int m, cta; long long r0, n; };
    std::vector<Seg> segs;
    const long long cap = gram_seg_cap(g);
    for (int k = 0; k < ncta; ++k) {
      long long a = total * k / ncta, b = total * (k + 1) / ncta;
      long long r = a;
      while (r < b) {
        int m = int(std::upper_bound(c->row_off.begin(), c->row_off.end(), r) - c->row_off.begin()) - 1;
        long long e = std::min(std::min(b, c->row_off[m + 1]), r + cap);
        segs.push_back({m, k, r, e - r});
        r = e;
      }
    }
    // slot of a segment = its index when segments are sorted by (m, cta)
    std::vector<int> order(segs.size());
    for (size_t i = 0; i < segs.size(); ++i) order[i] = int(i);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return segs[x].m < segs[y].m; });
    std::vector<int> slot_of(segs.size());
    for (size_t i = 0; i < order.size(); ++i) slot_of[order[i]] = int(i);
    std::vector<int> cnt(c->nsub, 0);
    for (auto& s : segs) cnt[s.m]++;
    for (int m = 0; m < c->nsub; ++m) c->m_slot0[m + 1] = c->m_slot0[m] + cnt[m];
    // per-CTA segment lists in row order; seg_m/row0/nrow indexed by slot
    c->seg_m.resize(segs.size()); c->seg_row0.resize(segs.size()); c->seg_nrow.resize(segs.size());
    for (size_t i = 0; i < segs.size(); ++i) {
      int sl = slot_of[i];
      c->seg_m[sl] = segs[i].m; c->seg_row0[sl] = segs[i].r0; c->seg_nrow[sl] = segs[i].n;
    }
    // cta_seg0 points into a per-CTA list of slots stored after the slot tables
    c->cta_seg0.assign(ncta + 1, 0);
    std::vector<int> cta_slots;
    for (int k = 0; k < ncta; ++k) {
      c->cta_seg0[k] = int(cta_slots.size());
      for (size_t i = 0; i < segs.size(); ++i) if (segs[i].cta == k) cta_slots.push_back(slot_of[i]);
    }
    c->cta_seg0[ncta] = int(cta_slots.size());
    c->cta_seg0.insert(c->cta_seg0.end(), cta_slots.begin(), cta_slots.end());
    c->nslot = int(segs.size());
  }
  plan_variant(c);
}

void layout(edt_ctx* c) {
  size_t off = 0;
  auto take = [&](Region& r, size_t bytes) {
    off = align_up(off, 256);
    r.off = off; r.bytes = bytes;
    off += bytes;
  };
  const size_t nf = c->nf, N = c->N, nk = c->nk, nz = c->nz, ns = c->nsub;
  const bool mixed = c->cfg.precision == EDT_MIXED;
  const size_t R = c->rows.size();
  take(c->r_fc, nf * sizeof(FreqConst));
  take(c->r_ltop, c->nlayer * sizeof(double));
  take(c->r_lvel, c->nlayer * sizeof(double));
  take(c->r_zl, nz * sizeof(int));
  take(c->r_zo, nz * sizeof(double));
  take(c->r_rows, std::max<size_t>(R, 1) * sizeof(uint32_t));
  take(c->r_roff, (ns + 1) * sizeof(long long));
  take(c->r_roffmf, ns * (nf + 1) * sizeof(long long));
  take(c->r_band, nf * sizeof(BandInfo));
  take(c->r_bcol, std::max<size_t>(std::max(c->ws_bcol, c->bcol.size()), 1) * sizeof(int2));
  take(c->r_cpre, std::max<size_t>(std::max(c->ws_cpre, c->cpre.size()), 1) * sizeof(long long));
  const size_t nxy = c->nxy, W = c->W, nzs = size_t((c->nz + 1) & ~1);
  take(c->r_kval, std::max<size_t>(c->kval.size(), 1) * sizeof(double));
  take(c->r_pairm, std::max<size_t>(c->pair_m.size(), 1) * sizeof(int));
  take(c->r_fjoff, std::max<size_t>(c->fj_off.size(), 1) * sizeof(int));
  take(c->r_fjent, std::max<size_t>(c->fj_ent.size(), 1) * sizeof(int2));
  take(c->r_jact, std::max<size_t>(c->jact.size(), 1) * sizeof(int));
  take(c->r_jmap, std::max<size_t>(c->jmap.size(), 1) * sizeof(int));
  take(c->r_Gs, c->win ? nz * nxy * sizeof(float2) : 0);
  const size_t wact = c->nact.empty() ? 1 : size_t(std::max(1, *std::max_element(c->nact.begin(), c->nact.end())));
  take(c->r_U, c->win ? wact * nz * (size_t(c->ny / 2 + 1) * N) * sizeof(float2) : 0);
  take(c->r_Dw, c->win ? nf * W * nxy * sizeof(float2) : 0);
  take(c->r_A32, c->win ? (R + 1) * nzs * sizeof(float2) : 0);
  take(c->r_tw64, (N / 2) * sizeof(double2));
  take(c->r_tw32, (N / 2) * sizeof(float2));
  take(c->r_segm, std::max<size_t>(c->seg_m.size(), 1) * sizeof(int));
  take(c->r_segr0, std::max<size_t>(c->seg_row0.size(), 1) * sizeof(long long));
  take(c->r_segn, std::max<size_t>(c->seg_nrow.size(), 1) * sizeof(long long));
  take(c->r_ctas, std::max<size_t>(c->cta_seg0.size(), 1) * sizeof(int));
  take(c->r_mslot, (ns + 1) * sizeof(int));
  take(c->r_zo32, nz * 4 * sizeof(float));
  take(c->r_fc32, nf * sizeof(float));
  take(c->r_coef, nf * nk * c->nlayer * 7 * sizeof(double2));
  take(c->r_coef32, mixed ? nf * nk * c->nlayer * 8 * sizeof(float) : 0);
  take(c->r_g64, nf * nk * nz * sizeof(double2));
  take(c->r_g32, mixed ? nf * nk * size_t((c->nz + 1) & ~1) * sizeof(float2) : 0);
  take(c->r_g32lo, c->resid_df ? nf * nk * size_t((c->nz + 1) & ~1) * sizeof(float2) : 0);
  take(c->r_rowmax, mixed && !c->win ? nf * nk * sizeof(float) : 0);
  take(c->r_gscale, mixed && !c->win ? std::max<size_t>(c->nslot, 1) * sizeof(int2) : 0);
  // full planes of the forward model (and of the FP64 transform), or the band spectra of
  // one chunk (Y, then Xc at a 256-byte boundary); one call uses one of the two
  take(c->r_X, std::max(size_t(c->fchunk) * N * N * (mixed ? sizeof(float2) : sizeof(double2)),
                        std::max(align_up(c->band_ymax * sizeof(float2), 256) + c->band_xmax * sizeof(float2),
                                 c->ws_band_elems * sizeof(float2))));
  c->dst_half = align_up((c->win ? nf * nxy * W : nf * N * N) * sizeof(double2), 256);
  take(c->r_Dst, 2 * c->dst_half);                 // two staging buffers
  take(c->r_Vst, (c->win ? nxy : N) * nz * sizeof(double));
  // right-hand sides; the mixed path's tensor-core Gram bulk-copies whole stages of 32 rows,
  // so its array (like the row metadata) carries 32 rows of padding
  take(c->r_rhs, (mixed ? R + 32 : std::max<size_t>(R, 1)) * 2 * (mixed ? sizeof(float2) : sizeof(double2)));
  take(c->r_gent, mixed ? (R + 32) * sizeof(GramRow) : 0);
  take(c->r_gpart, mixed ? size_t(c->nslot) * TC_M * tc_cols(c->nz) * sizeof(float) : 0);
  take(c->r_G, ns * nz * nz * sizeof(double));
  take(c->r_dinv, ns * nz * sizeof(double));
  take(c->r_L32, mixed && c->cfg.refine > 0 ? ns * nz * nz * sizeof(float) : 0);
  take(c->r_dinv32, mixed && c->cfg.refine > 0 ? ns * nz * sizeof(float) : 0);
  take(c->r_b, ns * nz * 2 * sizeof(double));
  take(c->r_tr, ns * sizeof(double));
  take(c->r_tpart, mixed ? std::max<size_t>(c->nslot, 1) * gram_trace_parts() * sizeof(double) : 0);
  take(c->r_x, ns * nz * 2 * sizeof(double));
  take(c->r_r, ns * nz * 2 * sizeof(double));
  take(c->r_rpart, mixed && c->cfg.refine > 0
                       ? ns * size_t(refine_stride(c->rows_max_sub)) * nz * 2 * sizeof(double) : 0);
  take(c->r_vhat, ns * nz * sizeof(double2));
  take(c->r_vfull, (c->win ? nxy : N) * nz * sizeof(double2));
  // misfit gradients: line geometry, mixed path (their dJ/dg buffer aliases r_g64, which
  // holds nf (N/2 + 1) nz complex doubles >= nf N nz complex floats)
  const bool grad = !c->win && mixed && c->nlayer <= GRAD_MAX_LAYERS && N >= 64;
  take(c->r_gscr, grad ? nf * size_t(c->nlayer) * 8 * nk * sizeof(double2) : 0);
  take(c->r_adj, grad ? size_t(N) * nz * sizeof(double2) : 0);
  take(c->r_gacc, grad ? size_t(1 + c->nlayer) * sizeof(double) : 0);
  take(c->r_gcpart, grad ? size_t(nf) * ((nk + 127) / 128) * 4 * c->nlayer * sizeof(double) : 0);
  const bool rg = ref_grad_planned(c);
  take(c->r_rowc, rg ? std::max<size_t>(R, 1) * 2 * sizeof(float4) : 0);
  take(c->r_xmu, rg ? ns * nz * sizeof(float4) : 0);
  take(c->r_gam, rg ? ns * sizeof(double) : 0);
  take(c->r_tref, rg ? std::max<size_t>(c->tref.size(), 1) * sizeof(int2) : 0);
  take(c->r_treoff, rg ? c->tref_off.size() * sizeof(long long) : 0);
  take(c->r_status, ns * sizeof(int));
  take(c->r_flags, 8 * sizeof(unsigned));
  const bool disk = !c->kz_p.empty();
  take(c->r_kzP, disk ? size_t(nz) * nz * sizeof(double) : 0);
  take(c->r_kzp, disk ? ns * sizeof(int) : 0);
  take(c->r_kzgoff, disk ? ns * sizeof(long long) : 0);
  take(c->r_kzvoff, disk ? ns * sizeof(long long) : 0);
  take(c->r_kzG, disk ? ns * nz * nz * sizeof(double) : 0);
  take(c->r_kzT, disk ? ns * nz * nz * sizeof(double) : 0);
  take(c->r_kzb, disk ? ns * nz * 2 * sizeof(double) : 0);
  take(c->r_kzx, disk ? ns * nz * 2 * sizeof(double) : 0);
  c->ws_bytes = align_up(off, 256);
}

template <typename P> P at(edt_ctx* c, const Region& r) {
  return reinterpret_cast<P>(static_cast<char*>(c->ws) + r.off);
}

void bind(edt_ctx* c) {
  Dev& d = c->dev;
  d.N = c->N; d.nk = c->nk; d.nz = c->nz; d.nf = c->nf; d.nsub = c->nsub; d.nlayer = c->nlayer;
  d.nzs = (c->nz + 1) & ~1;
  d.precision = c->cfg.precision; d.passes = c->cfg.passes; d.fold = c->cfg.fold;
  // the mixed path factors in double-float unless native FP64 is asked for (chol_df = 2)
  d.chol_df = c->cfg.precision == EDT_MIXED && c->cfg.chol_df != 2 ? 1 : 0;
  d.chol_tc = d.chol_df && c->cfg.chol_df == 3 ? 1 : 0;
  d.alpha = c->cfg.alpha; d.dx = c->cfg.dx; d.dz = c->cfg.dz;
  d.fc = at<const FreqConst*>(c, c->r_fc);
  d.layer_top = at<const double*>(c, c->r_ltop);
  d.layer_vel = at<const double*>(c, c->r_lvel);
  d.z_layer = at<const int*>(c, c->r_zl);
  d.z_off = at<const double*>(c, c->r_zo);
  d.rows = at<const uint32_t*>(c, c->r_rows);
  d.row_off = at<const long long*>(c, c->r_roff);
  d.row_off_mf = at<const long long*>(c, c->r_roffmf);
  d.fchunk = c->fchunk;
  d.rows_max_sub = c->rows_max_sub;
  d.tune_bc = c->tune_bc; d.tune_rf = c->tune_rf; d.tune_zc = c->tune_zc;
  d.geom = c->win ? EDT_GEOM_WINDOW : EDT_GEOM_LINE;
  d.ny = c->ny; d.wx = c->wx; d.wy = c->wy; d.W = c->W; d.nxy = c->nxy; d.dy = c->cfg.dy;
  d.kval = c->win ? at<const double*>(c, c->r_kval) : nullptr;
  d.pair_m = at<const int*>(c, c->r_pairm);
  d.fj_off = at<const int*>(c, c->r_fjoff);
  d.fj_ent = at<const int2*>(c, c->r_fjent);
  d.jact = at<const int*>(c, c->r_jact);
  d.jmap = at<const int*>(c, c->r_jmap);
  d.Gs = c->r_Gs.bytes ? at<float2*>(c, c->r_Gs) : nullptr;
  d.U = c->r_U.bytes ? at<float2*>(c, c->r_U) : nullptr;
  d.Dw = c->r_Dw.bytes ? at<float2*>(c, c->r_Dw) : nullptr;
  d.A32 = c->r_A32.bytes ? at<float2*>(c, c->r_A32) : nullptr;
  d.ones_row = (long long)c->rows.size();
  d.band = at<const BandInfo*>(c, c->r_band);
  d.bcol = at<const int2*>(c, c->r_bcol);
  d.cpre = at<const long long*>(c, c->r_cpre);
  d.Yc = at<float2*>(c, c->r_X);
  d.Xc = reinterpret_cast<float2*>(static_cast<char*>(c->ws) + c->r_X.off +
                                   align_up(c->band_ymax * sizeof(float2), 256));
  d.tw64 = at<const double2*>(c, c->r_tw64);
  d.tw32 = at<const float2*>(c, c->r_tw32);
  d.seg_m = at<const int*>(c, c->r_segm);
  d.seg_row0 = at<const long long*>(c, c->r_segr0);
  d.seg_nrow = at<const long long*>(c, c->r_segn);
  d.cta_seg0 = at<const int*>(c, c->r_ctas);
  d.m_slot0 = at<const int*>(c, c->r_mslot);
  d.nseg = c->nslot; d.ncta_gram = c->ncta_gram;
  d.coef = at<double2*>(c, c->r_coef);
  d.coef32 = c->r_coef32.bytes ? at<float*>(c, c->r_coef32) : nullptr;
  d.z_off32 = at<const float*>(c, c->r_zo32);
  d.fc32_sqrt_s = at<const float*>(c, c->r_fc32);
  d.g64 = at<double2*>(c, c->r_g64);
  d.g32 = c->r_g32.bytes ? at<float2*>(c, c->r_g32) : nullptr;
  d.g32lo = c->r_g32lo.bytes ? at<float2*>(c, c->r_g32lo) : nullptr;
  d.rowmax = c->r_rowmax.bytes ? at<float*>(c, c->r_rowmax) : nullptr;
  d.gscale = c->r_gscale.bytes ? at<int2*>(c, c->r_gscale) : nullptr;
  d.f16 = d.gscale != nullptr;
  d.resid_df = c->resid_df ? 1 : 0;
  d.rowtab32 = c->win ? d.A32 : d.g32;
  d.X = at<void*>(c, c->r_X);
  d.Dstage = at<void*>(c, c->r_Dst);
  d.Vstage = at<void*>(c, c->r_Vst);
  d.rhs = at<void*>(c, c->r_rhs);
  d.gent = c->r_gent.bytes ? at<GramRow*>(c, c->r_gent) : nullptr;
  d.gpart = c->r_gpart.bytes ? at<float*>(c, c->r_gpart) : nullptr;
  d.G = at<double*>(c, c->r_G);
  d.dinv = at<double*>(c, c->r_dinv);
  d.L32 = c->r_L32.bytes ? at<float*>(c, c->r_L32) : nullptr;
  d.dinv32 = c->r_dinv32.bytes ? at<float*>(c, c->r_dinv32) : nullptr;
  d.b = at<double*>(c, c->r_b);
  d.trace = at<double*>(c, c->r_tr);
  d.tpart = c->r_tpart.bytes ? at<double*>(c, c->r_tpart) : nullptr;
  d.x = at<double*>(c, c->r_x);
  d.r = at<double*>(c, c->r_r);
  d.rpart = c->r_rpart.bytes ? at<double*>(c, c->r_rpart) : nullptr;
  d.rf_stride = refine_stride(c->rows_max_sub);
  d.vhat = at<double2*>(c, c->r_vhat);
  d.vfull = at<double2*>(c, c->r_vfull);
  d.gscr = c->r_gscr.bytes ? at<double2*>(c, c->r_gscr) : nullptr;
  d.adj = c->r_adj.bytes ? at<double2*>(c, c->r_adj) : nullptr;
  d.gacc = c->r_gacc.bytes ? at<double*>(c, c->r_gacc) : nullptr;
  d.gcpart = c->r_gcpart.bytes ? at<double*>(c, c->r_gcpart) : nullptr;
  d.gbar = c->r_gscr.bytes ? reinterpret_cast<float2*>(d.g64) : nullptr;
  d.rowc = c->r_rowc.bytes ? at<float4*>(c, c->r_rowc) : nullptr;
  d.xmu = c->r_xmu.bytes ? at<float4*>(c, c->r_xmu) : nullptr;
  d.gam = c->r_gam.bytes ? at<double*>(c, c->r_gam) : nullptr;
  d.tref = c->r_tref.bytes ? at<const int2*>(c, c->r_tref) : nullptr;
  d.tref_off = c->r_treoff.bytes ? at<const long long*>(c, c->r_treoff) : nullptr;
  d.refine_nodata = 0;
  d.status = at<int*>(c, c->r_status);
  d.flags = at<unsigned*>(c, c->r_flags);
  d.solver = c->cfg.solver;
  d.tsvd_tol = c->cfg.tsvd_tol;
  const bool disk = c->r_kzP.bytes > 0;
  d.kz_P = disk ? at<const double*>(c, c->r_kzP) : nullptr;
  d.kz_p = disk ? at<const int*>(c, c->r_kzp) : nullptr;
  d.kz_goff = disk ? at<const long long*>(c, c->r_kzgoff) : nullptr;
  d.kz_voff = disk ? at<const long long*>(c, c->r_kzvoff) : nullptr;
  d.kz_G = disk ? at<double*>(c, c->r_kzG) : nullptr;
  d.kz_T = disk ? at<double*>(c, c->r_kzT) : nullptr;
  d.kz_b = disk ? at<double*>(c, c->r_kzb) : nullptr;
  d.kz_x = disk ? at<double*>(c, c->r_kzx) : nullptr;
}

template <typename T>
int upload(edt_ctx* c, const Region& r, const std::vector<T>& v) {
  if (v.empty()) return EDT_OK;
  cudaError_t e = cudaMemcpy(at<void*>(c, r), v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? EDT_OK : cuda_fail(e);
}

#define EDT_TRY(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) return cuda_fail(_e); } while (0)
#define EDT_TRYI(x) do { int _r = (x); if (_r != EDT_OK) return _r; } while (0)

// begin (end = 0) or end (end = 1) of a stage, recorded on the stream the stage runs on
void prof_ev(edt_ctx* c, int stage, int end, cudaStream_t s) {
  if (!c->prof || c->prof_calls >= kProfCalls) return;
  cudaEventRecord(c->ev[(size_t(c->prof_calls) * edt_ctx::NSTAGE + stage) * 2 + end], s);
  c->prof_used[stage] = 1;
}

// Tables the depth march writes for an inversion: FP64 (FP64 path); the FP32 table by the
// fast FP32 evaluation (mixed path with the FP32 residual, ~1e-7 relative; on the line
// geometry from FP32 coefficients, a few 1e-6, which the damping of that residual's regime,
// alpha >= 1e-3, keeps far below the result's tolerance); the FP32 table rounded from the FP64
// evaluation with its remainder, the double-float pair the FP64-accurate residual reads (mixed
// line path, resid 2).
int green_tables(const edt_ctx* c) {
  if (c->cfg.precision != EDT_MIXED) return GREEN_G64;
  if (c->resid_df) return GREEN_G32DF;
  return c->win ? GREEN_G32 : GREEN_G32F;
}

// Data transform and right-hand-side gather, chunk by chunk of frequency planes.
int transform_rhs(edt_ctx* c, const void* D, int D_dtype, cudaStream_t s) {
  const Dev& d = c->dev;
  const bool mixed = c->cfg.precision == EDT_MIXED;
  if (c->win) {
    EDT_TRY(launch_fa_data(d, D, D_dtype, s));
    return EDT_OK;
  }
  if (c->band_mode) {
    for (const BandChunk& ch : c->bchunks) EDT_TRY(launch_band_chunk(d, ch, D, D_dtype, s));
    return EDT_OK;
  }
  for (int f0 = 0; f0 < d.nf; f0 += d.fchunk) {
    const int nfc = std::min(d.fchunk, d.nf - f0);
    if (mixed) {
      EDT_TRY(launch_transform<float>(d, D, D_dtype, f0, nfc, s));
      EDT_TRY(launch_rhs<float>(d, f0, nfc, s));
    } else {
      EDT_TRY(launch_transform<double>(d, D, D_dtype, f0, nfc, s));
      EDT_TRY(launch_rhs<double>(d, f0, nfc, s));
    }
  }
  return EDT_OK;
}

// Window geometry: the assembled kernel rows of every frequency into the row table.
int kernel_rows(edt_ctx* c, cudaStream_t s) {
  if (!c->win) return EDT_OK;
  for (int f = 0; f < c->nf; ++f) EDT_TRY(launch_fa_rows(c->dev, f, c->nact[f], c->cf[f], s));
  return EDT_OK;
}

// One inversion on s.  do_transform = false: the right-hand sides were imported into the
// workspace (edt_import_rhs); do_inverse = false: the solutions stay in the workspace.
int run_invert(edt_ctx* c, const void* D, int D_dtype, void* V, int V_dtype, cudaStream_t s,
               bool do_transform = true, bool do_inverse = true) {
  const Dev& d = c->dev;
  const bool mixed = c->cfg.precision == EDT_MIXED;
  c->last_stream = s;
  // the Gram's wait-expired flag describes this call only
  if (mixed) EDT_TRY(cudaMemsetAsync(d.flags, 0, sizeof(unsigned), s));
  // fork: the depth march (FP64-bound) and, for the window geometry, the kernel rows it
  // feeds run on the auxiliary stream while the data transform (FP32 and memory) runs on s
  const bool ov = c->tune_ov != 0;
  cudaStream_t sg = ov ? c->aux : s;
  if (ov) {
    EDT_TRY(cudaEventRecord(c->ev_fork, s));
    EDT_TRY(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
  }
  prof_ev(c, 0, 0, sg);
  EDT_TRY(launch_green(d, sg, green_tables(c)));
  prof_ev(c, 0, 1, sg);
  prof_ev(c, 1, 0, sg);
  EDT_TRYI(kernel_rows(c, sg));
  prof_ev(c, 1, 1, sg);
  if (ov) EDT_TRY(cudaEventRecord(c->ev_join, c->aux));
  prof_ev(c, 2, 0, s);
  if (do_transform) EDT_TRYI(transform_rhs(c, D, D_dtype, s));
  prof_ev(c, 2, 1, s);
  if (ov) EDT_TRY(cudaStreamWaitEvent(s, c->ev_join, 0));
  prof_ev(c, 3, 0, s);
  if (mixed) EDT_TRY(launch_gram_scale(d, s, green_tables(c) != GREEN_G32DF));
  prof_ev(c, 3, 1, s);
  prof_ev(c, 4, 0, s);
  if (mixed) {
    EDT_TRY(launch_gram_tc(d, s));
    prof_ev(c, 4, 1, s);
    prof_ev(c, 5, 0, s);
    EDT_TRY(launch_gram_reduce(d, s, d.chol_df && !c->variant));
  } else {
    EDT_TRY(launch_gram_f64(d, s));
    prof_ev(c, 4, 1, s);
    prof_ev(c, 5, 0, s);
  }
  prof_ev(c, 5, 1, s);
  prof_ev(c, 6, 0, s);
  if (c->variant) EDT_TRY(launch_solve_variant(d, s));
  else {
    const CholLookahead la{c->aux, c->ev_la.data(), int(c->ev_la.size())};
    EDT_TRY(launch_chol_solve(d, mixed ? 1 : 0, s, &la));
  }
  prof_ev(c, 6, 1, s);
  prof_ev(c, 7, 0, s);
  if (mixed) {
    for (int it = 0; it < c->cfg.refine; ++it) {
      EDT_TRY(launch_refine(d, s));
      EDT_TRY(launch_refine_update(d, s));
    }
  }
  prof_ev(c, 7, 1, s);
  prof_ev(c, 8, 0, s);
  if (!do_inverse) {
  } else if (c->win) {
    EDT_TRY(launch_fa_inverse(d, V, V_dtype, s));
  } else {
    EDT_TRY(launch_inverse(d, V, V_dtype, s));
  }
  prof_ev(c, 8, 1, s);
  if (c->prof && c->prof_calls < kProfCalls) c->prof_calls++;
  return EDT_OK;
}

}  // namespace

extern "C" {

int edt_create(edt_ctx** out, const edt_config* cfg, size_t* workspace_bytes) {
  if (!out) return EDT_EINVAL;
  *out = nullptr;
  int v = validate(cfg);
  if (v != EDT_OK) return v;
  edt_ctx* c = new (std::nothrow) edt_ctx();
  if (!c) return EDT_EINVAL;
  c->cfg = *cfg;
  c->freq.assign(cfg->freq_hz, cfg->freq_hz + cfg->nfreq);
  c->tops.assign(cfg->layer_top_m, cfg->layer_top_m + cfg->nlayer);
  c->vel.assign(cfg->layer_vel_mps, cfg->layer_vel_mps + cfg->nlayer);
  c->cfg.freq_hz = c->freq.data();
  c->cfg.layer_top_m = c->tops.data();
  c->cfg.layer_vel_mps = c->vel.data();
  if (c->cfg.precision == EDT_FP64) { c->cfg.passes = 0; c->cfg.refine = 0; }
  // refinement residual: double-float on the line geometry when asked, or automatically
  // when the damping is weak enough for FP32 rounding in the residual to show
  c->win = c->cfg.geometry == EDT_GEOM_WINDOW;
  c->resid_df = c->cfg.precision == EDT_MIXED && !c->win && c->cfg.refine > 0 &&
                (c->cfg.resid == 2 || (c->cfg.resid == 0 && c->cfg.alpha < kResidDfAlpha));
  plan(c);
  layout(c);
  if (workspace_bytes) *workspace_bytes = c->ws_bytes;
  *out = c;
  return EDT_OK;
}

int edt_set_workspace(edt_ctx* c, void* ws, size_t bytes) {
  if (c) c->have_factor = false;
  if (!c || !ws) return EDT_EINVAL;
  if (bytes < c->ws_bytes) return EDT_ENOMEM_WS;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return EDT_EINVAL;
  c->ws = ws;
  bind(c);
  std::vector<double> zo(c->z_off);
  EDT_TRYI(upload(c, c->r_fc, c->fc));
  EDT_TRYI(upload(c, c->r_ltop, c->tops));
  EDT_TRYI(upload(c, c->r_lvel, c->vel));
  EDT_TRYI(upload(c, c->r_zl, c->z_layer));
  EDT_TRYI(upload(c, c->r_zo, zo));
  EDT_TRYI(upload(c, c->r_zo32, c->z_off32));
  EDT_TRYI(upload(c, c->r_fc32, c->fc32));
  EDT_TRYI(upload(c, c->r_rows, c->rows));
  if (!c->tref.empty()) EDT_TRYI(upload(c, c->r_tref, c->tref));
  if (!c->tref_off.empty()) EDT_TRYI(upload(c, c->r_treoff, c->tref_off));
  EDT_TRYI(upload(c, c->r_roff, c->row_off));
  EDT_TRYI(upload(c, c->r_roffmf, c->row_off_mf));
  EDT_TRYI(upload(c, c->r_band, c->band));
  if (!c->bcol.empty()) EDT_TRYI(upload(c, c->r_bcol, c->bcol));
  if (!c->cpre.empty()) EDT_TRYI(upload(c, c->r_cpre, c->cpre));
  EDT_TRYI(upload(c, c->r_kval, c->kval));
  EDT_TRYI(upload(c, c->r_pairm, c->pair_m));
  EDT_TRYI(upload(c, c->r_fjoff, c->fj_off));
  EDT_TRYI(upload(c, c->r_fjent, c->fj_ent));
  EDT_TRYI(upload(c, c->r_jact, c->jact));
  EDT_TRYI(upload(c, c->r_jmap, c->jmap));
  EDT_TRYI(upload(c, c->r_tw64, c->tw64));
  EDT_TRYI(upload(c, c->r_tw32, c->tw32));
  EDT_TRYI(upload(c, c->r_segm, c->seg_m));
  EDT_TRYI(upload(c, c->r_segr0, c->seg_row0));
  EDT_TRYI(upload(c, c->r_segn, c->seg_nrow));
  EDT_TRYI(upload(c, c->r_ctas, c->cta_seg0));
  EDT_TRYI(upload(c, c->r_mslot, c->m_slot0));
  EDT_TRY(cudaMemset(at<void*>(c, c->r_status), 0, c->r_status.bytes));
  EDT_TRY(cudaMemset(at<void*>(c, c->r_flags), 0, c->r_flags.bytes));
  EDT_TRY(cudaMemset(at<void*>(c, c->r_x), 0, c->r_x.bytes));
  if (c->r_g32.bytes) EDT_TRY(cudaMemset(at<void*>(c, c->r_g32), 0, c->r_g32.bytes));
  if (c->r_g32lo.bytes) EDT_TRY(cudaMemset(at<void*>(c, c->r_g32lo), 0, c->r_g32lo.bytes));
  if (c->r_gent.bytes) {
    EDT_TRY(cudaMemset(at<void*>(c, c->r_gent), 0, c->r_gent.bytes));
    EDT_TRY(cudaMemset(at<void*>(c, c->r_rhs), 0, c->r_rhs.bytes));
    if (c->win) {
      EDT_TRY(cudaMemset(at<void*>(c, c->r_A32), 0, c->r_A32.bytes));
      EDT_TRY(launch_fa_setup(c->dev, (long long)c->rows.size(), nullptr));
    } else if (!c->rows.empty()) {
      EDT_TRY(launch_gent_static(c->dev, nullptr));
    }
  }
  if (!c->kz_P.empty()) {
    EDT_TRYI(upload(c, c->r_kzP, c->kz_P));
    EDT_TRYI(upload(c, c->r_kzp, c->kz_p));
    EDT_TRYI(upload(c, c->r_kzgoff, c->kz_goff));
    EDT_TRYI(upload(c, c->r_kzvoff, c->kz_voff));
    EDT_TRY(prepare_chol_var(c->nz));
  }
  if (c->variant) EDT_TRY(prepare_variants(c->nz));
  EDT_TRY(prepare_fft(c->dev));
  EDT_TRY(prepare_grad(c->dev));
  EDT_TRY(prepare_chol(c->dev));
  if (c->cfg.precision == EDT_MIXED) EDT_TRY(prepare_gram_tc(c->dev));
  if (c->band_mode) EDT_TRY(prepare_band(c->dev));
  if (c->win) EDT_TRY(prepare_fa(c->dev));
  if (!c->aux) {
    EDT_TRY(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
    EDT_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    EDT_TRY(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    EDT_TRY(cudaStreamCreateWithFlags(&c->cpy, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      EDT_TRY(cudaEventCreateWithFlags(&c->ev_in[i], cudaEventDisableTiming));
      EDT_TRY(cudaEventCreateWithFlags(&c->ev_free[i], cudaEventDisableTiming));
    }
    c->ev_la.assign(2 * ((c->nz + 31) / 32) + 1, nullptr);
    for (auto& e : c->ev_la) EDT_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  EDT_TRY(cudaDeviceSynchronize());
  return EDT_OK;
}

static void drop_graph(edt_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
}

// Make the context's launch shapes current: re-plan the band chunks (line geometry), rebind
// and re-upload the band tables, forget a captured graph.
static int apply_tuning(edt_ctx* c) {
  drop_graph(c);
  if (c->band_mode) {
    const double cmin = *std::min_element(c->vel.begin(), c->vel.end());
    plan_band(c, cmin);
  }
  if (!c->ws) return EDT_OK;
  bind(c);
  if (c->band_mode) {
    EDT_TRYI(upload(c, c->r_band, c->band));
    if (!c->bcol.empty()) EDT_TRYI(upload(c, c->r_bcol, c->bcol));
    if (!c->cpre.empty()) EDT_TRYI(upload(c, c->r_cpre, c->cpre));
  }
  return EDT_OK;
}

static bool valid_tuning(const edt_tuning* t) {
  const bool mb = t->band_budget_mb == 16 || t->band_budget_mb == 32 || t->band_budget_mb == 48 ||
                  t->band_budget_mb == 96;
  const bool bc = t->band_cols == 4 || t->band_cols == 8 || t->band_cols == 16;
  const bool rf = t->refine_shape >= 0 && t->refine_shape <= 3;
  const bool zc = t->window_ztile == 2 || t->window_ztile == 4 || t->window_ztile == 8;
  const bool ov = t->overlap == 0 || t->overlap == 1;
  return mb && bc && rf && zc && ov;
}

int edt_invert(edt_ctx* c, const void* D, int D_dtype, void* V, int V_dtype, void* stream) {
  if (!c || !D || !V) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (D_dtype != EDT_C64 && D_dtype != EDT_C128) return EDT_EINVAL;
  if (V_dtype != EDT_F32 && V_dtype != EDT_F64) return EDT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int r;
  if (c->use_graph && !c->prof && s != nullptr) {
    // one captured graph of every stage, replayed while the call's arguments stay the same
    if (!c->gexec || c->g_D != D || c->g_V != V || c->g_Dt != D_dtype || c->g_Vt != V_dtype || c->g_s != s) {
      drop_graph(c);
      cudaGraph_t g = nullptr;
      EDT_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      r = run_invert(c, D, D_dtype, V, V_dtype, s);
      cudaError_t e = cudaStreamEndCapture(s, &g);
      if (r != EDT_OK) { if (g) cudaGraphDestroy(g); c->last_status = r; return r; }
      if (e != cudaSuccess) return cuda_fail(e);
      e = cudaGraphInstantiate(&c->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { c->gexec = nullptr; return cuda_fail(e); }
      c->g_D = D; c->g_V = V; c->g_Dt = D_dtype; c->g_Vt = V_dtype; c->g_s = s;
    }
    c->last_stream = s;
    cudaError_t e = cudaGraphLaunch(c->gexec, s);
    r = e == cudaSuccess ? EDT_OK : cuda_fail(e);
  } else {
    r = run_invert(c, D, D_dtype, V, V_dtype, s);
  }
  c->last_status = r;
  c->have_factor = r == EDT_OK;
  return r;
}

int edt_invert_vjp(edt_ctx* c, const void* Vbar, int Vbar_dtype, void* Dbar, int Dbar_dtype, double* gc,
                   void* stream) {
  if (!c || !Vbar || (!Dbar && !gc)) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (Dbar && Dbar_dtype != EDT_C64 && Dbar_dtype != EDT_C128) return EDT_EINVAL;
  if (Vbar_dtype != EDT_F32 && Vbar_dtype != EDT_F64) return EDT_EINVAL;
  if (c->win || c->cfg.precision != EDT_MIXED) return EDT_EUNSUPPORTED;
  if (gc && (!grad_supported(c->dev) || !c->dev.tref)) return EDT_EUNSUPPORTED;
  if (!c->have_factor) return EDT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  EDT_TRY(launch_invert_vjp(c->dev, Vbar, Vbar_dtype, Dbar, Dbar_dtype, gc, c->cfg.refine, s));
  c->have_factor = true;                  // the factors, tables and right-hand sides are untouched
  return EDT_OK;
}

int edt_invert_adjoint(edt_ctx* c, const void* Vbar, int Vbar_dtype, void* Dbar, int Dbar_dtype, void* stream) {
  if (!Dbar) return EDT_EINVAL;
  return edt_invert_vjp(c, Vbar, Vbar_dtype, Dbar, Dbar_dtype, nullptr, stream);
}

int edt_get_tuning(const edt_ctx* c, edt_tuning* o) {
  if (!c || !o) return EDT_EINVAL;
  o->band_budget_mb = c->band_budget_mb;
  o->band_cols = c->tune_bc;
  o->refine_shape = c->tune_rf;
  o->window_ztile = c->tune_zc;
  o->overlap = c->tune_ov;
  o->invert_ms = c->tuned_ms;
  return EDT_OK;
}

int edt_set_tuning(edt_ctx* c, const edt_tuning* t) {
  if (!c || !t || !valid_tuning(t)) return EDT_EINVAL;
  c->band_budget_mb = t->band_budget_mb;
  c->tune_bc = t->band_cols;
  c->tune_rf = t->refine_shape;
  c->tune_zc = t->window_ztile;
  c->tune_ov = t->overlap;
  return apply_tuning(c);
}

int edt_autotune(edt_ctx* c, const void* D, int D_dtype, void* V, int V_dtype, void* stream, int reps) {
  if (!c || !D || !V || reps < 1) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (D_dtype != EDT_C64 && D_dtype != EDT_C128) return EDT_EINVAL;
  if (V_dtype != EDT_F32 && V_dtype != EDT_F64) return EDT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool mixed = c->cfg.precision == EDT_MIXED;
  cudaEvent_t e0, e1;
  EDT_TRY(cudaEventCreate(&e0));
  EDT_TRY(cudaEventCreate(&e1));
  // steady-state time of one inversion: a warm-up call, then reps calls back to back between
  // two events (what a caller inverting line after line sees; isolated calls each start on an
  // idle device and rank some launch shapes differently)
  auto time_invert = [&](double* per_call) -> int {
    int rc = run_invert(c, D, D_dtype, V, V_dtype, s);
    if (rc != EDT_OK) return rc;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r)
      if ((rc = run_invert(c, D, D_dtype, V, V_dtype, s)) != EDT_OK) return rc;
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return cuda_fail(e);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *per_call = double(ms) / reps;
    return EDT_OK;
  };
  edt_tuning cur;
  edt_get_tuning(c, &cur);
  int rc = apply_tuning(c);
  double best = 0.0;
  if (rc == EDT_OK) rc = time_invert(&best);
  // one coordinate at a time; candidates that do not apply to this geometry are skipped
  struct Axis { int* field; std::vector<int> cand; bool on; };
  std::vector<Axis> axes = {
      {&cur.band_budget_mb, {16, 32, 48, 96}, c->band_mode},
      {&cur.band_cols, {4, 8, 16}, c->band_mode},
      {&cur.refine_shape, {0, 1, 2, 3}, mixed && c->cfg.refine > 0},
      {&cur.window_ztile, {2, 4, 8}, c->win},
      {&cur.overlap, {0, 1}, true},
  };
  for (Axis& a : axes) {
    if (rc != EDT_OK || !a.on) continue;
    const int keep = *a.field;
    int pick = keep;
    for (int v : a.cand) {
      if (v == keep) continue;
      *a.field = v;
      if ((rc = edt_set_tuning(c, &cur)) != EDT_OK) break;
      double ms = 0.0;
      if ((rc = time_invert(&ms)) != EDT_OK) break;
      if (ms < best) { best = ms; pick = v; }
    }
    *a.field = pick;
    if (rc == EDT_OK) rc = edt_set_tuning(c, &cur);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != EDT_OK) return rc;
  c->tuned_ms = best;
  c->last_stream = s;
  return run_invert(c, D, D_dtype, V, V_dtype, s);
}

int edt_set_graph(edt_ctx* c, int on) {
  if (!c) return EDT_EINVAL;
  c->use_graph = on != 0;
  drop_graph(c);
  return EDT_OK;
}

int edt_invert_host(edt_ctx* c, const void* D_host, int D_dtype, void* V_host, int V_dtype,
                    void* stream) {
  if (!c || !D_host || !V_host) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (D_dtype != EDT_C64 && D_dtype != EDT_C128) return EDT_EINVAL;
  if (V_dtype != EDT_F32 && V_dtype != EDT_F64) return EDT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t dbytes = size_t(c->nf) * (c->win ? size_t(c->nxy) * c->W : size_t(c->N) * c->N) *
                        (D_dtype == EDT_C64 ? 8 : 16);
  const size_t vbytes = size_t(c->win ? c->nxy : c->N) * c->nz * (V_dtype == EDT_F32 ? 4 : 8);
  c->last_stream = s;
  int r;
  if (!c->host_pipe) {
    EDT_TRY(cudaMemcpyAsync(c->dev.Dstage, D_host, dbytes, cudaMemcpyHostToDevice, s));
    r = run_invert(c, c->dev.Dstage, D_dtype, c->dev.Vstage, V_dtype, s);
  } else {
    // the copy waits only for the last call that read this staging buffer, not for earlier
    // work on `stream`; the stages wait for the copy
    const int b = c->host_buf;
    c->host_buf ^= 1;
    void* Dst = static_cast<char*>(c->dev.Dstage) + size_t(b) * c->dst_half;
    EDT_TRY(cudaStreamWaitEvent(c->cpy, c->ev_free[b], 0));
    EDT_TRY(cudaMemcpyAsync(Dst, D_host, dbytes, cudaMemcpyHostToDevice, c->cpy));
    EDT_TRY(cudaEventRecord(c->ev_in[b], c->cpy));
    EDT_TRY(cudaStreamWaitEvent(s, c->ev_in[b], 0));
    r = run_invert(c, Dst, D_dtype, c->dev.Vstage, V_dtype, s);
    if (r == EDT_OK) EDT_TRY(cudaEventRecord(c->ev_free[b], s));
  }
  c->last_status = r;
  c->have_factor = r == EDT_OK;
  if (r != EDT_OK) return r;
  EDT_TRY(cudaMemcpyAsync(V_host, c->dev.Vstage, vbytes, cudaMemcpyDeviceToHost, s));
  return EDT_OK;
}

int edt_set_host_pipeline(edt_ctx* c, int on) {
  if (!c) return EDT_EINVAL;
  c->host_pipe = on != 0;
  return EDT_OK;
}

int edt_forward(edt_ctx* c, const void* V, int V_dtype, void* D, int D_dtype, void* stream) {
  if (!c || !D || !V) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (D_dtype != EDT_C64 && D_dtype != EDT_C128) return EDT_EINVAL;
  if (V_dtype != EDT_F32 && V_dtype != EDT_F64) return EDT_EINVAL;
  if (c->win) return EDT_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  EDT_TRY(launch_green(c->dev, s, GREEN_G64));
  EDT_TRY(launch_forward(c->dev, V, V_dtype, D, D_dtype, s));
  return EDT_OK;
}

int edt_adjoint(edt_ctx* c, const void* D, int D_dtype, void* V, int V_dtype, void* stream) {
  if (!c || !D || !V) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (D_dtype != EDT_C64 && D_dtype != EDT_C128) return EDT_EINVAL;
  if (V_dtype != EDT_F32 && V_dtype != EDT_F64) return EDT_EINVAL;
  if (c->win) return EDT_EUNSUPPORTED;
  if (c->cfg.precision == EDT_MIXED && !grad_supported(c->dev)) return EDT_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  EDT_TRY(launch_green(c->dev, s, c->cfg.precision == EDT_MIXED ? GREEN_G32 : GREEN_G64));
  EDT_TRY(launch_adjoint(c->dev, D, D_dtype, V, V_dtype, s));
  return EDT_OK;
}

int edt_misfit_grad(edt_ctx* c, const void* V, int V_dtype, const void* D, int D_dtype,
                    double* J, void* gV, double* gc, void* stream) {
  if (!c || !V || !D || !J || !gV || !gc) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (D_dtype != EDT_C64 && D_dtype != EDT_C128) return EDT_EINVAL;
  if (V_dtype != EDT_F32 && V_dtype != EDT_F64) return EDT_EINVAL;
  if (!grad_supported(c->dev)) return EDT_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  EDT_TRY(launch_green(c->dev, s, GREEN_G32));
  EDT_TRY(launch_misfit_grad(c->dev, V, V_dtype, D, D_dtype, J, gV, gc, s));
  return EDT_OK;
}

int edt_set_reference(edt_ctx* c, const double* vel, void* stream) {
  if (!c || !vel) return EDT_EINVAL;
  for (int l = 0; l < c->nlayer; ++l)
    if (!(vel[l] > 0.0) || !std::isfinite(vel[l])) return EDT_EINVAL;
  if (c->cfg.cutoff > 0.0) {
    // the row plan (the evanescent cut) was made for the slowest velocity
    const double cmin_old = *std::min_element(c->vel.begin(), c->vel.end());
    const double cmin_new = *std::min_element(vel, vel + c->nlayer);
    if (cmin_new != cmin_old) return EDT_EINVAL;
  }
  std::copy(vel, vel + c->nlayer, c->vel.begin());
  c->have_factor = false;                 // the factors belong to the old reference
  if (c->ws) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    EDT_TRY(cudaMemcpyAsync(at<void*>(c, c->r_lvel), c->vel.data(), c->nlayer * sizeof(double),
                            cudaMemcpyHostToDevice, s));
  }
  return EDT_OK;
}

int edt_green(edt_ctx* c, void* g_dev, void* stream) {
  if (!c || !g_dev) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  EDT_TRY(launch_green(c->dev, s, GREEN_G64));
  EDT_TRY(cudaMemcpyAsync(g_dev, c->dev.g64, c->r_g64.bytes, cudaMemcpyDeviceToDevice, s));
  return EDT_OK;
}

int edt_row_offsets(const edt_ctx* c, long long* off) {
  if (!c || !off) return EDT_EINVAL;
  std::copy(c->row_off.begin(), c->row_off.end(), off);
  return c->nsub + 1;
}

static size_t rhs_row_bytes(const edt_ctx* c) {
  return 2 * (c->cfg.precision == EDT_MIXED ? sizeof(float2) : sizeof(double2));
}

int edt_export_rhs(edt_ctx* c, const void* D, int D_dtype, void* rhs_out, void* stream) {
  if (!c || !D || !rhs_out) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (D_dtype != EDT_C64 && D_dtype != EDT_C128) return EDT_EINVAL;
  if (c->win || c->variant) return EDT_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  c->have_factor = false;
  EDT_TRYI(transform_rhs(c, D, D_dtype, s));
  const size_t bytes = size_t(c->row_off[c->nsub]) * rhs_row_bytes(c);
  if (bytes) EDT_TRY(cudaMemcpyAsync(rhs_out, c->dev.rhs, bytes, cudaMemcpyDeviceToDevice, s));
  return EDT_OK;
}

int edt_import_rhs(edt_ctx* c, const void* block, long long nrows, int f_begin, int f_end,
                   void* stream) {
  if (!c || nrows < 0) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (f_begin < 0 || f_end < f_begin || f_end > c->nf) return EDT_EINVAL;
  if (c->win || c->variant) return EDT_EUNSUPPORTED;
  // the block must hold exactly this context's rows of those frequencies
  long long want = 0;
  for (int m = 0; m < c->nsub; ++m)
    want += c->row_off_mf[size_t(m) * (c->nf + 1) + f_end] - c->row_off_mf[size_t(m) * (c->nf + 1) + f_begin];
  if (nrows != want || (want > 0 && !block)) return EDT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  c->have_factor = false;
  const size_t rb = rhs_row_bytes(c);
  const char* src = static_cast<const char*>(block);
  char* dst = static_cast<char*>(c->dev.rhs);
  long long so = 0;
  for (int m = 0; m < c->nsub; ++m) {
    const long long a = c->row_off_mf[size_t(m) * (c->nf + 1) + f_begin];
    const long long b = c->row_off_mf[size_t(m) * (c->nf + 1) + f_end];
    if (b > a)
      EDT_TRY(cudaMemcpyAsync(dst + size_t(a) * rb, src + size_t(so) * rb, size_t(b - a) * rb,
                              cudaMemcpyDeviceToDevice, s));
    so += b - a;
  }
  return EDT_OK;
}

int edt_solve_imported(edt_ctx* c, void* vhat_dev, void* stream) {
  if (!c || !vhat_dev) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (c->win || c->variant) return EDT_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int r = run_invert(c, nullptr, EDT_C64, nullptr, EDT_F64, s, false, false);
  c->last_status = r;
  if (r != EDT_OK) return r;
  c->have_factor = true;
  // the solutions x[m][z][0..1] are Vhat(k_m, z) = x_+ + i x_- in complex128 layout (x_- = 0 at
  // the self-paired m; zero for failed subproblems and those outside the context's range)
  EDT_TRY(cudaMemcpyAsync(vhat_dev, c->dev.x, c->r_x.bytes, cudaMemcpyDeviceToDevice, s));
  return EDT_OK;
}

int edt_inverse_vhat(edt_ctx* c, const void* vhat_dev, void* V_dev, int V_dtype, void* stream) {
  if (!c || !vhat_dev || !V_dev) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (V_dtype != EDT_F32 && V_dtype != EDT_F64) return EDT_EINVAL;
  if (c->win) return EDT_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  c->have_factor = false;
  EDT_TRY(cudaMemcpyAsync(c->dev.x, vhat_dev, c->r_x.bytes, cudaMemcpyDeviceToDevice, s));
  EDT_TRY(cudaMemsetAsync(c->dev.status, 0, sizeof(int) * c->nsub, s));
  EDT_TRY(launch_inverse(c->dev, V_dev, V_dtype, s));
  return EDT_OK;
}

int edt_get_factor(edt_ctx* c, void* L_dev, void* stream) {
  if (!c || !L_dev) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (!c->have_factor || c->variant) return EDT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (c->dev.chol_df) EDT_TRY(launch_chol_dfloat_export(c->dev, static_cast<double*>(L_dev), s));
  else EDT_TRY(cudaMemcpyAsync(L_dev, c->dev.G, c->r_G.bytes, cudaMemcpyDeviceToDevice, s));
  return EDT_OK;
}

int edt_get_vhat(edt_ctx* c, void* vhat_dev, void* stream) {
  if (!c || !vhat_dev) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  EDT_TRY(cudaMemcpyAsync(vhat_dev, c->dev.vhat, c->r_vhat.bytes, cudaMemcpyDeviceToDevice, s));
  return EDT_OK;
}

int edt_gram(edt_ctx* c, const void* D, int D_dtype, void* G, void* b, void* tr, void* stream) {
  if (c) c->have_factor = false;
  if (!c || !D || !G || !b || !tr) return EDT_EINVAL;
  if (!c->ws) return EDT_ENOMEM_WS;
  if (D_dtype != EDT_C64 && D_dtype != EDT_C128) return EDT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Dev& d = c->dev;
  const bool mixed = c->cfg.precision == EDT_MIXED;
  c->last_stream = s;
  EDT_TRY(launch_green(d, s, green_tables(c)));
  EDT_TRYI(kernel_rows(c, s));
  EDT_TRYI(transform_rhs(c, D, D_dtype, s));
  if (mixed) {
    EDT_TRY(launch_gram_scale(d, s, green_tables(c) != GREEN_G32DF));
    EDT_TRY(launch_gram_tc(d, s));
    EDT_TRY(launch_gram_reduce(d, s));
  } else {
    EDT_TRY(launch_gram_f64(d, s));
    EDT_TRY(launch_trace_diag(d, s));
  }
  EDT_TRY(cudaMemcpyAsync(G, d.G, c->r_G.bytes, cudaMemcpyDeviceToDevice, s));
  EDT_TRY(cudaMemcpyAsync(b, d.b, c->r_b.bytes, cudaMemcpyDeviceToDevice, s));
  EDT_TRY(cudaMemcpyAsync(tr, d.trace, c->r_tr.bytes, cudaMemcpyDeviceToDevice, s));
  return EDT_OK;
}

int edt_row_counts(const edt_ctx* c, long long* counts) {
  if (!c || !counts) return EDT_EINVAL;
  for (int m = 0; m < c->nsub; ++m) counts[m] = c->counts_cut[m];
  return EDT_OK;
}

int edt_kz_disk_columns(const edt_ctx* c, int* p) {
  if (!c || !p || c->kz_p.empty()) return EDT_EINVAL;
  for (int m = 0; m < c->nsub; ++m) p[m] = c->kz_p[m];
  return c->nsub;
}

int edt_get_stats(edt_ctx* c, edt_stats* o) {
  if (!c || !o) return EDT_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->n_sub = c->nsub;
  long long tot = 0;
  int mn = 0x7fffffff, mx = 0;
  for (long long v : c->counts_cut) { tot += v; mn = std::min<long long>(mn, v); mx = std::max<long long>(mx, v); }
  o->rows_total = tot;
  o->rows_solved = (long long)c->rows.size();
  o->rows_min = mn; o->rows_max = mx;
  o->workspace_bytes = c->ws_bytes;
  o->gram_flop = 2.0 * 2.0 * double(o->rows_solved) * double(c->nz) * double(c->nz + 2);
  o->last_status = c->last_status;
  // kernels launched by one edt_invert: green (3), per frequency chunk transform (2) and
  // right-hand sides (1), Gram (FP64: 1; mixed: tensor-core + reduce 2), batched Cholesky,
  // per refinement step (3: partial residuals, their ordered sum, the update), inverse (1)
  int tr_launches = c->fchunk > 0 ? 3 * ((c->nf + c->fchunk - 1) / c->fchunk) : 0;
  if (c->band_mode) {
    tr_launches = 0;
    for (const BandChunk& ch : c->bchunks) tr_launches += 1 + (ch.nbcol > 0) + (ch.nrow > 0);
  }
  const int chol_n = c->dev.chol_df ? chol_dfloat_launches(c->nz) : chol_launches(c->nz);
  o->launches_per_invert = (c->cfg.precision == EDT_MIXED ? 6 + 3 * c->cfg.refine : 5) + tr_launches +
                           chol_n + gram_scale_launches(c->dev, green_tables(c) != GREEN_G32DF);
  // solver variants replace the Cholesky launch: trace, two projections, the solve (Cholesky
  // or Jacobi), the back-projection with the disk; the Jacobi kernel alone without it
  if (c->variant) o->launches_per_invert += (c->kz_p.empty() ? 1 : 5) - chol_launches(c->nz);
  if (c->win) {
    // green (3), rows (3) per frequency that keeps any, data (2), Gram (2), Cholesky,
    // refinement (3 per step), inverse (completion, FP64 row and column transforms, output: 3 or 4)
    int fk = 0;
    for (int n : c->nact) fk += n > 0;
    o->launches_per_invert = 3 + 3 * fk + 2 + 2 + chol_n + 3 * c->cfg.refine +
                             (c->ny > 1 ? 4 : 3);
  }
  o->freq_chunk = c->band_mode ? c->band_maxplanes : c->fchunk;
  // misfit gradient: green (3), zero, lateral DFT, per chunk transform (2) and three
  // contractions, depth march forward / field / reversed (3), inverse lateral DFT, finalize
  o->launches_per_grad = grad_supported(c->dev) && c->fchunk > 0
                             ? 3 + 2 + 5 * ((c->nf + c->fchunk - 1) / c->fchunk) + 5 : 0;
  o->gram_rows_padded = 0;
  for (long long n : c->seg_nrow) o->gram_rows_padded += (n + TC_KC - 1) / TC_KC * TC_KC;
  if (c->ws) {
    cudaError_t e = cudaStreamSynchronize(c->last_stream);
    if (e != cudaSuccess) return cuda_fail(e);
    std::vector<int> st(c->nsub);
    e = cudaMemcpy(st.data(), c->dev.status, sizeof(int) * c->nsub, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int v : st) {
      if (v == EDT_ENOTPD) o->n_notpd++;
      if (v == EDT_ENONFINITE) o->n_nonfinite++;
    }
    unsigned fl = 0;
    e = cudaMemcpy(&fl, c->dev.flags, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    o->gram_timeouts = fl ? 1 : 0;
    if (fl) o->last_status = EDT_ETIMEOUT;
  }
  return EDT_OK;
}

int edt_set_wait_test(edt_ctx* c, long long wait_cycles, int stall) {
  if (!c || wait_cycles < 0 || (stall != 0 && stall != 1) || (stall && wait_cycles == 0)) return EDT_EINVAL;
  c->dev.wait_cycles = wait_cycles;
  c->dev.wait_stall = stall;
  return EDT_OK;
}

int edt_set_profiling(edt_ctx* c, int on) {
  if (!c) return EDT_EINVAL;
  if (on && c->ev.empty()) {
    c->ev.resize(size_t(kProfCalls) * edt_ctx::NSTAGE * 2);
    for (auto& e : c->ev) EDT_TRY(cudaEventCreate(&e));
  }
  c->prof = on != 0;
  c->prof_calls = 0;
  std::memset(c->prof_used, 0, sizeof(c->prof_used));
  return EDT_OK;
}

int edt_read_profile(edt_ctx* c, double* ms, const char** names, int max_stages, int* n_calls) {
  if (!c || !ms) return EDT_EINVAL;
  const int ns = std::min(max_stages, edt_ctx::NSTAGE);
  for (int i = 0; i < ns; ++i) { ms[i] = 0.0; if (names) names[i] = kStageNames[i]; }
  if (n_calls) *n_calls = c->prof_calls;
  if (c->prof_calls > 0) {
    const int K = edt_ctx::NSTAGE;
    // the last stage of the last call ends after every other event of that call
    EDT_TRY(cudaEventSynchronize(c->ev[(size_t(c->prof_calls - 1) * K + (K - 1)) * 2 + 1]));
    for (int call = 0; call < c->prof_calls; ++call)
      for (int i = 0; i < ns; ++i) {
        float t = 0.f;
        EDT_TRY(cudaEventElapsedTime(&t, c->ev[(size_t(call) * K + i) * 2], c->ev[(size_t(call) * K + i) * 2 + 1]));
        ms[i] += t;
      }
  }
  c->prof_calls = 0;
  return ns;
}

const char* edt_strerror(int code) {
  switch (code) {
    case EDT_OK: return "ok";
    case EDT_EINVAL: return "invalid argument";
    case EDT_ENOMEM_WS: return "workspace missing or too small";
    case EDT_ENOTPD: return "damped normal matrix not positive definite";
    case EDT_ETIMEOUT: return "bounded device wait expired";
    case EDT_ENONFINITE: return "non-finite value";
    case EDT_ECUDA: return "CUDA runtime error";
    case EDT_EUNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

const char* edt_last_cuda_error(void) { return g_last_cuda.c_str(); }

void edt_destroy(edt_ctx* c) {
  if (!c) return;
  drop_graph(c);
  for (auto& e : c->ev) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i) {
    if (c->ev_in[i]) cudaEventDestroy(c->ev_in[i]);
    if (c->ev_free[i]) cudaEventDestroy(c->ev_free[i]);
  }
  if (c->cpy) cudaStreamDestroy(c->cpy);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  for (auto e : c->ev_la) if (e) cudaEventDestroy(e);
  if (c->aux) cudaStreamDestroy(c->aux);
  delete c;
}

}  // extern "C"
