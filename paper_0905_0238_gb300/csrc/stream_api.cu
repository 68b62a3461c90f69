// Host side of the streaming 1D solver: request validation, the device-memory admission plan,
// the arena layout of a batch, pinned double-buffered staging, and the C ABI (edt_stream_*).
#include "edt_internal.h"
#include "stream_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <queue>
#include <vector>

namespace edt {

namespace {

int st_cuda_fail(cudaError_t e) { return record_cuda_error(e); }

constexpr size_t AL = 256;                       // array alignment inside an arena
constexpr size_t TILE_AL = 1024;                 // per-request tile alignment (bulk copies)
constexpr size_t FIXED_BYTES = 64 * 1024;        // per-batch tables and alignment slack

size_t al(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct ReqShape {
  int nz, nl, nf, nk, nrow, nzs, nzt, kst;
  long long fk;            // nf * nk
  size_t tile_bytes;       // kst * 2 * (nzt * 128 + 16) * 128
};

ReqShape shape_of(const edt_sub1d& s) {
  ReqShape r;
  r.nz = s.nz; r.nl = s.nlayer; r.nf = s.nfreq; r.nk = s.nk; r.nrow = s.nrow;
  r.nzs = (s.nz + 31) / 32 * 32;
  r.nzt = (s.nz + ST_TILE - 1) / ST_TILE;
  r.kst = (s.nrow + ST_KC - 1) / ST_KC;
  r.fk = (long long)s.nfreq * s.nk;
  r.tile_bytes = size_t(r.kst) * 2 * size_t(r.nzt * ST_TILE + ST_DROWS) * 128;
  return r;
}

// Device bytes of one request inside a batch (every per-request slice, plus its alignment).
size_t bytes_of(const ReqShape& r) {
  size_t b = 0;
  b += sizeof(StSub) + 8 * sizeof(long long) + sizeof(int) + 2 * sizeof(long long);
  b += size_t(r.nzt) * (r.nzt + 1) / 2 * sizeof(StItem);
  b += sizeof(double) * size_t(3 * r.nl + r.nf + r.nk);
  b += size_t(r.nrow) * (sizeof(int4) + 2 * sizeof(float4));        // rows, data, rotated data
  b += size_t(r.nz) * (sizeof(float4) + sizeof(int));               // depth tables
  b += size_t(r.fk) * r.nl * 8 * sizeof(float);                     // recursion coefficients
  b += size_t(r.fk) * r.nzs * sizeof(float2) + 32 * sizeof(float2); // Green's table (+ alignment)
  b += r.tile_bytes + TILE_AL;                                       // operand tiles
  b += size_t(r.nz) * r.nz * (sizeof(double) + sizeof(float));      // G, L32
  b += size_t(r.nz) * (sizeof(double) + sizeof(float) + 6 * sizeof(double));   // dinv(32), b, x, r
  b += sizeof(double) + sizeof(int);                                 // trace, status
  b += size_t(r.kst) * (4 * r.nzt + 1) * sizeof(double);            // trace parts
  b += size_t((r.nrow + ST_REFINE_ROWS - 1) / ST_REFINE_ROWS) * r.nz * 2 * sizeof(double);  // residual partials
  b += size_t(ST_MAX_NZ / 32) * (sizeof(int) + 2 * sizeof(long long));   // blocked-Cholesky step lists
  return al(b, 64);
}

int validate(const edt_sub1d& s) {
  if (s.nz < 1 || s.nz > ST_MAX_NZ) return EDT_EINVAL;
  if (!(s.dz > 0.0) || !(s.dx > 0.0) || !(s.eps >= 0.0) || !(s.alpha >= 0.0) || !std::isfinite(s.z0))
    return EDT_EINVAL;
  if (s.nlayer < 1 || s.nlayer > ST_MAX_LAYERS || !s.layer_top_m || !s.layer_vel_mps) return EDT_EINVAL;
  if (s.layer_top_m[0] != 0.0) return EDT_EINVAL;
  for (int j = 0; j < s.nlayer; ++j) {
    if (!(s.layer_vel_mps[j] > 0.0) || !std::isfinite(s.layer_vel_mps[j])) return EDT_EINVAL;
    if (j > 0 && !(s.layer_top_m[j] > s.layer_top_m[j - 1])) return EDT_EINVAL;
  }
  if (s.nfreq < 1 || !s.freq_hz || s.nk < 1 || !s.kval || s.nrow < 0) return EDT_EINVAL;
  if ((long long)s.nfreq * s.nk * s.nz >= (1ll << 31)) return EDT_EINVAL;
  for (int f = 0; f < s.nfreq; ++f)
    if (!(s.freq_hz[f] > 0.0) || !std::isfinite(s.freq_hz[f])) return EDT_EINVAL;
  for (int k = 0; k < s.nk; ++k)
    if (!(s.kval[k] >= 0.0) || !std::isfinite(s.kval[k])) return EDT_EINVAL;
  if (s.nrow > 0 && (!s.rows || !s.data)) return EDT_EINVAL;
  for (int i = 0; i < s.nrow; ++i) {
    const int* r = s.rows + 3 * size_t(i);
    if (r[0] < 0 || r[0] >= s.nfreq || r[1] < 0 || r[1] >= s.nk || r[2] < 0 || r[2] >= s.nk) return EDT_EINVAL;
  }
  return EDT_OK;
}

int plan_batches(int n, const long long* bytes, long long arena, int max_batch, int* batch_of) {
  if (n < 0 || !bytes || !batch_of || max_batch < 1 || arena <= 0) return EDT_EINVAL;
  const long long cap = arena - (long long)FIXED_BYTES;
  int nb = 0, cnt = 0;
  long long used = 0;
  for (int i = 0; i < n; ++i) {
    if (bytes[i] < 0) return EDT_EINVAL;
    if (bytes[i] > cap) return EDT_ENOMEM_WS;
    if (cnt > 0 && (cnt == max_batch || used + bytes[i] > cap)) { ++nb; cnt = 0; used = 0; }
    batch_of[i] = nb;
    used += bytes[i];
    ++cnt;
  }
  return n > 0 ? nb + 1 : 0;
}

// The workspace bytes that admit the largest request (nz = 512, nrow = 4096, 64 layers, and a
// Green's table of 64 frequencies x 600 wavenumbers) in each of the two arenas.
size_t min_workspace() {
  ReqShape r;
  r.nz = ST_MAX_NZ; r.nl = ST_MAX_LAYERS; r.nf = 64; r.nk = 600; r.nrow = 4096;
  r.nzs = ST_MAX_NZ; r.nzt = ST_MAX_NZ / ST_TILE; r.kst = 4096 / ST_KC; r.fk = 64 * 600;
  r.tile_bytes = size_t(r.kst) * 2 * size_t(r.nzt * ST_TILE + ST_DROWS) * 128;
  return 2 * al(bytes_of(r) + FIXED_BYTES + 4096, AL);
}

}  // namespace

}  // namespace edt

using namespace edt;

struct edt_stream {
  int max_batch = 0;
  int nsm = 0;
  cudaStream_t user = nullptr;       // caller's stream: every batch follows its prior work
  cudaEvent_t ev_user = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0, arena_bytes = 0;
  cudaEvent_t epoch = nullptr;
  bool have_epoch = false;
  struct Slot {
    void* pin_in = nullptr;
    size_t cap_in = 0;
    void* pin_out = nullptr;
    size_t cap_out = 0;
    cudaStream_t st = nullptr;       // the slot's own stream: consecutive batches overlap
    cudaEvent_t t0 = nullptr, t1 = nullptr, done = nullptr;
    cudaEvent_t kev[ST_NKERNEL + 1] = {};   // per-launch events (profiling on)
    bool profiled = false;
    long long batch = -1;            // batch occupying the slot (results not yet delivered)
  } slot[2];
  bool profiling = false;
  long long wait_cycles = 0;         // wait test (edt_stream_set_wait_test)
  int wait_stall = 0;
  std::vector<std::pair<double, double>> busy;   // [t0, t1] of delivered batches after the epoch
  double kernel_ms[ST_NKERNEL] = {};
  long long profiled_batches = 0;
  struct Batch {
    int slot = 0;
    int nreq = 0;
    long long nz_total = 0;
    double* vhat_user = nullptr;     // where this batch's Vhat go
    int* status_user = nullptr;
    size_t x_bytes = 0;              // output section: x [sum nz][2], then status [nreq], flags
    bool delivered = false;
    double done_ms = -1.0;
    int err = EDT_OK;
  };
  std::map<long long, Batch> batches;
  struct Ticket { std::vector<long long> batch_ids; };
  std::map<long long, Ticket> tickets;
  long long next_batch = 0, next_ticket = 1;
  edt_stream_stats stats{};
};

namespace {

// Copy a finished batch's results from pinned staging to the caller's arrays.
int deliver(edt_stream* s, long long id) {
  auto it = s->batches.find(id);
  if (it == s->batches.end()) return EDT_OK;
  auto& B = it->second;
  if (B.delivered) return B.err;
  auto& sl = s->slot[B.slot];
  cudaError_t e = cudaEventSynchronize(sl.done);
  if (e != cudaSuccess) { B.err = st_cuda_fail(e); B.delivered = true; sl.batch = -1; return B.err; }
  const char* out = static_cast<const char*>(sl.pin_out);
  std::memcpy(B.vhat_user, out, B.x_bytes);
  const int* st = reinterpret_cast<const int*>(out + B.x_bytes);
  const unsigned flags = *reinterpret_cast<const unsigned*>(out + B.x_bytes + al(sizeof(int) * B.nreq, 16));
  for (int i = 0; i < B.nreq; ++i) B.status_user[i] = flags ? EDT_ETIMEOUT : st[i];
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, sl.t0, sl.t1) == cudaSuccess) s->stats.compute_ms += ms;
  if (s->have_epoch && cudaEventElapsedTime(&ms, s->epoch, sl.done) == cudaSuccess) B.done_ms = ms;
  float a0 = 0.f, a1 = 0.f;
  if (s->have_epoch && cudaEventElapsedTime(&a0, s->epoch, sl.t0) == cudaSuccess &&
      cudaEventElapsedTime(&a1, s->epoch, sl.t1) == cudaSuccess)
    s->busy.push_back({double(a0), double(a1)});
  if (sl.profiled) {
    for (int i = 0; i < ST_NKERNEL; ++i)
      if (cudaEventElapsedTime(&ms, sl.kev[i], sl.kev[i + 1]) == cudaSuccess) s->kernel_ms[i] += ms;
    s->profiled_batches += 1;
    sl.profiled = false;
  }
  B.delivered = true;
  sl.batch = -1;
  return EDT_OK;
}

int grow_pinned(void** p, size_t* cap, size_t need) {
  if (*cap >= need) return EDT_OK;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  const size_t n = al(std::max(need, size_t(1) << 20) + need / 4, 4096);
  cudaError_t e = cudaHostAlloc(p, n, cudaHostAllocDefault);
  if (e != cudaSuccess) { *p = nullptr; return st_cuda_fail(e); }
  *cap = n;
  return EDT_OK;
}

// Lay out, pack and launch requests [i0, i1) of `subs` in slot k.
int run_batch(edt_stream* s, const edt_sub1d* subs, int i0, int i1, double* vhat_user, int* status_user,
              long long* batch_id) {
  const int n = i1 - i0;
  const int k = int(s->next_batch & 1);
  auto& sl = s->slot[k];
  if (sl.batch >= 0) {
    const int e = deliver(s, sl.batch);
    if (e == EDT_ECUDA) return e;
  }
  std::vector<ReqShape> sh(n);
  for (int i = 0; i < n; ++i) sh[i] = shape_of(subs[i0 + i]);

  // ---- Gram items (request, ti, tj >= ti), longest first onto the least-loaded CTA
  std::vector<std::pair<long long, StItem>> all;
  for (int i = 0; i < n; ++i) {
    if (sh[i].nrow == 0) continue;
    for (int ti = 0; ti < sh[i].nzt; ++ti)
      for (int tj = ti; tj < sh[i].nzt; ++tj) {
        const long long cost = (long long)sh[i].kst * ((tj == sh[i].nzt - 1 ? 144 : 128) + (ti == tj ? 0 : 64));
        all.push_back({cost, StItem{i, ti, tj, 0}});
      }
  }
  std::stable_sort(all.begin(), all.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  const int ncta = int(std::min<size_t>(size_t(s->nsm), all.size()));
  std::vector<std::vector<StItem>> per(ncta);
  {
    using E = std::pair<long long, int>;
    std::priority_queue<E, std::vector<E>, std::greater<E>> pq;
    for (int c = 0; c < ncta; ++c) pq.push({0, c});
    for (auto& a : all) {
      E t = pq.top();
      pq.pop();
      per[t.second].push_back(a.second);
      pq.push({t.first + a.first, t.second});
    }
  }

  // ---- arena layout: inputs (one host-to-device copy), device scratch, outputs (one copy back)
  size_t off = 0;
  auto take = [&](size_t bytes, size_t a = AL) { off = al(off, a); size_t o = off; off += bytes; return o; };
  long long n_dbl = 0, n_rows = 0, n_z = 0, n_coef = 0, n_g = 0, n_G = 0, n_tw = 0, n_rz = 0;
  size_t n_tile = 0;
  for (int i = 0; i < n; ++i) {
    n_dbl += 3 * sh[i].nl + sh[i].nf + sh[i].nk;
    n_rows += sh[i].nrow;
    n_z += sh[i].nz;
    n_coef += sh[i].fk * sh[i].nl * 8;
    n_g = (n_g + 31) / 32 * 32 + sh[i].fk * sh[i].nzs;
    n_tile = al(n_tile, TILE_AL) + sh[i].tile_bytes;
    n_G += (long long)sh[i].nz * sh[i].nz;
    n_tw += (long long)sh[i].kst * (4 * sh[i].nzt + 1);
    n_rz += (long long)((sh[i].nrow + ST_REFINE_ROWS - 1) / ST_REFINE_ROWS) * sh[i].nz;
  }
  const size_t o_sub = take(sizeof(StSub) * n);
  const size_t o_pre = take(sizeof(long long) * 7 * size_t(n + 1));
  const size_t o_subn = take(sizeof(int) * n);
  const size_t o_goff = take(sizeof(long long) * n);
  const size_t o_voff = take(sizeof(long long) * n);
  const size_t o_order = take(sizeof(int) * n);
  int nmax = 1;
  for (int i = 0; i < n; ++i) nmax = std::max(nmax, sh[i].nz);
  const int nb_cols = chol_block_cols();
  const int nstep = (nmax + nb_cols - 1) / nb_cols;
  const size_t o_cbact = take(sizeof(int) * size_t(nstep) * n);
  const size_t o_cbpre = take(sizeof(long long) * size_t(nstep) * (n + 1));
  const size_t o_cbcpre = take(sizeof(long long) * size_t(nstep) * (n + 1));
  const size_t o_items = take(sizeof(StItem) * std::max<size_t>(all.size(), 1));
  const size_t o_cta = take(sizeof(int) * (ncta + 1));
  const size_t o_dbl = take(sizeof(double) * n_dbl);
  const size_t o_rows = take(sizeof(int4) * n_rows);
  const size_t o_data = take(sizeof(float4) * n_rows);
  const size_t in_bytes = off;
  const size_t o_drot = take(sizeof(float4) * n_rows);
  const size_t o_zt = take(sizeof(float4) * n_z);
  const size_t o_zl = take(sizeof(int) * n_z);
  const size_t o_coef = take(sizeof(float) * n_coef);
  const size_t o_g = take(sizeof(float2) * n_g);
  const size_t o_tile = take(n_tile, TILE_AL);
  const size_t o_G = take(sizeof(double) * n_G);
  const size_t o_L32 = take(sizeof(float) * n_G);
  const size_t o_dinv = take(sizeof(double) * n_z);
  const size_t o_dinv32 = take(sizeof(float) * n_z);
  const size_t o_b = take(sizeof(double) * 2 * n_z);
  const size_t o_r = take(sizeof(double) * 2 * n_z);
  const size_t o_trace = take(sizeof(double) * n);
  const size_t o_twtr = take(sizeof(double) * std::max<long long>(n_tw, 1));
  const size_t o_rcp = take(sizeof(double) * 2 * std::max<long long>(n_rz, 1));
  const size_t x_bytes = sizeof(double) * 2 * size_t(n_z);
  const size_t o_x = take(x_bytes);                          // output section: x, status, flags
  const size_t o_status = o_x + x_bytes;
  const size_t o_flags = o_status + al(sizeof(int) * n, 16);
  off = o_flags + 16;
  const size_t out_bytes = off - o_x;
  if (off > s->arena_bytes) return EDT_ENOMEM_WS;

  int e = grow_pinned(&sl.pin_in, &sl.cap_in, in_bytes);
  if (e != EDT_OK) return e;
  e = grow_pinned(&sl.pin_out, &sl.cap_out, out_bytes);
  if (e != EDT_OK) return e;

  // ---- pack
  char* P = static_cast<char*>(sl.pin_in);
  StSub* sub = reinterpret_cast<StSub*>(P + o_sub);
  long long* pre = reinterpret_cast<long long*>(P + o_pre);
  long long *pre_z = pre, *pre_fk = pre + (n + 1), *pre_eb = pre + 2 * (n + 1), *pre_tw = pre + 3 * (n + 1),
            *pre_rc = pre + 4 * (n + 1), *row_off = pre + 5 * (n + 1), *pre_rz = pre + 6 * (n + 1);
  int* subn = reinterpret_cast<int*>(P + o_subn);
  long long* goff = reinterpret_cast<long long*>(P + o_goff);
  long long* voff = reinterpret_cast<long long*>(P + o_voff);
  int* order = reinterpret_cast<int*>(P + o_order);
  double* dbl = reinterpret_cast<double*>(P + o_dbl);
  int4* rows = reinterpret_cast<int4*>(P + o_rows);
  float* data = reinterpret_cast<float*>(P + o_data);
  long long c_dbl = 0, c_rows = 0, c_z = 0, c_coef = 0, c_g = 0, c_G = 0;
  size_t c_tile = 0;
  pre_z[0] = pre_fk[0] = pre_eb[0] = pre_tw[0] = pre_rc[0] = row_off[0] = pre_rz[0] = 0;
  for (int i = 0; i < n; ++i) {
    const edt_sub1d& q = subs[i0 + i];
    const ReqShape& r = sh[i];
    StSub S{};
    S.nz = r.nz; S.nl = r.nl; S.nf = r.nf; S.nk = r.nk; S.nrow = r.nrow;
    S.nzs = r.nzs; S.nzt = r.nzt; S.kst = r.kst;
    S.dz = q.dz; S.z0 = q.z0; S.eps = q.eps; S.dx = q.dx; S.alpha = q.alpha;
    S.eps2 = float(q.eps * q.eps); S.dzdx = float(q.dz / q.dx);
    S.o_lay = c_dbl;
    std::memcpy(dbl + c_dbl, q.layer_top_m, sizeof(double) * r.nl);
    std::memcpy(dbl + c_dbl + r.nl, q.layer_vel_mps, sizeof(double) * r.nl);
    for (int j = 0; j < r.nl; ++j) dbl[c_dbl + 2 * r.nl + j] = 1.0 / (q.layer_vel_mps[j] * q.layer_vel_mps[j]);
    c_dbl += 3 * r.nl;
    S.o_freq = c_dbl;
    std::memcpy(dbl + c_dbl, q.freq_hz, sizeof(double) * r.nf);
    c_dbl += r.nf;
    S.o_kval = c_dbl;
    std::memcpy(dbl + c_dbl, q.kval, sizeof(double) * r.nk);
    c_dbl += r.nk;
    S.o_row = c_rows;
    for (int j = 0; j < r.nrow; ++j)
      rows[c_rows + j] = make_int4(q.rows[3 * j], q.rows[3 * j + 1], q.rows[3 * j + 2], 0);
    if (r.nrow) std::memcpy(data + 4 * c_rows, q.data, sizeof(float) * 4 * size_t(r.nrow));
    c_rows += r.nrow;
    S.o_v = c_z;
    c_z += r.nz;
    S.o_coef = c_coef;
    c_coef += r.fk * r.nl * 8;
    c_g = (c_g + 31) / 32 * 32;
    S.o_g = c_g;
    c_g += r.fk * r.nzs;
    c_tile = al(c_tile, TILE_AL);
    S.o_tile = (long long)c_tile;
    c_tile += r.tile_bytes;
    S.o_G = c_G;
    c_G += (long long)r.nz * r.nz;
    sub[i] = S;
    subn[i] = r.nz; goff[i] = S.o_G; voff[i] = S.o_v;
    pre_z[i + 1] = pre_z[i] + r.nz;
    pre_fk[i + 1] = pre_fk[i] + r.fk;
    pre_eb[i + 1] = pre_eb[i] + (r.fk + 7) / 8;
    pre_tw[i + 1] = pre_tw[i] + (long long)r.kst * (4 * r.nzt + 1);
    pre_rc[i + 1] = pre_rc[i] + (r.nrow + ST_REFINE_ROWS - 1) / ST_REFINE_ROWS;
    pre_rz[i + 1] = pre_rz[i] + (long long)((r.nrow + ST_REFINE_ROWS - 1) / ST_REFINE_ROWS) * r.nz;
    row_off[i + 1] = row_off[i] + r.nrow;
  }
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order, order + n, [&](int a, int b) { return sh[a].nz > sh[b].nz; });
  // blocked Cholesky step lists: requests with rows and more than 32 k unknowns, largest first
  int* cbact = reinterpret_cast<int*>(P + o_cbact);
  long long* cbpre = reinterpret_cast<long long*>(P + o_cbpre);
  long long* cbcpre = reinterpret_cast<long long*>(P + o_cbcpre);
  std::vector<int> cb_nact(nstep, 0);
  std::vector<long long> cb_ntile(nstep, 0), cb_nchunk(nstep, 0);
  for (int k = 0; k < nstep; ++k) {
    int na = 0;
    long long* tp = cbpre + size_t(k) * (n + 1);
    long long* cp = cbcpre + size_t(k) * (n + 1);
    tp[0] = 0;
    cp[0] = 0;
    for (int ii = 0; ii < n; ++ii) {
      const int i = order[ii];
      if (sh[i].nrow == 0 || sh[i].nz <= k * nb_cols) continue;
      cbact[size_t(k) * n + na] = i;
      tp[na + 1] = tp[na] + chol_blocked_tiles(sh[i].nz, k * nb_cols);
      cp[na + 1] = cp[na] + chol_blocked_chunks(sh[i].nz, k * nb_cols);
      ++na;
    }
    cb_nact[k] = na;
    cb_ntile[k] = tp[na];
    cb_nchunk[k] = cp[na];
  }
  StItem* items = reinterpret_cast<StItem*>(P + o_items);
  int* cta0 = reinterpret_cast<int*>(P + o_cta);
  int ni = 0;
  for (int c = 0; c < ncta; ++c) {
    cta0[c] = ni;
    for (auto& it : per[c]) items[ni++] = it;
  }
  cta0[ncta] = ni;

  // ---- device view
  char* A = s->ws + size_t(k) * s->arena_bytes;
  StBatch b{};
  b.nreq = n; b.ncta = ncta;
  b.sub = reinterpret_cast<const StSub*>(A + o_sub);
  const long long* dpre = reinterpret_cast<const long long*>(A + o_pre);
  b.pre_z = dpre; b.pre_fk = dpre + (n + 1); b.pre_eb = dpre + 2 * (n + 1); b.pre_tw = dpre + 3 * (n + 1);
  b.pre_rc = dpre + 4 * (n + 1);
  b.pre_rz = dpre + 6 * (n + 1);
  b.row_off = const_cast<long long*>(dpre + 5 * (n + 1));
  b.items = reinterpret_cast<const StItem*>(A + o_items);
  b.cta_item0 = reinterpret_cast<const int*>(A + o_cta);
  b.dbl = reinterpret_cast<const double*>(A + o_dbl);
  b.rows = reinterpret_cast<const int4*>(A + o_rows);
  b.data = reinterpret_cast<const float4*>(A + o_data);
  b.drot = reinterpret_cast<float4*>(A + o_drot);
  b.zt = reinterpret_cast<float4*>(A + o_zt);
  b.zl = reinterpret_cast<int*>(A + o_zl);
  b.coef = reinterpret_cast<float*>(A + o_coef);
  b.g32 = reinterpret_cast<float2*>(A + o_g);
  b.tiles = reinterpret_cast<unsigned char*>(A + o_tile);
  b.G = reinterpret_cast<double*>(A + o_G);
  b.L32 = reinterpret_cast<float*>(A + o_L32);
  b.dinv = reinterpret_cast<double*>(A + o_dinv);
  b.dinv32 = reinterpret_cast<float*>(A + o_dinv32);
  b.b = reinterpret_cast<double*>(A + o_b);
  b.x = reinterpret_cast<double*>(A + o_x);
  b.r = reinterpret_cast<double*>(A + o_r);
  b.trace = reinterpret_cast<double*>(A + o_trace);
  b.twtr = reinterpret_cast<double*>(A + o_twtr);
  b.rcp = reinterpret_cast<double*>(A + o_rcp);
  b.status = reinterpret_cast<int*>(A + o_status);
  b.sub_n = reinterpret_cast<int*>(A + o_subn);
  b.sub_goff = reinterpret_cast<long long*>(A + o_goff);
  b.sub_voff = reinterpret_cast<long long*>(A + o_voff);
  b.sub_order = reinterpret_cast<int*>(A + o_order);
  b.flags = reinterpret_cast<unsigned int*>(A + o_flags);
  b.wait_cycles = s->wait_cycles;
  b.wait_stall = s->wait_stall;
  b.tot_z = pre_z[n]; b.tot_fk = pre_fk[n]; b.tot_eb = pre_eb[n]; b.tot_tw = pre_tw[n]; b.tot_rc = pre_rc[n];
  b.cb_nstep = nstep;
  b.cb_act = reinterpret_cast<const int*>(A + o_cbact);
  b.cb_tpre = reinterpret_cast<const long long*>(A + o_cbpre);
  b.cb_cpre = reinterpret_cast<const long long*>(A + o_cbcpre);
  b.cb_nact_host = cb_nact.data();
  b.cb_ntile_host = cb_ntile.data();
  b.cb_nchunk_host = cb_nchunk.data();
  int nlaunch = 1 + (b.tot_fk > 0) + (b.tot_eb > 0) + 2 * (b.tot_tw > 0) + (ncta > 0) + 1 + 2 * (b.tot_rc > 0) + 1;
  nlaunch += nstep > 0 && cb_nact[0] > 0;
  for (int k = 0; k < nstep; ++k)
    if (cb_nact[k] > 0) nlaunch += (cb_nchunk[k] > 0) + (cb_ntile[k] > 0);

  cudaError_t ce = cudaSuccess;
  if (s->profiling && s->slot[k ^ 1].batch >= 0)       // profiled batches run one at a time
    ce = cudaStreamWaitEvent(sl.st, s->slot[k ^ 1].done, 0);
  if (ce == cudaSuccess && s->user) {
    ce = cudaEventRecord(s->ev_user, s->user);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(sl.st, s->ev_user, 0);
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(A, P, in_bytes, cudaMemcpyHostToDevice, sl.st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(A + o_flags, 0, 16, sl.st);
  if (ce == cudaSuccess) ce = cudaEventRecord(sl.t0, sl.st);
  sl.profiled = s->profiling;
  if (ce == cudaSuccess) ce = launch_stream_batch(b, nmax, sl.st, s->profiling ? sl.kev : nullptr);
  if (ce == cudaSuccess) ce = cudaEventRecord(sl.t1, sl.st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(sl.pin_out, A + o_x, out_bytes, cudaMemcpyDeviceToHost, sl.st);
  if (ce == cudaSuccess) ce = cudaEventRecord(sl.done, sl.st);
  if (ce != cudaSuccess) return st_cuda_fail(ce);

  const long long id = s->next_batch++;
  edt_stream::Batch B;
  B.slot = k; B.nreq = n; B.nz_total = n_z;
  B.vhat_user = vhat_user; B.status_user = status_user; B.x_bytes = x_bytes;
  s->batches[id] = B;
  sl.batch = id;
  s->stats.requests += n;
  s->stats.batches += 1;
  s->stats.launches += nlaunch;
  s->stats.launches_per_batch = std::max(s->stats.launches_per_batch, nlaunch);
  s->stats.bytes_in += (long long)in_bytes;
  s->stats.bytes_out += (long long)out_bytes;
  *batch_id = id;
  return EDT_OK;
}

}  // namespace

extern "C" {

long long edt_stream_request_bytes(const edt_sub1d* sub) {
  if (!sub || validate(*sub) != EDT_OK) return EDT_EINVAL;
  return (long long)bytes_of(shape_of(*sub));
}

int edt_stream_plan(int n, const long long* request_bytes, long long arena_bytes, int max_batch,
                    int* batch_of) {
  return plan_batches(n, request_bytes, arena_bytes, max_batch, batch_of);
}

int edt_stream_create(edt_stream** out, int max_batch, void* stream, size_t* workspace_min) {
  if (!out) return EDT_EINVAL;
  *out = nullptr;
  if (max_batch < 1 || max_batch > 4096) return EDT_EINVAL;
  auto* s = new edt_stream();
  s->max_batch = max_batch;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = prepare_stream();
  s->user = static_cast<cudaStream_t>(stream);
  if (e == cudaSuccess) e = cudaEventCreate(&s->epoch);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_user, cudaEventDisableTiming);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&s->slot[k].st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&s->slot[k].t0);
    if (e == cudaSuccess) e = cudaEventCreate(&s->slot[k].t1);
    if (e == cudaSuccess) e = cudaEventCreate(&s->slot[k].done);
    for (int i = 0; i <= ST_NKERNEL && e == cudaSuccess; ++i) e = cudaEventCreate(&s->slot[k].kev[i]);
  }
  if (e != cudaSuccess) {
    edt_stream_destroy(s);
    return st_cuda_fail(e);
  }
  s->stats.max_batch = max_batch;
  if (workspace_min) *workspace_min = min_workspace();
  *out = s;
  return EDT_OK;
}

int edt_stream_set_workspace(edt_stream* s, void* ws, size_t bytes) {
  if (!s || !ws || (reinterpret_cast<uintptr_t>(ws) & (AL - 1))) return EDT_EINVAL;
  if (bytes < min_workspace()) return EDT_ENOMEM_WS;
  for (int k = 0; k < 2; ++k)
    if (s->slot[k].batch >= 0) {
      const int e = deliver(s, s->slot[k].batch);
      if (e == EDT_ECUDA) return e;
    }
  s->ws = static_cast<char*>(ws);
  s->ws_bytes = bytes;
  s->arena_bytes = bytes / 2 / AL * AL;
  s->stats.arena_bytes = s->arena_bytes;
  return EDT_OK;
}

int edt_stream_submit(edt_stream* s, int n, const edt_sub1d* subs, double* vhat_host, int* status_host,
                      long long* ticket) {
  if (!s || n < 0 || (n > 0 && (!subs || !vhat_host || !status_host)) || !ticket) return EDT_EINVAL;
  if (!s->ws) return EDT_ENOMEM_WS;
  std::vector<long long> bytes(n);
  for (int i = 0; i < n; ++i) {
    const int v = validate(subs[i]);
    if (v != EDT_OK) return v;
    bytes[i] = (long long)bytes_of(shape_of(subs[i]));
  }
  std::vector<int> batch_of(n);
  const int nb = plan_batches(n, bytes.data(), (long long)s->arena_bytes, s->max_batch, batch_of.data());
  if (nb < 0) return nb;
  edt_stream::Ticket T;
  size_t vo = 0;
  int i0 = 0;
  while (i0 < n) {
    int i1 = i0;
    size_t nzs = 0;
    while (i1 < n && batch_of[i1] == batch_of[i0]) nzs += size_t(subs[i1++].nz);
    long long id = -1;
    const int e = run_batch(s, subs, i0, i1, vhat_host + 2 * vo, status_host + i0, &id);
    if (e != EDT_OK) return e;
    T.batch_ids.push_back(id);
    vo += nzs;
    i0 = i1;
  }
  const long long t = s->next_ticket++;
  s->tickets[t] = T;
  *ticket = t;
  return EDT_OK;
}

int edt_stream_wait(edt_stream* s, long long ticket, double* done_ms) {
  if (!s) return EDT_EINVAL;
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return EDT_EINVAL;
  int rc = EDT_OK;
  double last = -1.0;
  for (long long id : it->second.batch_ids) {
    const int e = deliver(s, id);
    if (e != EDT_OK && rc == EDT_OK) rc = e;
    auto b = s->batches.find(id);
    if (b != s->batches.end()) {
      last = std::max(last, b->second.done_ms);
      s->batches.erase(b);
    }
  }
  s->tickets.erase(it);
  if (done_ms) *done_ms = last;
  return rc;
}

int edt_stream_query(edt_stream* s, long long ticket, int* done) {
  if (!s || !done) return EDT_EINVAL;
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return EDT_EINVAL;
  *done = 1;
  for (long long id : it->second.batch_ids) {
    auto b = s->batches.find(id);
    if (b == s->batches.end() || b->second.delivered) continue;
    const cudaError_t e = cudaEventQuery(s->slot[b->second.slot].done);
    if (e == cudaErrorNotReady) { *done = 0; break; }
    if (e != cudaSuccess) return st_cuda_fail(e);
  }
  return EDT_OK;
}

int edt_stream_epoch(edt_stream* s) {
  if (!s) return EDT_EINVAL;
  cudaError_t e = cudaStreamSynchronize(s->slot[0].st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->slot[1].st);
  if (e == cudaSuccess) e = cudaEventRecord(s->epoch, s->slot[0].st);
  if (e == cudaSuccess) e = cudaEventSynchronize(s->epoch);
  if (e != cudaSuccess) return st_cuda_fail(e);
  s->have_epoch = true;
  s->busy.clear();
  return EDT_OK;
}

int edt_stream_get_stats(const edt_stream* s, edt_stream_stats* out) {
  if (!s || !out) return EDT_EINVAL;
  *out = s->stats;
  // device busy time: union of the [t0, t1] intervals of the batches delivered since the epoch
  std::vector<std::pair<double, double>> v = s->busy;
  std::sort(v.begin(), v.end());
  double busy = 0.0, a = -1.0, b = -1.0;
  for (auto& iv : v) {
    if (iv.first > b) {
      if (b > a) busy += b - a;
      a = iv.first;
      b = iv.second;
    } else {
      b = std::max(b, iv.second);
    }
  }
  if (b > a) busy += b - a;
  out->busy_ms = busy;
  return EDT_OK;
}

int edt_stream_set_profiling(edt_stream* s, int on) {
  if (!s) return EDT_EINVAL;
  s->profiling = on != 0;
  return EDT_OK;
}

int edt_stream_set_wait_test(edt_stream* s, long long wait_cycles, int stall) {
  if (!s || wait_cycles < 0 || (stall != 0 && stall != 1) || (stall && wait_cycles == 0)) return EDT_EINVAL;
  s->wait_cycles = wait_cycles;
  s->wait_stall = stall;
  return EDT_OK;
}

int edt_stream_read_profile(edt_stream* s, double* ms, const char** names, int max_kernels,
                            long long* n_batches) {
  if (!s || max_kernels < 0 || (max_kernels > 0 && (!ms || !names))) return EDT_EINVAL;
  for (int k = 0; k < 2; ++k)
    if (s->slot[k].batch >= 0) {
      const int e = deliver(s, s->slot[k].batch);
      if (e == EDT_ECUDA) return e;
    }
  const int n = std::min(max_kernels, ST_NKERNEL);
  for (int i = 0; i < n; ++i) {
    ms[i] = s->kernel_ms[i];
    names[i] = kStreamKernels[i];
  }
  if (n_batches) *n_batches = s->profiled_batches;
  for (double& v : s->kernel_ms) v = 0.0;
  s->profiled_batches = 0;
  return n;
}

void edt_stream_destroy(edt_stream* s) {
  if (!s) return;
  for (auto& sl : s->slot)
    if (sl.st) cudaStreamSynchronize(sl.st);
  for (auto& sl : s->slot) {
    if (sl.pin_in) cudaFreeHost(sl.pin_in);
    if (sl.pin_out) cudaFreeHost(sl.pin_out);
    if (sl.t0) cudaEventDestroy(sl.t0);
    if (sl.t1) cudaEventDestroy(sl.t1);
    if (sl.done) cudaEventDestroy(sl.done);
    for (auto& ev : sl.kev)
      if (ev) cudaEventDestroy(ev);
  }
  if (s->epoch) cudaEventDestroy(s->epoch);
  for (auto& sl : s->slot)
    if (sl.st) cudaStreamDestroy(sl.st);
  if (s->ev_user) cudaEventDestroy(s->ev_user);
  delete s;
}

}  // extern "C"
