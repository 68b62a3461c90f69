// Allocation-free entry point for the reference Green's-function table.
//
// Some callers cannot allocate device memory: code that runs while another component owns
// the device allocator (an embedded solver inside a host application with its own memory
// pool, a plugin that is handed only input and output buffers), or a caller that must not
// grow the device footprint after start-up.  edt_green_noalloc serves them: the caller
// passes its problem description in host arrays and one device output buffer, and the
// depth march runs with every scratch value (per-frequency constants, the layer stack,
// the per-(frequency, wavenumber, layer) recursion coefficients) held in one file-scope
// device array of fixed size instead of a workspace.  The frequencies are processed in
// chunks small enough for that array, so the table size is limited only by one frequency's
// coefficients having to fit.
#include "edt_internal.h"
#include "cplx.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

namespace edt {

namespace {

// Scratch of the allocation-free depth march.  Every GPU that loads the library holds
// these bytes until the process exits.  Calls share the array and overlap-free use is the
// caller's duty: two calls whose work overlaps on the GPU race on it.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (host code only knows a
// host-side stand-in for the symbol).  Looked up once per device and kept for the life of
// the process, so it does not survive a cudaDeviceReset of that device.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

}  // namespace edt

using namespace edt;

extern "C" int edt_green_noalloc(int nx, double dx, int nz, double dz, double z0, int nfreq,
                                 const double* freq_hz, double eps, int nlayer,
                                 const double* layer_top_m, const double* layer_vel_mps,
                                 void* g_dev, void* stream) {
  if (nx < 2 || (nx & (nx - 1)) || !(dx > 0) || nz < 1 || !(dz > 0) || !(z0 >= 0) || nfreq < 1 ||
      !freq_hz || !(eps >= 0) || nlayer < 1 || !layer_top_m || !layer_vel_mps || !g_dev)
    return EDT_EINVAL;
  if (layer_top_m[0] != 0.0) return EDT_EINVAL;
  for (int j = 0; j < nlayer; ++j) {
    if (!(layer_vel_mps[j] > 0) || !std::isfinite(layer_vel_mps[j])) return EDT_EINVAL;
    if (j > 0 && !(layer_top_m[j] > layer_top_m[j - 1])) return EDT_EINVAL;
  }
  for (int f = 0; f < nfreq; ++f)
    if (!(freq_hz[f] > 0) || !std::isfinite(freq_hz[f])) return EDT_EINVAL;
  const int nk = nx / 2 + 1;
  // scratch layout: [layer tops | layer velocities | depth layer | depth offset | freq
  // constants of one chunk | coefficients of one chunk]
  const size_t o_top = 0;
  const size_t o_vel = up256(o_top + sizeof(double) * nlayer);
  const size_t o_zl = up256(o_vel + sizeof(double) * nlayer);
  const size_t o_zo = up256(o_zl + sizeof(int) * nz);
  const size_t o_fc = up256(o_zo + sizeof(double) * nz);
  const size_t per_f_coef = size_t(nk) * nlayer * 7 * sizeof(double2);
  const size_t fixed = o_fc;
  if (fixed + up256(sizeof(FreqConst)) + per_f_coef > kNoAllocScratchBytes)
    return EDT_EUNSUPPORTED;   // one frequency's recursion coefficients exceed the 8 MiB scratch
  int chunk = int(std::min<size_t>(nfreq, (kNoAllocScratchBytes - fixed - 256) /
                                              (per_f_coef + sizeof(FreqConst))));
  while (chunk > 1 && fixed + up256(sizeof(FreqConst) * chunk) + per_f_coef * chunk > kNoAllocScratchBytes)
    --chunk;
  const size_t o_coef = up256(o_fc + sizeof(FreqConst) * chunk);

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The call stages host arrays that die when it returns (pageable copies), so it must
  // never be recorded into a graph: refuse it while its stream (or, for the legacy
  // stream, any global-mode capture) is capturing.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t ce = cudaStreamIsCapturing(s, &cs);
  if (ce == cudaErrorStreamCaptureImplicit) {
    (void)cudaGetLastError();
    return EDT_EINVAL;
  }
  if (ce != cudaSuccess) return record_cuda_error(ce);
  if (cs != cudaStreamCaptureStatusNone) return EDT_EINVAL;

  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return EDT_ECUDA;
  char* sb = static_cast<char*>(base);

  std::vector<int> zl(nz);
  std::vector<double> zo(nz);
  for (int j = 0; j < nz; ++j) {
    const double z = z0 + (j + 0.5) * dz;
    int l = int(std::upper_bound(layer_top_m, layer_top_m + nlayer, z) - layer_top_m) - 1;
    l = std::max(0, std::min(l, nlayer - 1));
    zl[j] = l;
    zo[j] = z - layer_top_m[l];
  }
  // pageable-host copies: each returns once the source has been consumed
  if (cudaMemcpyAsync(sb + o_top, layer_top_m, sizeof(double) * nlayer, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(sb + o_vel, layer_vel_mps, sizeof(double) * nlayer, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(sb + o_zl, zl.data(), sizeof(int) * nz, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(sb + o_zo, zo.data(), sizeof(double) * nz, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return EDT_ECUDA;

  Dev d{};
  d.N = nx; d.nk = nk; d.nz = nz; d.nzs = (nz + 1) & ~1; d.nlayer = nlayer; d.dx = dx; d.dz = dz;
  d.layer_top = reinterpret_cast<const double*>(sb + o_top);
  d.layer_vel = reinterpret_cast<const double*>(sb + o_vel);
  d.z_layer = reinterpret_cast<const int*>(sb + o_zl);
  d.z_off = reinterpret_cast<const double*>(sb + o_zo);
  d.fc = reinterpret_cast<const FreqConst*>(sb + o_fc);
  d.coef = reinterpret_cast<double2*>(sb + o_coef);
  d.g32 = nullptr;
  std::vector<FreqConst> fc(chunk);
  for (int f0 = 0; f0 < nfreq; f0 += chunk) {
    const int nf = std::min(chunk, nfreq - f0);
    for (int f = 0; f < nf; ++f) {
      FreqConst& q = fc[f];
      q.om_re = 2.0 * M_PI * freq_hz[f0 + f];
      q.om_im = eps;
      const double2 om = make_double2(q.om_re, q.om_im);
      double2 sv = om * om;
      sv = make_double2(sv.x * dz / dx, sv.y * dz / dx);
      q.s_abs = std::hypot(sv.x, sv.y);
      q.rot_re = sv.x / q.s_abs;
      q.rot_im = -sv.y / q.s_abs;
      q.lim = 0.0;
    }
    if (cudaMemcpyAsync(sb + o_fc, fc.data(), sizeof(FreqConst) * nf, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return EDT_ECUDA;
    d.nf = nf;
    d.g64 = static_cast<double2*>(g_dev) + size_t(f0) * nk * nz;
    if (launch_green(d, s, GREEN_G64) != cudaSuccess) return EDT_ECUDA;
  }
  return EDT_OK;
}
