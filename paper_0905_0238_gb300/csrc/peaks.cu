// Measured arithmetic peaks of the current GPU: FP64 and FP32 fused multiply-add throughput.
//
// The double-float factorisation and residual trade FP64 work for FP32 work; their roofline is
// stated against these two rates, measured here rather than taken from a data sheet (GB300
// runs FP64 at a small fraction of FP32).  Each thread runs eight independent multiply-add
// chains of 2048 steps (enough independent work to keep every pipe busy), over eight CTAs of
// 256 threads per SM; the rate is 2 flops per multiply-add over the CUDA-event time of the
// launch, the best of three.  The chains' results are stored so nothing is optimised away.
#include "edt_internal.h"

#include <algorithm>

namespace edt {

namespace {

constexpr int PK_CHAINS = 8, PK_STEPS = 2048, PK_THREADS = 256, PK_CTAS_PER_SM = 8;

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(PK_THREADS) fma_rate_kernel(T* out, T a, T b) {
  T c[PK_CHAINS];
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) c[k] = T(threadIdx.x + k);
  for (int s = 0; s < PK_STEPS; ++s) {
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) c[k] = fma_t(c[k], a, b);
  }
  T r = 0;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) r += c[k];
  out[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = r;
}

template <typename T>
cudaError_t time_rate(int nsm, T* out, double* tflops) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  const int grid = nsm * PK_CTAS_PER_SM;
  // a, b near 1 keep the chains finite
  fma_rate_kernel<T><<<grid, PK_THREADS>>>(out, T(0.999999), T(1e-7));       // warm-up
  double best = 0.0;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0);
    fma_rate_kernel<T><<<grid, PK_THREADS>>>(out, T(0.999999), T(1e-7));
    cudaEventRecord(e1);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flop = 2.0 * double(grid) * PK_THREADS * PK_CHAINS * PK_STEPS;
    if (ms > 0.f) best = std::max(best, flop / (double(ms) * 1e-3) / 1e12);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *tflops = best;
  return e;
}

}  // namespace

}  // namespace edt

using namespace edt;

extern "C" int edt_measure_fma_rates(double* fp64_tflops, double* fp32_tflops) {
  if (!fp64_tflops || !fp32_tflops) return EDT_EINVAL;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return record_cuda_error(e);
  const size_t n = size_t(nsm) * PK_CTAS_PER_SM * PK_THREADS;
  void* buf = nullptr;
  if ((e = cudaMalloc(&buf, n * sizeof(double))) != cudaSuccess) return record_cuda_error(e);
  e = time_rate<double>(nsm, static_cast<double*>(buf), fp64_tflops);
  if (e == cudaSuccess) e = time_rate<float>(nsm, static_cast<float*>(buf), fp32_tflops);
  cudaFree(buf);
  return e == cudaSuccess ? EDT_OK : record_cuda_error(e);
}
