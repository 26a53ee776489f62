// Measured compute ceilings for the roofline of the partition kernels: the
// rate of dependent-free fused multiply-adds per second in FP32 and FP64 on
// the current device, timed with CUDA events.  (Measurement only; the paper
// has no counterpart.)
#include <cuda_runtime.h>

#include "pma.h"

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(T *sink, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-12345.0) sink[threadIdx.x] = s;  // keeps the chains alive; never true
}

template <typename T>
int probe(double *fma_per_s, int *sm_count) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PMA_ERR_CUDA;
  T *sink = nullptr;
  if (cudaMalloc(&sink, kThreads * sizeof(T)) != cudaSuccess) return PMA_ERR_NOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = sms * 8;
  const int iters = sizeof(T) == 4 ? 4096 : 256;
  const T a = (T)0.999999, b = (T)1e-6;
  double best = 0.0;
  int rc = PMA_OK;
  for (int rep = 0; rep < 6 && rc == PMA_OK; ++rep) {
    cudaEventRecord(e0);
    fma_probe_kernel<T><<<grid, kThreads>>>(sink, iters, a, b);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = PMA_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double fmas = (double)grid * kThreads * kChains * iters;
    if (rep > 0 && ms > 0.f) best = fmas / (ms * 1e-3) > best ? fmas / (ms * 1e-3) : best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (rc == PMA_OK && cudaGetLastError() != cudaSuccess) rc = PMA_ERR_CUDA;
  *fma_per_s = best;
  if (sm_count) *sm_count = sms;
  return rc;
}

}  // namespace

extern "C" int pma_probe_fma(int precision, double *fma_per_s, int *sm_count) {
  if (!fma_per_s || (precision != PMA_FP64 && precision != PMA_MIXED)) return PMA_ERR_INVALID_ARG;
  return precision == PMA_FP64 ? probe<double>(fma_per_s, sm_count)
                               : probe<float>(fma_per_s, sm_count);
}
