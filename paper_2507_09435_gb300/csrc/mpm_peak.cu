// Arithmetic-peak microbenchmark: the FP64 and FP32 fused multiply-add
// throughput of the current device, measured with CUDA events.  The residual
// and constitutive pass (FP64) and the assembly (FP32) are ALU-bound; their
// achieved rates are reported against these measured peaks.
//
// Each thread advances 8 independent FMA chains a = a * b + c (enough
// independent work to keep the FMA pipe busy), over a grid of 8 blocks of 256
// threads per SM; 2 flops per FMA.
#include <cuda_runtime.h>

#include "mpm.h"

namespace {

constexpr int PEAK_TPB = 256;
constexpr int PEAK_CHAINS = 8;

template <class T>
__global__ void __launch_bounds__(PEAK_TPB) k_fma_peak(T* sink, int iters, T b, T c) {
  T a[PEAK_CHAINS];
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  T s = (T)0;
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
  // never true for the inputs used; keeps the chains live
  if (s == (T)-1.2345e30) sink[0] = s;
}

template <class T>
mpm_status run_peak(double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPM_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MPM_ERR_CUDA;
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return MPM_ERR_OOM;
  const int blocks = sms * 8;
  const int iters = (sizeof(T) == 8) ? 4096 : 65536;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // warm-up, then the timed launch
  k_fma_peak<T><<<blocks, PEAK_TPB>>>(sink, iters / 16, (T)0.999999, (T)1e-7);
  cudaEventRecord(e0);
  k_fma_peak<T><<<blocks, PEAK_TPB>>>(sink, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess || !(ms > 0.0f)) return MPM_ERR_CUDA;
  const double flops = 2.0 * PEAK_CHAINS * (double)iters * blocks * PEAK_TPB;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return MPM_OK;
}

}  // namespace

extern "C" mpm_status mpm_fma_peak(int precision, double* tflops) {
  if (!tflops) return MPM_ERR_INVALID_ARG;
  if (precision == MPM_FP64) return run_peak<double>(tflops);
  if (precision == MPM_MIXED) return run_peak<float>(tflops);
  return MPM_ERR_INVALID_ARG;
}
