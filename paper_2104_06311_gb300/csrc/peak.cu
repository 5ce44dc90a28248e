// Measured arithmetic peaks of the plain ALUs: the roofline denominators of the
// kernels bound by FP32 (or FP64) SIMT arithmetic rather than by HBM or the
// tensor pipe.  Every thread runs kChains independent fused multiply-add chains
// x <- x a + b (a < 1, so the values settle near b / (1 - a) and never overflow
// or turn subnormal); a grid of 8 CTAs of 256 threads per SM keeps every
// scheduler supplied with independent FMAs.  Not from the paper: measurement
// support for the per-stage rooflines.
#include <cuda_runtime.h>

#include "../../include/rx.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

__device__ double g_sink;   // written only if the chains produce an impossible value

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains(int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (T)(threadIdx.x & 7) + (T)j;
#pragma unroll 1
  for (int i = 0; i < iters; i += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == (T)-1234.5) g_sink = (double)s;   // keeps every chain live
}

template <typename T>
rx_status run(cudaStream_t st, int iters, double *tflops, double *ms) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RX_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RX_ECUDA;
  const int grid = sms * kCtasPerSm;
  const T a = (T)0.999999, b = (T)1e-6;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return RX_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RX_ECUDA;
  }
  fma_chains<T><<<grid, kThreads, 0, st>>>(iters, a, b);   // warm-up (clocks, instruction cache)
  cudaEventRecord(e0, st);
  fma_chains<T><<<grid, kThreads, 0, st>>>(iters, a, b);
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float t = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return RX_ECUDA;
  const double flop = 2.0 * (double)iters * kChains * (double)grid * kThreads;
  if (ms) *ms = t;
  if (tflops) *tflops = t > 0.f ? flop / (t * 1e-3) / 1e12 : 0.0;
  return RX_OK;
}

}  // namespace

extern "C" rx_status rx_measure_alu_peak(int kind, int iters, void *cuda_stream, double *tflops, double *ms) {
  if (iters <= 0 || iters % 8 != 0 || !tflops) return RX_EINVAL;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  if (kind == 0) return run<float>(st, iters, tflops, ms);
  if (kind == 1) return run<double>(st, iters, tflops, ms);
  return RX_EINVAL;
}
