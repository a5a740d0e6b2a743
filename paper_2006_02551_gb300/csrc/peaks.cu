// Measured fused multiply-add throughput of the CUDA cores (FP32 and FP64),
// the roofline denominators of the CUDA-core stage kernels.  Each thread runs
// independent FMA chains on registers (enough chains to cover the pipe
// latency), every block on every SM, timed with CUDA events; the result
// feeds nothing back into the method.
#include <cuda_runtime.h>

#include "../../include/wadg.h"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kIters = 4096;    // iterations of the unrolled chain block

template <typename T>
__global__ void fma_peak_kernel(T seed, T* sink) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
  const T m = (T)0.999999, b = (T)1e-7;
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == (T)12345.678) *sink = s;   // keeps the chains live; never true in practice
}

template <typename T>
wadg_status run(int device, double* tflops) {
  if (cudaSetDevice(device) != cudaSuccess) return WADG_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (sms <= 0) return WADG_ECUDA;
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return WADG_ENOMEM;
  const int threads = 512, blocks = sms * 4;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_peak_kernel<T><<<blocks, threads>>>((T)1, sink);   // warm-up
  cudaEventRecord(e0);
  const int reps = 3;
  for (int r = 0; r < reps; ++r) fma_peak_kernel<T><<<blocks, threads>>>((T)1, sink);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess || ms <= 0.f) return WADG_ECUDA;
  const double flops = 2.0 * kChains * 8.0 * kIters * (double)threads * blocks * reps;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return WADG_OK;
}

}  // namespace

extern "C" wadg_status wadg_fma_peak(int device, int fp64, double* tflops) {
  if (!tflops) return WADG_EINVAL;
  return fp64 ? run<double>(device, tflops) : run<float>(device, tflops);
}
