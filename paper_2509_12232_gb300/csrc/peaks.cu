// Measured issue peaks of the two pipes the scoring kernels are judged
// against: FP32 fused multiply-add and the special-function unit (MUFU:
// ex2). Each kernel runs independent dependency chains per thread, enough of
// them that latency is hidden, on every SM; the host times it with events.
// These replace peaks derived from unit counts and the clock.
#include <cuda_runtime.h>

#include <algorithm>

#include "dock.h"
#include "dock_internal.h"

namespace {

constexpr int kChains = 8;      // independent chains per thread
constexpr int kIters = 4096;    // iterations of the chain loop
constexpr int kUnroll = 16;     // FMAs per chain per iteration

__global__ void __launch_bounds__(256) ffma_peak_kernel(float a, float b, float *sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 1.2345f) *sink = s;  // keeps the chains live
}

__global__ void __launch_bounds__(256) mufu_peak_kernel(float a, float *sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * -1e-3f;
  for (int i = 0; i < kIters / 8; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        float y;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
        x[c] = y * a;  // stays in (0, 1]: a < 0 keeps the argument negative
      }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 1.2345f) *sink = s;
}

}  // namespace

// Measured peaks (see dock.h).
extern "C" int dock_measure_peaks(double *fp32_tflops, double *mufu_tops, void *stream) {
  if (!fp32_tflops || !mufu_tops) return DOCK_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DOCK_ECUDA;
  float *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return DOCK_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = n_sm * 8, threads = 256;
  double best_f = 0.0, best_m = 0.0;
  int st = DOCK_OK;
  for (int rep = 0; rep < 4 && st == DOCK_OK; ++rep) {
    float ms = 0.0f;
    cudaEventRecord(e0, s);
    ffma_peak_kernel<<<blocks, threads, 0, s>>>(0.999f, 1e-4f, sink);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = DOCK_ECUDA;
      break;
    }
    const double flops = 2.0 * blocks * threads * (double)kIters * kUnroll * kChains;
    if (rep > 0) best_f = std::max(best_f, flops / (ms * 1e-3) / 1e12);
    cudaEventRecord(e0, s);
    mufu_peak_kernel<<<blocks, threads, 0, s>>>(-0.5f, sink);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = DOCK_ECUDA;
      break;
    }
    const double ops = (double)blocks * threads * (double)(kIters / 8) * kUnroll * kChains;
    if (rep > 0) best_m = std::max(best_m, ops / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  *fp32_tflops = best_f;
  *mufu_tops = best_m;
  return st;
}
