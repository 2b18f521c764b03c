// Throughput probes for the roofline denominators that no library measures
// on this GPU: the FP64 FMA pipe (the eigendecomposition's back-
// transformation and the exact FP64 scans) and the special-function unit
// (the approximate reciprocal and base-2 logarithm the eigenvalue solve's
// grid reductions issue once per term each).  Every thread runs independent
// dependency chains long enough to hide the pipe latency; the host times one
// launch with CUDA events.
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace gmgm {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fp64_fma_kernel(long long iters, double seed, double* sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x * 1e-9 + c;
  const double m = 0.999999, b = 1e-7;
  for (long long i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, b);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678) sink[0] = s;  // keeps the chains alive
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One reciprocal and one logarithm per step and chain (what a grid term of
// the solve costs the special-function unit), plus two FP32 adds.
__global__ void __launch_bounds__(256) mufu_kernel(long long iters, float seed, float* sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x * 1e-6f + c;
  for (long long i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = rcp_approx(a[c]) + lg2_approx(a[c] + 3.0f) + 1.5f;
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678f) sink[0] = s;
}

}  // namespace

int peak_probe(gmgm_handle* h, int kind, long long iters, double* rate) {
  const int blocks = h->num_sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  GMGM_CUDA_TRY(h, cudaEventCreate(&e0));
  GMGM_CUDA_TRY(h, cudaEventCreate(&e1));
  void* sink = h->scratch;
  GMGM_CUDA_TRY(h, cudaEventRecord(e0, h->stream));
  if (kind == 0)
    fp64_fma_kernel<<<blocks, threads, 0, h->stream>>>(iters, 1.0, static_cast<double*>(sink));
  else
    mufu_kernel<<<blocks, threads, 0, h->stream>>>(iters, 1.0f, static_cast<float*>(sink));
  GMGM_CUDA_TRY(h, cudaEventRecord(e1, h->stream));
  GMGM_CUDA_TRY(h, cudaEventSynchronize(e1));
  note_launch(1);
  float ms = 0.f;
  GMGM_CUDA_TRY(h, cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double ops = double(blocks) * threads * double(iters) * kChains;
  // FP64: 2 flop per FMA; special functions: operations (one rcp or one lg2)
  *rate = (kind == 0 ? 2.0 * ops : 2.0 * ops) / (ms * 1e-3);
  return GMGM_OK;
}

}  // namespace gmgm
