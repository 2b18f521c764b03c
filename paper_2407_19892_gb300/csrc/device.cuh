// Device-side helpers: reductions, status word, bounded grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gmgm.h"

namespace gmgm {

__device__ __forceinline__ void set_status(int* status, int bits) { atomicOr(status, bits); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum for blockDim.x a multiple of 32 (<= 1024); every thread gets
// the result.  `red` is shared scratch of >= 33 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

__device__ __forceinline__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? red[lane] : -1.0e308;
    t = warp_max(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Spin limit for grid barriers: ~2^26 polls (a few seconds at most).
constexpr long long kBarrierSpinLimit = 1ll << 26;

// Grid barrier for a cooperative launch (all CTAs resident), on a counter
// of arrivals that only grows during the launch: bar[0] = arrivals (zeroed
// before the launch), bar[2] = abort flag.  `epoch` counts the barriers this
// CTA has passed (every CTA passes the same ones), so barrier e completes
// when bar[0] reaches (e + 1) * nblocks: one atomic per CTA and no reset or
// generation word on the critical path.  Every wait is bounded: on timeout
// the TIMEOUT status bit and the abort flag are set and the function
// returns false; callers then leave the kernel.  Once aborted, every later
// call returns false immediately.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned& epoch, int* status) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vb = bar;
    int ok = vb[2] == 0u;
    if (ok) {
      const unsigned target = (epoch + 1u) * nblocks;
      __threadfence();  // this CTA's writes (ordered before by the CTA barrier) before the arrival
      const unsigned arrived = atomicAdd(&bar[0], 1u) + 1u;
      if (arrived != target) {
        long long spins = 0;
        while (static_cast<int>(vb[0] - target) < 0) {
          if (vb[2] != 0u || ++spins > kBarrierSpinLimit) {
            ok = 0;
            break;
          }
          __nanosleep(32);
        }
        if (!ok) {
          atomicExch(&bar[2], 1u);
          set_status(status, GMGM_DEV_TIMEOUT);
        }
      }
      __threadfence();
    }
    ok_s = ok;
  }
  ++epoch;
  __syncthreads();
  return ok_s != 0;
}

}  // namespace gmgm
