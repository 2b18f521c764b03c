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

// A grid barrier gives up after this long.
constexpr unsigned long long kBarrierWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long device_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier for a cooperative launch (all CTAs resident), on a counter
// of arrivals that only grows during the launch: bar[0] = arrivals (zeroed
// before the launch), bar[2] = abort flag.  `epoch` counts the barriers this
// CTA has passed (every CTA passes the same ones), so barrier e completes
// when bar[0] reaches (e + 1) * nblocks.  One CTA-wide sync, then thread 0
// arrives with one acquire-release atomic (the CTA's writes, ordered before
// it by the sync, become visible to every CTA that acquires the count) and
// polls the count with acquire loads; no other global access sits on the
// path.  Every wait is bounded: after kBarrierWaitNs, or once another CTA
// has raised the abort flag (read every 64 polls), the TIMEOUT status bit
// and the abort flag are set and the function returns false; callers then
// leave the kernel, and any CTA still waiting at a later barrier sees the
// flag and leaves too.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned& epoch, int* status) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = (epoch + 1u) * nblocks;
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
    if (old + 1u != target) {
      unsigned spins = 0;
      unsigned long long t0 = 0;
      for (;;) {
        unsigned cur;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(bar) : "memory");
        if (static_cast<int>(cur - target) >= 0) break;
        if ((++spins & 63u) == 0u) {
          const unsigned long long t = device_ns();
          if (t0 == 0) {
            t0 = t;
          } else if (reinterpret_cast<volatile unsigned*>(bar)[2] != 0u || t - t0 > kBarrierWaitNs) {
            ok = 0;
            break;
          }
        }
      }
      if (!ok) {
        atomicExch(&bar[2], 1u);
        set_status(status, GMGM_DEV_TIMEOUT);
      }
    }
    ok_s = ok;
  }
  ++epoch;
  __syncthreads();
  return ok_s != 0;
}

}  // namespace gmgm
