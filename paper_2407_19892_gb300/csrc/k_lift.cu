// Dual lift U = X W_r diag(E_r)^-1/2 (rows x r, FP32): the top-r left
// singular vectors of X from the right ones.  One thread per row of X keeps
// its r outputs in registers; X is staged through shared memory in 32-column
// tiles (coalesced loads, conflict-free transposed reads); the scaled W chunk
// is broadcast from shared memory.  HBM-bound on reading X once.
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace gmgm {
namespace {

constexpr int kRows = 256, kG = 32;

__global__ void scale_w_kernel(const double* __restrict__ W, int64_t ldw, const double* __restrict__ E,
                               int64_t p, int r, int rpad, float* __restrict__ ws) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= p * rpad) return;
  const int64_t g = i / rpad;
  const int c = int(i - g * rpad);
  ws[i] = c < r ? float(W[g * ldw + c] / sqrt(E[c])) : 0.f;
}

template <int RC>
__global__ void __launch_bounds__(kRows, 2) lift_kernel(const float* __restrict__ x, int64_t n, int64_t p, int64_t ld,
                                                     const float* __restrict__ ws, int rpad, int c0, int r,
                                                     float* __restrict__ U, int64_t ldu) {
  __shared__ float xs[kG][kRows + 1];
  __shared__ __align__(16) float wsh[kG][RC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t row0 = int64_t(blockIdx.x) * kRows;
  float acc[RC];
#pragma unroll
  for (int c = 0; c < RC; ++c) acc[c] = 0.f;
  for (int64_t g0 = 0; g0 < p; g0 += kG) {
    // X tile: warp w loads rows w, w+8, ...; lane = column
    for (int rr = warp; rr < kRows; rr += kRows / 32) {
      const int64_t row = row0 + rr, g = g0 + lane;
      xs[lane][rr] = (row < n && g < p) ? x[row * ld + g] : 0.f;
    }
    for (int e = threadIdx.x; e < kG * RC; e += kRows) {
      const int gg = e / RC, c = e - gg * RC;
      const int64_t g = g0 + gg;
      wsh[gg][c] = g < p ? ws[g * rpad + c0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int gg = 0; gg < kG; ++gg) {
      const float xv = xs[gg][threadIdx.x];
      const float4* w4 = reinterpret_cast<const float4*>(&wsh[gg][0]);
#pragma unroll
      for (int q = 0; q < RC / 4; ++q) {
        const float4 w = w4[q];
        acc[4 * q + 0] = fmaf(xv, w.x, acc[4 * q + 0]);
        acc[4 * q + 1] = fmaf(xv, w.y, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(xv, w.z, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(xv, w.w, acc[4 * q + 3]);
      }
    }
    __syncthreads();
  }
  const int64_t row = row0 + threadIdx.x;
  if (row >= n) return;
#pragma unroll
  for (int c = 0; c < RC; ++c)
    if (c0 + c < r) U[row * ldu + c0 + c] = acc[c];
}

}  // namespace

cudaError_t launch_lift(gmgm_handle* h, const gmgm_matrix* m, int32_t r, const double* W, int64_t ldw,
                        const double* E, float* U, int64_t ldu, float* wscr) {
  const int RC = r <= 16 ? 16 : (r <= 32 ? 32 : 64);
  const int rpad = ((r + RC - 1) / RC) * RC;
  const int64_t p = m->cols, n = m->rows;
  scale_w_kernel<<<unsigned((p * rpad + 255) / 256), 256, 0, h->stream>>>(W, ldw, E, p, r, rpad, wscr);
  const unsigned blocks = unsigned((n + kRows - 1) / kRows);
  for (int c0 = 0; c0 < r; c0 += RC) {
    if (RC == 16)
      lift_kernel<16><<<blocks, kRows, 0, h->stream>>>(m->x, n, p, m->ld, wscr, rpad, c0, r, U, ldu);
    else if (RC == 32)
      lift_kernel<32><<<blocks, kRows, 0, h->stream>>>(m->x, n, p, m->ld, wscr, rpad, c0, r, U, ldu);
    else
      lift_kernel<64><<<blocks, kRows, 0, h->stream>>>(m->x, n, p, m->ld, wscr, rpad, c0, r, U, ldu);
  }
  note_launch(1 + (r + RC - 1) / RC);
  return cudaGetLastError();
}

}  // namespace gmgm
