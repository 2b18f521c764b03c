// Preprocessing: X = log1p(counts) - column means, with an optional BF16
// hi/lo split of X^T (gene-major) for the tensor-core Gram.
// HBM-bound: pass 1 reads counts once (column sums), pass 2 reads counts and
// writes X (and the two BF16 planes).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace gmgm {
namespace {

constexpr int kColThreads = 256;
constexpr int kRowChunk = 2048;

// Column sums of log1p(counts): one thread per column, a chunk of rows per
// CTA, Kahan-compensated FP32 inside the chunk, FP64 atomics across chunks.
__global__ void colsum_log1p_kernel(const float* __restrict__ c, int64_t n, int64_t p, int64_t ldc,
                                    double* __restrict__ colsum) {
  const int64_t col = int64_t(blockIdx.y) * kColThreads + threadIdx.x;
  const int64_t r0 = int64_t(blockIdx.x) * kRowChunk;
  const int64_t r1 = min(n, r0 + kRowChunk);
  if (col >= p) return;
  float s = 0.f, comp = 0.f;
  const float* src = c + r0 * ldc + col;
#pragma unroll 8
  for (int64_t r = r0; r < r1; ++r, src += ldc) {
    float y = log1pf(__ldg(src)) - comp;
    float t = s + y;
    comp = (t - s) - y;
    s = t;
  }
  atomicAdd(&colsum[col], double(s));
}

// 64 x 64 tiles: rows = cells, columns = genes.
constexpr int kT = 64;

// c and x may alias (in-place); each element is read and then written by
// the same thread.
// The mean of column j is colsum[j] / n_mean (n_mean = n, or the total row
// count of a matrix whose rows are split over several calls).
__global__ void centre_split_kernel(const float* c, int64_t n, int64_t p,
                                    int64_t ldc, float* x, int64_t ldx,
                                    __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                    int64_t ld_t, const double* __restrict__ colsum, int64_t n_mean) {
  __shared__ float tile[kT][kT + 1];
  const int64_t row0 = int64_t(blockIdx.x) * kT, col0 = int64_t(blockIdx.y) * kT;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 256 threads: 64 x 4
  const int64_t col = col0 + tx;
  const float mean = col < p ? float(colsum[col] / double(n_mean)) : 0.f;
  for (int rr = ty; rr < kT; rr += 4) {
    const int64_t row = row0 + rr;
    float v = 0.f;
    if (row < n && col < p) {
      v = log1pf(c[row * ldc + col]) - mean;
      if (x) x[row * ldx + col] = v;  // (null: only the planes are wanted)
    }
    tile[rr][tx] = v;
  }
  if (hi == nullptr) return;
  __syncthreads();
  // transposed write: xt[gene][cell], 64 consecutive cells per gene row,
  // two cells per thread (bf16x2 stores: a warp writes 128 contiguous bytes)
  const int cp = threadIdx.x & 31, gy = threadIdx.x >> 5;  // 32 cell pairs x 8 genes
  for (int cc = gy; cc < kT; cc += 8) {
    const int64_t gene = col0 + cc;
    const int64_t cell = row0 + 2 * cp;
    if (gene >= p || cell >= n) continue;
    const float v0 = tile[2 * cp][cc];
    const float v1 = cell + 1 < n ? tile[2 * cp + 1][cc] : 0.f;
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
    if (cell + 1 < n) {
      *reinterpret_cast<__nv_bfloat162*>(hi + gene * ld_t + cell) = __halves2bfloat162(h0, h1);
      *reinterpret_cast<__nv_bfloat162*>(lo + gene * ld_t + cell) = __halves2bfloat162(l0, l1);
    } else {
      hi[gene * ld_t + cell] = h0;
      lo[gene * ld_t + cell] = l0;
    }
  }
}

__global__ void zero_pad_kernel(__nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                int64_t n, int64_t p, int64_t ld_t) {
  const int64_t w = ld_t - n;
  const int64_t total = w * p;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t g = i / w, cc = n + i % w;
    hi[g * ld_t + cc] = __float2bfloat16_rn(0.f);
    lo[g * ld_t + cc] = __float2bfloat16_rn(0.f);
  }
}

__global__ void colmean_kernel(const double* __restrict__ colsum, int64_t n, int64_t p,
                               double* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < p) out[i] = colsum[i] / double(n);
}

}  // namespace

cudaError_t launch_preprocess(gmgm_handle* h, int64_t n, int64_t p, const float* counts,
                              int64_t ldc, float* x_out, int64_t ldx, uint16_t* xt_hi,
                              uint16_t* xt_lo, int64_t ld_t, double* colsum, double* colmean_out) {
  cudaStream_t s = h->stream;
  cudaError_t e = cudaMemsetAsync(colsum, 0, size_t(p) * sizeof(double), s);
  if (e != cudaSuccess) return e;
  dim3 g1(unsigned((n + kRowChunk - 1) / kRowChunk), unsigned((p + kColThreads - 1) / kColThreads));
  colsum_log1p_kernel<<<g1, kColThreads, 0, s>>>(counts, n, p, ldc, colsum);
  dim3 g2(unsigned((n + kT - 1) / kT), unsigned((p + kT - 1) / kT));
  centre_split_kernel<<<g2, 256, 0, s>>>(counts, n, p, ldc, x_out, ldx,
                                         reinterpret_cast<__nv_bfloat16*>(xt_hi),
                                         reinterpret_cast<__nv_bfloat16*>(xt_lo), ld_t, colsum, n);
  if (xt_hi && ld_t > n) {
    int blocks = int(std::min<int64_t>(4096, ((ld_t - n) * p + 255) / 256));
    zero_pad_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<__nv_bfloat16*>(xt_hi),
                                           reinterpret_cast<__nv_bfloat16*>(xt_lo), n, p, ld_t);
  }
  if (colmean_out) colmean_kernel<<<unsigned((p + 255) / 256), 256, 0, s>>>(colsum, n, p, colmean_out);
  note_launch(2 + (xt_hi && ld_t > n ? 1 : 0) + (colmean_out ? 1 : 0));
  return cudaGetLastError();
}

cudaError_t launch_colsum_log1p(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc,
                                double* colsum, int accumulate) {
  cudaStream_t s = h->stream;
  if (!accumulate) {
    cudaError_t e = cudaMemsetAsync(colsum, 0, size_t(p) * sizeof(double), s);
    if (e != cudaSuccess) return e;
  }
  dim3 g1(unsigned((n + kRowChunk - 1) / kRowChunk), unsigned((p + kColThreads - 1) / kColThreads));
  colsum_log1p_kernel<<<g1, kColThreads, 0, s>>>(counts, n, p, ldc, colsum);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_centre(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc,
                          const double* colsum, int64_t n_total, float* x_out, int64_t ldx, uint16_t* xt_hi,
                          uint16_t* xt_lo, int64_t ld_t) {
  cudaStream_t s = h->stream;
  dim3 g2(unsigned((n + kT - 1) / kT), unsigned((p + kT - 1) / kT));
  centre_split_kernel<<<g2, 256, 0, s>>>(counts, n, p, ldc, x_out, ldx, reinterpret_cast<__nv_bfloat16*>(xt_hi),
                                         reinterpret_cast<__nv_bfloat16*>(xt_lo), ld_t, colsum, n_total);
  if (xt_hi && ld_t > n) {
    int blocks = int(std::min<int64_t>(4096, ((ld_t - n) * p + 255) / 256));
    zero_pad_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<__nv_bfloat16*>(xt_hi),
                                           reinterpret_cast<__nv_bfloat16*>(xt_lo), n, p, ld_t);
  }
  note_launch(1 + (xt_hi && ld_t > n ? 1 : 0));
  return cudaGetLastError();
}

}  // namespace gmgm
