// Preprocessing of a sparse (CSR) count matrix without its dense form (the
// appendix "Preserving input sparsity": the transformed matrix is a matrix
// with the input's sparsity plus a rank-one term).  log1p keeps every zero
// at zero, and centring subtracts the rank-one 1 mu^T, so the centred matrix
// is X = log1p(C) - 1 mu^T with log1p(C) sparse.  Here:
//   pass 1  mu = column sums of log1p over the non-zeros / n (FP64; a
//           CTA's sums gathered in shared memory, one global add per column
//           and CTA);
//   pass 2  the BF16 hi/lo planes of X^T (genes x cells, the layout the
//           tensor-core Gram and lift read) written tile by tile: a 64-cell x
//           64-gene tile starts at -mu_g (the rank-one term) and each row's
//           non-zeros inside the tile are scattered over it.
// Neither the dense counts nor the dense FP32 X is formed; the Gram
// X^T X = log1p(C)^T log1p(C) - n mu mu^T and the lift X W D follow from the
// planes on the tensor cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace gmgm {
namespace {

constexpr int kRowsPerCta = 256;

// Column sums of log1p over the non-zeros of a block of rows, gathered in
// shared memory first (p <= 16384 columns); invalid entries set
// GMGM_DEV_NOT_COUNTS and are left out.
__global__ void csr_colsum_kernel(int64_t n, int64_t p, const int64_t* __restrict__ indptr,
                                  const int32_t* __restrict__ indices, const float* __restrict__ data,
                                  double* __restrict__ colsum, int* __restrict__ status) {
  extern __shared__ double cs[];
  for (int64_t g = threadIdx.x; g < p; g += blockDim.x) cs[g] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t r0 = int64_t(blockIdx.x) * kRowsPerCta, r1 = min(n, r0 + kRowsPerCta);
  bool bad = false;
  for (int64_t i = r0 + w; i < r1; i += nw) {
    const int64_t eb = indptr[i];
    for (int64_t e = eb + lane; e < indptr[i + 1]; e += 32) {
      const int g = indices[e];
      const float v = data[e];
      // counts: finite, non-negative; columns in range and ascending
      if (g < 0 || g >= p || !(v >= 0.f) || v > 3.0e38f || (e > eb && indices[e - 1] >= g)) {
        bad = true;
        continue;
      }
      atomicAdd(&cs[g], double(log1pf(v)));
    }
  }
  if (bad) set_status(status, GMGM_DEV_NOT_COUNTS);
  __syncthreads();
  for (int64_t g = threadIdx.x; g < p; g += blockDim.x)
    if (cs[g] != 0.0) atomicAdd(&colsum[g], cs[g]);
}

__global__ void csr_mean_kernel(const double* __restrict__ colsum, int64_t n, int64_t p, float* __restrict__ mean32,
                                double* __restrict__ colmean_out) {
  const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= p) return;
  const double m = colsum[g] / double(n);
  mean32[g] = float(m);
  if (colmean_out) colmean_out[g] = m;
}

constexpr int kT = 64;

// One CTA per 64-cell block: for every 64-gene chunk, the tile of X^T is
// -mu_g, then the non-zeros of the 64 rows inside the chunk (each row's
// columns ascending: a cursor per row walks them chunk by chunk), then it is
// written as the BF16 hi/lo planes, 128 bytes per gene row.
__global__ void __launch_bounds__(256) csr_planes_kernel(int64_t n, int64_t p, const int64_t* __restrict__ indptr,
                                                         const int32_t* __restrict__ indices,
                                                         const float* __restrict__ data,
                                                         const float* __restrict__ mean32,
                                                         __nv_bfloat16* __restrict__ hi,
                                                         __nv_bfloat16* __restrict__ lo, int64_t ld_t) {
  __shared__ float tile[kT][kT + 1];  // [gene][cell]
  __shared__ int64_t cur[kT], end_[kT];
  const int64_t c0 = int64_t(blockIdx.x) * kT;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // 8 warps, 8 rows each
  for (int t = threadIdx.x; t < kT; t += blockDim.x) {
    const int64_t i = c0 + t;
    cur[t] = i < n ? indptr[i] : 0;
    end_[t] = i < n ? indptr[i + 1] : 0;
  }
  __syncthreads();
  for (int64_t g0 = 0; g0 < p; g0 += kT) {
    // the rank-one term
    for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) {
      const int gg = e / kT, cc = e - gg * kT;
      const int64_t g = g0 + gg;
      tile[gg][cc] = (g < p && c0 + cc < n) ? -mean32[g] : 0.f;
    }
    __syncthreads();
    // the non-zeros of each row inside [g0, g0 + 64)
    for (int rr = w; rr < kT; rr += 8) {
      int64_t e0 = cur[rr];
      const int64_t e1 = end_[rr];
      for (;;) {
        const int64_t e = e0 + lane;
        const int g = e < e1 ? indices[e] : INT32_MAX;
        const bool in = g < g0 + kT;
        if (in && g >= g0 && g < p) tile[g - g0][rr] = log1pf(data[e]) - mean32[g];
        const unsigned m = __ballot_sync(0xffffffffu, in);
        e0 += __popc(m);
        if (m != 0xffffffffu) break;
      }
      if (lane == 0) cur[rr] = e0;
    }
    __syncthreads();
    // the planes: gene rows of 64 cells, two cells per thread
    const int cp = threadIdx.x & 31, gy = threadIdx.x >> 5;
    for (int gg = gy; gg < kT; gg += 8) {
      const int64_t g = g0 + gg, cell = c0 + 2 * cp;
      if (g >= p || cell >= ld_t) continue;
      const float v0 = tile[gg][2 * cp], v1 = tile[gg][2 * cp + 1];
      const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
      const __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
      const __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
      *reinterpret_cast<__nv_bfloat162*>(hi + g * ld_t + cell) = __halves2bfloat162(h0, h1);
      *reinterpret_cast<__nv_bfloat162*>(lo + g * ld_t + cell) = __halves2bfloat162(l0, l1);
    }
    __syncthreads();
  }
}

}  // namespace

size_t preprocess_csr_scratch_bytes(int64_t p) { return Carve::round(size_t(p) * 8) + Carve::round(size_t(p) * 4) + 512; }

cudaError_t launch_preprocess_csr(gmgm_handle* h, int64_t n, int64_t p, const int64_t* indptr, const int32_t* indices,
                                  const float* data, uint16_t* xt_hi, uint16_t* xt_lo, int64_t ld_t,
                                  double* colmean_out) {
  cudaStream_t s = h->stream;
  Carve c(h->scratch);
  double* colsum = c.take<double>(size_t(p));
  float* mean32 = c.take<float>(size_t(p));
  cudaError_t e = cudaMemsetAsync(colsum, 0, size_t(p) * 8, s);
  if (e != cudaSuccess) return e;
  const size_t smem = size_t(p) * 8;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(csr_colsum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  csr_colsum_kernel<<<unsigned((n + kRowsPerCta - 1) / kRowsPerCta), 256, smem, s>>>(n, p, indptr, indices, data,
                                                                                     colsum, h->d_status);
  csr_mean_kernel<<<unsigned((p + 255) / 256), 256, 0, s>>>(colsum, n, p, mean32, colmean_out);
  // cells n..ld_t-1 of the last blocks are written as zero by the tile pass
  csr_planes_kernel<<<unsigned((ld_t + kT - 1) / kT), 256, 0, s>>>(n, p, indptr, indices, data, mean32,
                                                                   reinterpret_cast<__nv_bfloat16*>(xt_hi),
                                                                   reinterpret_cast<__nv_bfloat16*>(xt_lo), ld_t);
  note_launch(3);
  return cudaGetLastError();
}

}  // namespace gmgm
