// Rank-based statistics of a count matrix on the GPU: the Nonparanormal
// Skeptic in the COCA form of Section "Algorithm" (Section "The model":
// Gaussian copula; the worked example of the appendix "Preserving input
// sparsity" fixes the conventions): every row of mat_l[D] is ranked across
// its entries, ties taking the lowest rank of their group (rank = 1 + the
// number of strictly smaller entries), and rank k of a row of N entries
// maps to the score Phi^-1(k / (N + 1)).
//
// The inputs are counts (non-negative integers, exact in FP32), so ranks
// come from counting, not sorting:
//   axis COLS (each column ranked over the n rows; genes over cells):
//     per-column maxima -> one histogram per column (bins 0..max, laid out
//     back to back) -> per-column exclusive prefix sums = #smaller entries
//     -> scores per (column, value) -> one pass writing the scores.
//   axis ROWS (each row ranked over its p entries; cells over genes):
//     one warp per row: a shared-memory histogram of the values below
//     kRB (equal values grouped with match_any, one add per group), an
//     exclusive prefix, then rank = 1 + prefix; a value >= kRB (rare in
//     counts) is ranked by counting the row's larger entries directly.
// Both write the scores row-major (FP32) and/or as the BF16 hi/lo split of
// the transpose (the layout the tensor-core Gram and lift read).
// Scores: Phi^-1 evaluated in FP64 (normcdfinv), rounded to FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace gmgm {
namespace {

constexpr float kCountMax = 16777216.f;  // 2^24: integers exact in FP32

__device__ __forceinline__ bool is_count(float v) { return v >= 0.f && v <= kCountMax && v == truncf(v); }

// tbl[k - 1] = Phi^-1(k / (N + 1)), k = 1..N
__global__ void quantile_table_kernel(int64_t N, float* __restrict__ tbl) {
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < N; k += int64_t(gridDim.x) * blockDim.x)
    tbl[k] = float(normcdfinv(double(k + 1) / double(N + 1)));
}

// ---- axis ROWS -----------------------------------------------------------------

constexpr int kRB = 1024;      // histogram bins per row
constexpr int kRWarps = 8;

__global__ void __launch_bounds__(kRWarps * 32) row_rank_kernel(const float* __restrict__ c, int64_t n, int64_t p,
                                                                  int64_t ldc, const float* __restrict__ tbl,
                                                                  float* __restrict__ z, int64_t ldz,
                                                                  int32_t* __restrict__ ranks, int64_t ldr,
                                                                  int* __restrict__ status) {
  extern __shared__ unsigned rsm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned* h = rsm + w * kRB;
  const int64_t gw = int64_t(blockIdx.x) * kRWarps + w, nw = int64_t(gridDim.x) * kRWarps;
  for (int64_t i = gw; i < n; i += nw) {
    const float* row = c + i * ldc;
    for (int b = lane; b < kRB; b += 32) h[b] = 0u;
    __syncwarp();
    int nsmall = 0, kmax = -1;
    bool bad = false;
    for (int64_t j0 = 0; j0 < p; j0 += 32) {
      const int64_t j = j0 + lane;
      const float v = j < p ? row[j] : 0.f;
      const bool ok = j < p && is_count(v);
      bad |= j < p && !ok;
      const int key = (ok && v < float(kRB)) ? int(v) : -1 - lane;  // unique keys outside the bins
      const unsigned grp = __match_any_sync(0xffffffffu, key);
      if (key >= 0 && lane == __ffs(grp) - 1) h[key] += unsigned(__popc(grp));
      nsmall += key >= 0;
      kmax = max(kmax, key);
      __syncwarp();
    }
    nsmall = warp_sum(nsmall);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(status, GMGM_DEV_NOT_COUNTS);
    // exclusive prefix over the bins in use, 32 at a time
    unsigned run = 0;
    for (int b0 = 0; b0 <= kmax; b0 += 32) {
      const unsigned x = h[b0 + lane];
      unsigned s = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      h[b0 + lane] = run + s - x;
      run += __shfl_sync(0xffffffffu, s, 31);
    }
    __syncwarp();
    for (int64_t j0 = 0; j0 < p; j0 += 32) {
      const int64_t j = j0 + lane;
      if (j >= p) continue;
      const float v = row[j];
      int64_t rank;
      if (is_count(v) && v < float(kRB)) {
        rank = 1 + int64_t(h[int(v)]);
      } else {
        // a large value: every binned entry is smaller; count the larger
        // entries below it directly
        int64_t cnt = 0;
        for (int64_t u = 0; u < p; ++u) {
          const float x = row[u];
          cnt += (x >= float(kRB) && x < v) ? 1 : 0;
        }
        rank = 1 + nsmall + cnt;
      }
      rank = rank < 1 ? 1 : (rank > p ? p : rank);
      if (z) z[i * ldz + j] = tbl[rank - 1];
      if (ranks) ranks[i * ldr + j] = int32_t(rank);
    }
    __syncwarp();
  }
}

// ---- axis COLS -----------------------------------------------------------------

constexpr int kCT = 256;      // columns per CTA (one per thread)
constexpr int kCR = 2048;     // rows per CTA
constexpr int kCSmall = 32;   // per-thread shared-memory bins (values below)

__global__ void col_max_kernel(const float* __restrict__ c, int64_t n, int64_t p, int64_t ldc, int* __restrict__ vmax,
                               int* __restrict__ status) {
  const int64_t col = int64_t(blockIdx.y) * kCT + threadIdx.x;
  const int64_t r0 = int64_t(blockIdx.x) * kCR, r1 = min(n, r0 + kCR);
  if (col >= p) return;
  int m = 0;
  bool bad = false;
  const float* src = c + r0 * ldc + col;
#pragma unroll 8
  for (int64_t r = r0; r < r1; ++r, src += ldc) {
    const float v = __ldg(src);
    if (is_count(v))
      m = max(m, int(v));
    else
      bad = true;
  }
  atomicMax(&vmax[col], m);
  if (bad) set_status(status, GMGM_DEV_NOT_COUNTS);
}

__global__ void __launch_bounds__(kCT) col_hist_kernel(const float* __restrict__ c, int64_t n, int64_t p, int64_t ldc,
                                                       const int64_t* __restrict__ off, const int* __restrict__ vmax,
                                                       unsigned* __restrict__ hist) {
  __shared__ unsigned short hs[kCSmall][kCT];
  const int64_t col = int64_t(blockIdx.y) * kCT + threadIdx.x;
  const int64_t r0 = int64_t(blockIdx.x) * kCR, r1 = min(n, r0 + kCR);
#pragma unroll
  for (int b = 0; b < kCSmall; ++b) hs[b][threadIdx.x] = 0;
  if (col >= p) return;
  const int vm = vmax[col];
  unsigned* hc = hist + off[col];
  const float* src = c + r0 * ldc + col;
#pragma unroll 4
  for (int64_t r = r0; r < r1; ++r, src += ldc) {
    const float v = __ldg(src);
    if (!is_count(v)) continue;  // flagged by col_max_kernel
    const int k = int(v);
    if (k > vm) continue;
    if (k < kCSmall)
      hs[k][threadIdx.x] += 1;
    else
      atomicAdd(hc + k, 1u);
  }
  const int top = min(vm, kCSmall - 1);
  for (int b = 0; b <= top; ++b)
    if (hs[b][threadIdx.x]) atomicAdd(hc + b, unsigned(hs[b][threadIdx.x]));
}

// One CTA per column: exclusive prefix of its bins (the number of strictly
// smaller entries) and the score of each value.
__global__ void __launch_bounds__(256) col_prefix_kernel(int64_t n, const int64_t* __restrict__ off,
                                                         unsigned* __restrict__ hist, float* __restrict__ score) {
  __shared__ unsigned wsum[8];
  __shared__ unsigned carry;
  const int64_t col = blockIdx.x;
  const int64_t b0 = off[col], b1 = off[col + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = b0; base < b1; base += 256) {
    const int64_t b = base + threadIdx.x;
    const unsigned x = b < b1 ? hist[b] : 0u;
    unsigned s = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane == 31) wsum[w] = s;
    __syncthreads();
    unsigned before = carry;
    for (int q = 0; q < w; ++q) before += wsum[q];
    const unsigned ex = before + s - x;
    if (b < b1) {
      hist[b] = ex;
      score[b] = float(normcdfinv(double(ex + 1) / double(n + 1)));
    }
    __syncthreads();
    if (threadIdx.x == 255) carry = before + s;
    __syncthreads();
  }
}

constexpr int kT = 64;

// Scores (and ranks) of a count matrix from per-(column, value) tables,
// written row-major and/or as the BF16 split of the transpose; 64 x 64 tiles.
__global__ void col_out_kernel(const float* __restrict__ c, int64_t n, int64_t p, int64_t ldc,
                               const int64_t* __restrict__ off, const int* __restrict__ vmax,
                               const unsigned* __restrict__ pre, const float* __restrict__ score,
                               float* __restrict__ z, int64_t ldz, int32_t* __restrict__ ranks, int64_t ldr,
                               __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t ld_t) {
  __shared__ float tile[kT][kT + 1];
  const int64_t row0 = int64_t(blockIdx.x) * kT, col0 = int64_t(blockIdx.y) * kT;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t col = col0 + tx;
  for (int rr = ty; rr < kT; rr += 4) {
    const int64_t row = row0 + rr;
    float s = 0.f;
    if (row < n && col < p) {
      const float v = c[row * ldc + col];
      const int k = is_count(v) ? min(int(v), vmax[col]) : 0;
      const int64_t b = off[col] + k;
      s = score[b];
      if (z) z[row * ldz + col] = s;
      if (ranks) ranks[row * ldr + col] = int32_t(1 + pre[b]);
    }
    tile[rr][tx] = s;
  }
  if (hi == nullptr) return;
  __syncthreads();
  const int cp = threadIdx.x & 31, gy = threadIdx.x >> 5;
  for (int cc = gy; cc < kT; cc += 8) {
    const int64_t gene = col0 + cc, cell = row0 + 2 * cp;
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

// BF16 split of the transpose of an FP32 row-major matrix (the axis-ROWS
// scores), 64 x 64 tiles.
__global__ void split_t_kernel(const float* __restrict__ z, int64_t n, int64_t p, int64_t ldz,
                               __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t ld_t) {
  __shared__ float tile[kT][kT + 1];
  const int64_t row0 = int64_t(blockIdx.x) * kT, col0 = int64_t(blockIdx.y) * kT;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t col = col0 + tx;
  for (int rr = ty; rr < kT; rr += 4) {
    const int64_t row = row0 + rr;
    tile[rr][tx] = (row < n && col < p) ? z[row * ldz + col] : 0.f;
  }
  __syncthreads();
  const int cp = threadIdx.x & 31, gy = threadIdx.x >> 5;
  for (int cc = gy; cc < kT; cc += 8) {
    const int64_t gene = col0 + cc, cell = row0 + 2 * cp;
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

__global__ void zero_cols_kernel(__nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t n,
                                 int64_t p, int64_t ld_t) {
  const int64_t wdt = ld_t - n, total = wdt * p;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t g = i / wdt, cc = n + i % wdt;
    hi[g * ld_t + cc] = __float2bfloat16_rn(0.f);
    lo[g * ld_t + cc] = __float2bfloat16_rn(0.f);
  }
}

void zero_pad(gmgm_handle* h, uint16_t* hi, uint16_t* lo, int64_t n, int64_t p, int64_t ld_t) {
  if (!hi || ld_t <= n) return;
  const unsigned blocks = unsigned(std::min<int64_t>(4096, ((ld_t - n) * p + 255) / 256));
  zero_cols_kernel<<<blocks, 256, 0, h->stream>>>(reinterpret_cast<__nv_bfloat16*>(hi),
                                                  reinterpret_cast<__nv_bfloat16*>(lo), n, p, ld_t);
  note_launch(1);
}

}  // namespace

int skeptic_rows(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc, float* z, int64_t ldz,
                 uint16_t* hi, uint16_t* lo, int64_t ld_t, int32_t* ranks, int64_t ldr) {
  int rc = ensure_scratch(h, Carve::round(size_t(p) * 4) + 1024);
  if (rc) return rc;
  Carve cv(h->scratch);
  float* tbl = cv.take<float>(size_t(p));
  cudaStream_t s = h->stream;
  quantile_table_kernel<<<unsigned(std::min<int64_t>((p + 255) / 256, 1024)), 256, 0, s>>>(p, tbl);
  const size_t smem = size_t(kRWarps) * kRB * sizeof(unsigned);
  GMGM_CUDA_TRY(h, cudaFuncSetAttribute(row_rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const unsigned blocks = unsigned(std::min<int64_t>((n + kRWarps - 1) / kRWarps, int64_t(h->num_sms) * 8));
  row_rank_kernel<<<blocks, kRWarps * 32, smem, s>>>(counts, n, p, ldc, tbl, z, ldz, ranks, ldr, h->d_status);
  note_launch(2);
  if (hi) {
    dim3 g2(unsigned((n + kT - 1) / kT), unsigned((p + kT - 1) / kT));
    split_t_kernel<<<g2, 256, 0, s>>>(z, n, p, ldz, reinterpret_cast<__nv_bfloat16*>(hi),
                                      reinterpret_cast<__nv_bfloat16*>(lo), ld_t);
    note_launch(1);
    zero_pad(h, hi, lo, n, p, ld_t);
  }
  GMGM_CUDA_TRY(h, cudaGetLastError());
  return GMGM_OK;
}

int skeptic_cols(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc, float* z, int64_t ldz,
                 uint16_t* hi, uint16_t* lo, int64_t ld_t, int32_t* ranks, int64_t ldr) {
  cudaStream_t s = h->stream;
  // pass 1: per-column maxima (read back: they size the histograms)
  int rc = ensure_scratch(h, Carve::round(size_t(p) * 4) + 1024);
  if (rc) return rc;
  int* vmax_d = static_cast<int*>(h->scratch);
  GMGM_CUDA_TRY(h, cudaMemsetAsync(vmax_d, 0, size_t(p) * 4, s));
  dim3 g1(unsigned((n + kCR - 1) / kCR), unsigned((p + kCT - 1) / kCT));
  col_max_kernel<<<g1, kCT, 0, s>>>(counts, n, p, ldc, vmax_d, h->d_status);
  note_launch(1);
  std::vector<int> vmax(static_cast<size_t>(p));
  GMGM_CUDA_TRY(h, cudaMemcpyAsync(vmax.data(), vmax_d, size_t(p) * 4, cudaMemcpyDeviceToHost, s));
  GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
  std::vector<int64_t> off(static_cast<size_t>(p) + 1, 0);
  for (int64_t g = 0; g < p; ++g) off[g + 1] = off[g] + int64_t(vmax[g]) + 1;
  const int64_t bins = off[p];
  if (bins > (int64_t(1) << 31))
    return fail(h, GMGM_E_ARG, "gmgm_skeptic: column value ranges need more than 2^31 histogram bins");
  rc = ensure_scratch(h, Carve::round(size_t(p) * 4) + Carve::round(size_t(p + 1) * 8) +
                             2 * Carve::round(size_t(bins) * 4) + 4096);
  if (rc) return rc;
  Carve cv(h->scratch);
  int* vm = cv.take<int>(size_t(p));
  int64_t* offd = cv.take<int64_t>(size_t(p) + 1);
  unsigned* hist = cv.take<unsigned>(size_t(bins));
  float* score = cv.take<float>(size_t(bins));
  GMGM_CUDA_TRY(h, cudaMemcpyAsync(vm, vmax.data(), size_t(p) * 4, cudaMemcpyHostToDevice, s));
  GMGM_CUDA_TRY(h, cudaMemcpyAsync(offd, off.data(), size_t(p + 1) * 8, cudaMemcpyHostToDevice, s));
  GMGM_CUDA_TRY(h, cudaMemsetAsync(hist, 0, size_t(bins) * 4, s));
  // pass 2: histograms; prefix sums and scores per (column, value)
  col_hist_kernel<<<g1, kCT, 0, s>>>(counts, n, p, ldc, offd, vm, hist);
  col_prefix_kernel<<<unsigned(p), 256, 0, s>>>(n, offd, hist, score);
  // pass 3: the scores of every entry
  dim3 g3(unsigned((n + kT - 1) / kT), unsigned((p + kT - 1) / kT));
  col_out_kernel<<<g3, 256, 0, s>>>(counts, n, p, ldc, offd, vm, hist, score, z, ldz, ranks, ldr,
                                    reinterpret_cast<__nv_bfloat16*>(hi), reinterpret_cast<__nv_bfloat16*>(lo), ld_t);
  note_launch(3);
  zero_pad(h, hi, lo, n, p, ld_t);
  // the host vectors must outlive the async copies
  GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
  GMGM_CUDA_TRY(h, cudaGetLastError());
  return GMGM_OK;
}

}  // namespace gmgm
