// Plain-FP32 SIMT Gram S = M M^T (the comparator form of the tensor-core
// Gram).  For side COLS, M[a, t] = X_b[k, a] over all (b, k) rows; for side
// ROWS, M[a, t] = X_b[a, j] over all (b, j) columns.  64 x 64 output tiles of
// the upper triangle, split-K across CTAs, FP32 FMAs inside 4096-long K
// chunks folded into FP64 per thread, FP64 partials combined by a second
// kernel that writes both triangles.
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace gmgm {
namespace {

constexpr int kTile = 64, kBK = 16, kChunk = 4096;

struct MView {
  const float* x;
  int64_t rows, cols, ld, bs;  // per-batch shape and strides
  int side;
  int64_t dS, K;
  __device__ __forceinline__ float at(int64_t a, int64_t t) const {
    if (side == GMGM_SIDE_COLS) {
      const int64_t b = t / rows, k = t - b * rows;
      return x[b * bs + k * ld + a];
    }
    const int64_t b = t / cols, j = t - b * cols;
    return x[b * bs + a * ld + j];
  }
};

__global__ void __launch_bounds__(256) gram_fp32_kernel(MView m, int64_t k_per_split,
                                                        const int2* __restrict__ tiles,
                                                        double* __restrict__ partials) {
  __shared__ float As[kBK][kTile];
  __shared__ float Bs[kBK][kTile];
  const int2 tl = tiles[blockIdx.x];
  const int64_t a0 = int64_t(tl.x) * kTile, c0 = int64_t(tl.y) * kTile;
  const int64_t kbeg = int64_t(blockIdx.y) * k_per_split;
  const int64_t kend = min(m.K, kbeg + k_per_split);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double accd[4][4];
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accd[i][j] = 0.0, acc[i][j] = 0.f;
  int64_t next_fold = kbeg + kChunk;
  for (int64_t k0 = kbeg; k0 < kend; k0 += kBK) {
    // load: 16 x 64 of each operand, 4 elements per thread
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = threadIdx.x + q * 256;
      int kk, aa;
      if (m.side == GMGM_SIDE_COLS) {
        kk = e >> 6, aa = e & 63;   // consecutive threads -> consecutive a (coalesced)
      } else {
        kk = e & 15, aa = e >> 4;   // consecutive threads -> consecutive t
      }
      const int64_t t = k0 + kk;
      const int64_t a = a0 + aa, c = c0 + aa;
      As[kk][aa] = (t < kend && a < m.dS) ? m.at(a, t) : 0.f;
      Bs[kk][aa] = (t < kend && c < m.dS) ? m.at(c, t) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i], bv[i] = Bs[kk][tx * 4 + i];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
    if (k0 + kBK >= next_fold) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) accd[i][j] += double(acc[i][j]), acc[i][j] = 0.f;
      next_fold += kChunk;
    }
  }
  const int64_t ntile = (m.dS + kTile - 1) / kTile;
  double* out = partials + (int64_t(blockIdx.y) * ntile * ntile + int64_t(tl.x) * ntile + tl.y) *
                               (kTile * kTile);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * kTile + tx * 4 + j] = accd[i][j] + double(acc[i][j]);
}

__global__ void gram_combine_kernel(const double* __restrict__ partials, int splits, int64_t dS,
                                    double* __restrict__ S, int64_t lds, int accumulate) {
  const int64_t ntile = (dS + kTile - 1) / kTile;
  const int64_t a = int64_t(blockIdx.y) * blockDim.y + threadIdx.y;
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (a >= dS || c >= dS) return;
  // read from the upper-triangle tile holding (min, max)
  const int64_t lo = min(a, c), hi = max(a, c);
  const int64_t ti = lo / kTile, tj = hi / kTile;
  const int64_t ii = lo % kTile, jj = hi % kTile;
  double s = 0.0;
  for (int sp = 0; sp < splits; ++sp) {
    const double* tp = partials + (int64_t(sp) * ntile * ntile + ti * ntile + tj) * (kTile * kTile);
    // inside a diagonal tile only entries with ii <= jj... both were computed
    s += tp[ii * kTile + jj];
  }
  if (accumulate)
    S[a * lds + c] += s;
  else
    S[a * lds + c] = s;
}

__global__ void make_tiles_kernel(int2* tiles, int ntile) {
  int idx = 0;
  for (int i = 0; i < ntile; ++i)
    for (int j = i; j < ntile; ++j) tiles[idx++] = make_int2(i, j);
}

}  // namespace

size_t gram_fp32_scratch_bytes(int64_t dS, int splits) {
  const int64_t nt = (dS + kTile - 1) / kTile;
  return size_t(splits) * nt * nt * kTile * kTile * sizeof(double) + size_t(nt * (nt + 1) / 2) * 8 + 512;
}

int gram_fp32_splits(gmgm_handle* h, const gmgm_matrix* m, int side) {
  const int64_t dS = side == GMGM_SIDE_COLS ? m->cols : m->rows;
  const int64_t K = side == GMGM_SIDE_COLS ? m->batch * m->rows : m->batch * m->cols;
  const int64_t nt = (dS + kTile - 1) / kTile;
  const int64_t tiles = nt * (nt + 1) / 2;
  int64_t want = (int64_t(h->num_sms) * 4 + tiles - 1) / tiles;
  want = std::max<int64_t>(1, std::min<int64_t>(want, (K + kChunk - 1) / kChunk));
  // cap FP64 partials at 1 GiB
  const int64_t per = nt * nt * kTile * kTile * 8;
  want = std::min<int64_t>(want, std::max<int64_t>(1, (int64_t(1) << 30) / per));
  return int(want);
}

cudaError_t launch_gram_fp32(gmgm_handle* h, const gmgm_matrix* m, int side, double* S,
                             int64_t lds, int accumulate, float* partials_f, int splits) {
  MView v;
  v.x = m->x;
  v.rows = m->rows;
  v.cols = m->cols;
  v.ld = m->ld;
  v.bs = m->batch_stride;
  v.side = side;
  v.dS = side == GMGM_SIDE_COLS ? m->cols : m->rows;
  v.K = side == GMGM_SIDE_COLS ? m->batch * m->rows : m->batch * m->cols;
  const int64_t nt = (v.dS + kTile - 1) / kTile;
  const int64_t ntiles = nt * (nt + 1) / 2;
  double* partials = reinterpret_cast<double*>(partials_f);
  // tile list after the partials (the scratch request leaves room)
  int2* tiles = reinterpret_cast<int2*>(partials + int64_t(splits) * nt * nt * kTile * kTile);
  make_tiles_kernel<<<1, 1, 0, h->stream>>>(tiles, int(nt));
  int64_t kps = (v.K + splits - 1) / splits;
  kps = ((kps + kBK - 1) / kBK) * kBK;
  dim3 grid((unsigned)ntiles, (unsigned)splits);
  gram_fp32_kernel<<<grid, 256, 0, h->stream>>>(v, kps, tiles, partials);
  dim3 cb(32, 8), cg(unsigned((v.dS + 31) / 32), unsigned((v.dS + 7) / 8));
  gram_combine_kernel<<<cg, cb, 0, h->stream>>>(partials, splits, v.dS, S, lds, accumulate);
  note_launch(3);
  return cudaGetLastError();
}

}  // namespace gmgm
