// Recomposition + per-row top-k, Psi = V diag(psi) V^T never materialised
// (Algorithm 1 last loop: threshold while recomposing).
//
// Every row is certified before it is trusted:
//   screen   per-row candidate lists of the kC largest screened |Psi_ij|,
//            j != i, over all columns: FP32 SIMT tiles here (the
//            tensor-core screens live in k_topk_tc.cu);
//   rescore  one warp per row recomputes every candidate in FP64 from V and
//            psi, sorts (|value| desc, column asc) and certifies the row: the
//            k-th exact value must exceed the best excluded screened value
//            plus a rigorous bound on the screen's error;
//   repair   rows that fail are scanned exactly in FP64, column-parallel
//            (a row's columns split over many CTAs, then merged).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstring>

#include "device.cuh"
#include "df.cuh"
#include "internal.cuh"
#include "topk_common.cuh"

namespace gmgm {
namespace {

constexpr int kBM = 128, kBN = 64, kBK = 32;

// A = fl32(V * psi), B = fl32(V), both d x rpad, zero padded; colmax_k =
// max_j |B_jk| as float bits (non-negative floats order like their bits).
__global__ void prep_ab_kernel(const void* V, int v64, int64_t ldv, const double* __restrict__ psi, int64_t d,
                               int r, int rpad, float* __restrict__ A, float* __restrict__ B) {
  const int64_t total = d * rpad;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / rpad;
    const int k = int(e - i * rpad);
    double v = 0.0;
    if (k < r)
      v = v64 ? static_cast<const double*>(V)[i * ldv + k] : double(static_cast<const float*>(V)[i * ldv + k]);
    A[e] = k < r ? float(v * psi[k]) : 0.f;
    B[e] = float(v);
  }
}

// Statistics of the screen's error bound, from b = float(V): colmax[k] =
// max_j |b_jk| (float bits) and colmax[r] = max_j ||b_j||_2, rounded up so
// the bound stays an upper bound.  A thread per row; column maxima reduced
// in shared memory, one global atomic per block and column.
__global__ void bound_stats_kernel(const void* V, int v64, int64_t ldv, int64_t d, int r,
                                   unsigned* __restrict__ colmax_bits) {
  extern __shared__ unsigned cm[];  // [r]
  for (int k = threadIdx.x; k < r; k += blockDim.x) cm[k] = 0u;
  __syncthreads();
  float best = 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < d; i += int64_t(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < r; ++k) {
      const float b = v64 ? float(static_cast<const double*>(V)[i * ldv + k]) : static_cast<const float*>(V)[i * ldv + k];
      s = fmaf(b, b, s);
      atomicMax(&cm[k], __float_as_uint(fabsf(b)));
    }
    best = fmaxf(best, s);
  }
  best = sqrtf(best) * (1.f + 1.2e-7f * float(r + 8));
  for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&colmax_bits[r], __float_as_uint(best));
  __syncthreads();
  for (int k = threadIdx.x; k < r; k += blockDim.x) atomicMax(&colmax_bits[k], cm[k]);
}

// FP32 screen.  Rows: rows[mi] for mi < m (m = *count_dev when count_dev is
// set, else m_host), or mi itself when rows is NULL.  Writes, per listed row
// position mi, cand_idx/cand_val [mi][kC] and thr[mi] (the kC-th screened
// value, or -1 when the row saw fewer than kC columns).
__global__ void __launch_bounds__(256) screen_fp32_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                          int64_t d, int rpad, const int* __restrict__ rows,
                                                          int64_t m_host, const int* __restrict__ count_dev,
                                                          int32_t* __restrict__ cand_idx,
                                                          float* __restrict__ cand_val, float* __restrict__ thr) {
  extern __shared__ float sm[];
  float* As = sm;                   // [kBK][kBM + 1]
  float* Bs = As + kBK * (kBM + 1); // [kBK][kBN + 1]
  float* T = Bs + kBK * (kBN + 1);  // [kBM][kBN + 1]
  float* lv = T + kBM * (kBN + 1);  // [kBM][kC]
  int* li = reinterpret_cast<int*>(lv + kBM * kC);
  __shared__ int64_t row_id[kBM];
  const int64_t m_rows = count_dev ? int64_t(*count_dev) : m_host;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t nblk = (m_rows + kBM - 1) / kBM;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t m0 = blk * kBM;
    for (int t = threadIdx.x; t < kBM; t += blockDim.x) {
      const int64_t mi = m0 + t;
      row_id[t] = mi < m_rows ? (rows ? int64_t(rows[mi]) : mi) : -1;
    }
    int cnt = 0, minpos = 0;
    float minv = -1.f;
    __syncthreads();
    for (int64_t j0 = 0; j0 < d; j0 += kBN) {
      float acc[8][4];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
      for (int k0 = 0; k0 < rpad; k0 += kBK) {
        for (int e = threadIdx.x; e < kBK * kBM; e += blockDim.x) {
          const int rr = e / kBK, kk = e - rr * kBK;  // consecutive threads -> consecutive k
          const int64_t gi = row_id[rr];
          As[kk * (kBM + 1) + rr] = gi >= 0 ? A[gi * rpad + k0 + kk] : 0.f;
        }
        for (int e = threadIdx.x; e < kBK * kBN; e += blockDim.x) {
          const int cc = e / kBK, kk = e - cc * kBK;
          const int64_t gj = j0 + cc;
          Bs[kk * (kBN + 1) + cc] = gj < d ? B[gj * rpad + k0 + kk] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kBK; ++kk) {
          float av[8], bv[4];
#pragma unroll
          for (int a = 0; a < 8; ++a) av[a] = As[kk * (kBM + 1) + ty * 8 + a];
#pragma unroll
          for (int b = 0; b < 4; ++b) bv[b] = Bs[kk * (kBN + 1) + tx * 4 + b];
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) T[(ty * 8 + a) * (kBN + 1) + tx * 4 + b] = acc[a][b];
      __syncthreads();
      if (threadIdx.x < kBM) {
        const int t = threadIdx.x;
        const int64_t gi = row_id[t];
        if (gi >= 0) {
          const int jn = d - j0 < kBN ? int(d - j0) : kBN;
          for (int c = 0; c < jn; ++c) {
            const int64_t j = j0 + c;
            if (j == gi) continue;
            const float v = fabsf(T[t * (kBN + 1) + c]);
            list_offer(lv + t * kC, li + t * kC, cnt, minv, minpos, v, int(j));
          }
        }
      }
      __syncthreads();
    }
    if (threadIdx.x < kBM) {
      const int t = threadIdx.x;
      const int64_t mi = m0 + t;
      if (mi < m_rows) {
        for (int c = 0; c < kC; ++c) {
          cand_idx[mi * kC + c] = c < cnt ? li[t * kC + c] : -1;
          cand_val[mi * kC + c] = c < cnt ? lv[t * kC + c] : -1.f;
        }
        thr[mi] = cnt >= kC ? minv : -1.f;
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ double vload(const void* V, int v64, int64_t idx) {
  return v64 ? static_cast<const double*>(V)[idx] : double(static_cast<const float*>(V)[idx]);
}

__device__ __forceinline__ bool better(double a, int ja, double b, int jb) { return a > b || (a == b && ja < jb); }

// (|value|, column) order on double-float magnitudes: larger first, then
// the lower column.
__device__ __forceinline__ bool df_better(dfl a, int ja, dfl b, int jb) {
  return a.h > b.h || (a.h == b.h && (a.l > b.l || (a.l == b.l && ja < jb)));
}

__device__ __forceinline__ dfl df_shfl(dfl a, int src) {
  return dfl{__shfl_sync(0xffffffffu, a.h, src), __shfl_sync(0xffffffffu, a.l, src)};
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// (screened value, column) order of the candidate merge; empty slots are
// (-1, INT_MAX) and sort last.
__device__ __forceinline__ bool fbetter(float a, int ja, float b, int jb) { return a > b || (a == b && ja < jb); }

// Bitonic sort of one (value, column) pair per lane across the warp,
// descending or ascending in fbetter order.
__device__ __forceinline__ void warp_sort_pairs(float& v, int& j, bool descending) {
  const int lane = threadIdx.x & 31;
  for (int size = 2; size <= 32; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, v, stride);
      const int oj = __shfl_xor_sync(0xffffffffu, j, stride);
      const bool desc = ((lane & size) == 0) == descending;
      const bool take_better = ((lane & stride) == 0) == desc;
      if (take_better != fbetter(v, j, ov, oj)) v = ov, j = oj;
    }
  }
}

// Bitonic merge of a bitonic sequence (one pair per lane) into descending
// fbetter order.
__device__ __forceinline__ void warp_merge_desc(float& v, int& j) {
  const int lane = threadIdx.x & 31;
  for (int stride = 16; stride > 0; stride >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, stride);
    const int oj = __shfl_xor_sync(0xffffffffu, j, stride);
    const bool take_better = (lane & stride) == 0;
    if (take_better != fbetter(v, j, ov, oj)) v = ov, j = oj;
  }
}

// One warp per listed row: exact FP64 values of the kC candidates, warp
// bitonic sort (|value| desc, column asc), certification, output.
// Candidate lists: nl = 1 (FP32 screen): cidx/cval[mi][kC], thr[mi];
// nl = 2 ncs (tensor-core screens: two column halves x ncs column slices):
// list l of row mi at [(l / 2) * lstride + mi][2 kC] + (l % 2) kC, its
// minimum at thr[((l / 2) * lstride + mi) * 2 + l % 2].  Several lists are
// merged pairwise, keeping the kC largest screened values (the running list
// descending, the next ascending, the larger of each lane's pair: a bitonic
// split), and every dropped value joins the row's threshold t: every column
// that is not rescored has a screened value <= t.
__global__ void rescore_kernel(int64_t d, int r, const void* V, int v64, int64_t ldv, const double* __restrict__ psi,
                               int k, const int* __restrict__ rows, int64_t m_host, const int* __restrict__ count_dev,
                               const int32_t* __restrict__ cidx, const float* __restrict__ cval,
                               const float* __restrict__ thr, int nl, int64_t lstride,
                               const unsigned* __restrict__ colmax_bits, double u, int32_t* __restrict__ idx_out,
                               float* __restrict__ val_out, int64_t orow0, int* __restrict__ flag_list,
                               int* __restrict__ flag_count, unsigned* __restrict__ err_bits) {
  extern __shared__ dfl rs_psi[];  // [r] psi as double-float, then [r] |psi| rounded up (FP32)
  float* psi_up = reinterpret_cast<float*>(rs_psi + r);
  for (int q = threadIdx.x; q < r; q += blockDim.x) {
    rs_psi[q] = df_from(psi[q]);
    psi_up[q] = __double2float_ru(fabs(psi[q]));
  }
  __syncthreads();
  const float u_up = __double2float_ru(u);
  const int lane = threadIdx.x & 31;
  const int64_t m = count_dev ? int64_t(*count_dev) : m_host;
  const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t mi = w0; mi < m; mi += nw) {
    const int64_t i = rows ? int64_t(rows[mi]) : mi;
    int j;
    float cv;
    float t;  // every input is an FP32 screened value: the maximum is exact in FP32
    if (nl == 1) {
      j = cidx[mi * kC + lane];
      cv = cval[mi * kC + lane];
      t = thr[mi];
    } else {
      t = -1.f;
      for (int l = 0; l < nl; ++l) {
        const int64_t pair = int64_t(l >> 1) * lstride + mi;
        const int64_t base = pair * (2 * kC) + (l & 1) * kC;
        int j2 = cidx[base + lane];
        float v2 = cval[base + lane];
        if (j2 < 0) v2 = -1.f, j2 = INT_MAX;
        t = fmaxf(t, thr[pair * 2 + (l & 1)]);
        if (l == 0) {
          cv = v2, j = j2;
          warp_sort_pairs(cv, j, true);
          continue;
        }
        warp_sort_pairs(v2, j2, false);
        const bool keep2 = fbetter(v2, j2, cv, j);
        const float dropped = keep2 ? cv : v2;
        if (keep2) cv = v2, j = j2;
        t = fmaxf(t, warp_max_f(dropped));
        if (l + 1 < nl) warp_merge_desc(cv, j);
      }
      if (j == INT_MAX) j = -1;
    }
    // exact value of the lane's candidate: an FP64 V in FP64; an FP32 V in
    // double-float (a_q = V_iq psi_q exact to 2^-48 from lane q % 32, the
    // products with V_jq and the sum by TwoProd/TwoSum).  Its error, about
    // 2^-46 of sum_q |a_q V_jq|, is far inside the slack of the screen bound.
    dfl ex = df_zero();
    if (v64) {
      double e = 0.0;
      const double* Vd = static_cast<const double*>(V);
      if (j >= 0)
        for (int q = 0; q < r; ++q) e += Vd[i * ldv + q] * psi[q] * Vd[int64_t(j) * ldv + q];
      ex = df_from(e);
    } else {
      const float* Vf = static_cast<const float*>(V);
      const float* vj = Vf + int64_t(j >= 0 ? j : 0) * ldv;
      for (int q0 = 0; q0 < r; q0 += 32) {
        const int qn = min(32, r - q0);
        const dfl aq = lane < qn ? df_mul(dfl{Vf[i * ldv + q0 + lane], 0.f}, rs_psi[q0 + lane]) : df_zero();
#pragma unroll 8
        for (int c = 0; c < qn; ++c) {
          const dfl a = df_shfl(aq, c);
          if (j >= 0) ex = df_fma(ex, a, dfl{vj[q0 + c], 0.f});
        }
      }
    }
    // self-check of the screen: |screened - |exact|| must stay within the bound
    const dfl aex = ex.h < 0.f ? df_neg(ex) : ex;
    const float serr = j >= 0 ? fabsf(__fsub_rn(cv, aex.h)) : 0.f;
    dfl key = j >= 0 ? aex : dfl{-1.f, 0.f};
    int kj = j >= 0 ? j : INT_MAX;
    float sv = ex.h;  // the nearest FP32 of the exact value
    for (int size = 2; size <= 32; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        const dfl ok = df_shfl_xor(key, stride);
        const int oj = __shfl_xor_sync(0xffffffffu, kj, stride);
        const float os = __shfl_xor_sync(0xffffffffu, sv, stride);
        const bool desc = (lane & size) == 0;
        const bool lower = (lane & stride) == 0;
        const bool take_better = lower == desc;
        const bool self_better = df_better(key, kj, ok, oj);
        if (take_better != self_better) key = ok, kj = oj, sv = os;
      }
    }
    // error bound of the screen for this row, rounded up in FP32
    // (sum_k |a_ik| max_j |b_jk|, or ||a_i|| max_j ||b_j|| by Cauchy-Schwarz;
    // colmax_bits[r] holds max_j ||b_j||)
    float bsum = 0.f, nsq = 0.f;
    for (int q = lane; q < r; q += 32) {
      const float vq = v64 ? __double2float_ru(fabs(static_cast<const double*>(V)[i * ldv + q]))
                           : fabsf(static_cast<const float*>(V)[i * ldv + q]);
      const float aq = __fmul_ru(vq, psi_up[q]);
      bsum = __fmaf_ru(aq, __uint_as_float(colmax_bits[q]), bsum);
      nsq = __fmaf_ru(aq, aq, nsq);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      bsum = __fadd_ru(bsum, __shfl_xor_sync(0xffffffffu, bsum, o));
      nsq = __fadd_ru(nsq, __shfl_xor_sync(0xffffffffu, nsq, o));
    }
    const float bnd = __fmul_ru(fminf(bsum, __fmul_ru(__fsqrt_ru(nsq), __uint_as_float(colmax_bits[r]))), u_up);
    {
      float ratio = bnd > 0.f ? serr / bnd : (serr > 0.f ? 1e30f : 0.f);
      ratio = warp_max_f(ratio);
      if (lane == 0 && ratio > 0.f) atomicMax(err_bits, __float_as_uint(fminf(ratio, 1e30f)));
    }
    // certified when the k-th exact value beats every column left out:
    // those have screened values <= t, exact values <= t + bnd
    const dfl qk = df_shfl(key, k - 1);
    const float rhs = __fadd_ru(t, bnd);
    const bool certified = t < 0.f || qk.h > rhs || (qk.h == rhs && qk.l > 0.f);
    if (lane < k) {
      idx_out[(i - orow0) * k + lane] = kj == INT_MAX ? -1 : kj;
      val_out[(i - orow0) * k + lane] = sv;
    }
    if (!certified && lane == 0) {
      const int pos = atomicAdd(flag_count, 1);
      flag_list[pos] = int(i);
    }
  }
}

constexpr int kExThreads = 256;

// Exact FP64 top-k of one (listed row, column chunk) work item per CTA:
// per-thread sorted lists, then k rounds of a block-wide arg-best over the
// list heads.  Writes the chunk's k best (value, column) to part[w][k].
__global__ void __launch_bounds__(kExThreads) exact_chunk_kernel(int64_t d, int r, const void* V, int v64, int64_t ldv,
                                                                  const double* __restrict__ psi, int k,
                                                                  const int* __restrict__ rows, int row0, int nb,
                                                                  int nchunks, int64_t chunk,
                                                                  double* __restrict__ part_v,
                                                                  int* __restrict__ part_j) {
  extern __shared__ double esm[];
  double* a = esm;                                         // [r]
  double* lvv = a + r;                                     // [threads][k]
  int* lj = reinterpret_cast<int*>(lvv + kExThreads * k);  // [threads][k]
  __shared__ double bkey[kExThreads];
  __shared__ int bj[kExThreads];
  __shared__ int bt[kExThreads];
  const int64_t items = int64_t(nb) * nchunks;
  for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
    const int rl = int(w / nchunks), ch = int(w - int64_t(rl) * nchunks);
    const int64_t i = rows[row0 + rl];
    for (int q = threadIdx.x; q < r; q += blockDim.x) a[q] = vload(V, v64, i * ldv + q) * psi[q];
    __syncthreads();
    double* mv = lvv + threadIdx.x * k;
    int* mj = lj + threadIdx.x * k;
    int cnt = 0;
    const int64_t jb = int64_t(ch) * chunk, je = jb + chunk < d ? jb + chunk : d;
    for (int64_t j = jb + threadIdx.x; j < je; j += blockDim.x) {
      if (j == i) continue;
      double ex = 0.0;
      for (int q = 0; q < r; ++q) ex += a[q] * vload(V, v64, j * ldv + q);
      const double ax = fabs(ex);
      int pos = cnt < k ? cnt : k;
      while (pos > 0 && better(ax, int(j), fabs(mv[pos - 1]), mj[pos - 1])) --pos;
      if (pos < k) {
        const int last = cnt < k ? cnt : k - 1;
        for (int q = last; q > pos; --q) mv[q] = mv[q - 1], mj[q] = mj[q - 1];
        mv[pos] = ex;
        mj[pos] = int(j);
        if (cnt < k) ++cnt;
      }
    }
    int head = 0;
    for (int out = 0; out < k; ++out) {
      bkey[threadIdx.x] = head < cnt ? fabs(mv[head]) : -1.0;
      bj[threadIdx.x] = head < cnt ? mj[head] : INT_MAX;
      bt[threadIdx.x] = threadIdx.x;
      __syncthreads();
      for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
          const int o = threadIdx.x + s;
          if (better(bkey[o], bj[o], bkey[threadIdx.x], bj[threadIdx.x]))
            bkey[threadIdx.x] = bkey[o], bj[threadIdx.x] = bj[o], bt[threadIdx.x] = bt[o];
        }
        __syncthreads();
      }
      if (threadIdx.x == bt[0]) {
        part_v[w * k + out] = head < cnt ? mv[head] : 0.0;
        part_j[w * k + out] = head < cnt ? mj[head] : -1;
        ++head;
      }
      __syncthreads();
    }
  }
}

// Merge the per-chunk lists of one listed row into its exact top-k.
__global__ void __launch_bounds__(kExThreads) exact_merge_kernel(const int* __restrict__ rows, int row0, int nchunks,
                                                                  int k, const double* __restrict__ part_v,
                                                                  const int* __restrict__ part_j,
                                                                  int32_t* __restrict__ idx_out,
                                                                  float* __restrict__ val_out, int64_t orow0) {
  extern __shared__ double msm[];
  const int rl = blockIdx.x;
  const int64_t i = rows[row0 + rl];
  const int m = nchunks * k;
  double* key = msm;                                // [m] |value|, -2 once taken
  int* col = reinterpret_cast<int*>(key + m);      // [m]
  __shared__ double bkey[kExThreads];
  __shared__ int bj[kExThreads];
  __shared__ int bp[kExThreads];
  const double* pv = part_v + int64_t(rl) * m;
  const int* pj = part_j + int64_t(rl) * m;
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    key[e] = pj[e] >= 0 ? fabs(pv[e]) : -1.0;
    col[e] = pj[e] >= 0 ? pj[e] : INT_MAX;
  }
  __syncthreads();
  for (int out = 0; out < k; ++out) {
    double bk = -3.0;
    int bc = INT_MAX, bpos = -1;
    for (int e = threadIdx.x; e < m; e += blockDim.x)
      if (better(key[e], col[e], bk, bc)) bk = key[e], bc = col[e], bpos = e;
    bkey[threadIdx.x] = bk;
    bj[threadIdx.x] = bc;
    bp[threadIdx.x] = bpos;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        const int o = threadIdx.x + s;
        if (better(bkey[o], bj[o], bkey[threadIdx.x], bj[threadIdx.x]))
          bkey[threadIdx.x] = bkey[o], bj[threadIdx.x] = bj[o], bp[threadIdx.x] = bp[o];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const int e = bp[0];
      const bool ok = e >= 0 && pj[e] >= 0;
      idx_out[(i - orow0) * k + out] = ok ? pj[e] : -1;
      val_out[(i - orow0) * k + out] = ok ? float(pv[e]) : 0.f;
      if (e >= 0) key[e] = -2.0;
    }
    __syncthreads();
  }
}

constexpr int64_t kExactCap = int64_t(1) << 22;  // partial entries held at once

}  // namespace

double screen_unit(gmgm_prec prec, int r) {
  const double u32 = 1.0 / 16777216.0;  // 2^-24
  const double kf = 1.02;               // slack over the first-order bound
  const double ub = 1.0 / 256.0;        // BF16 unit roundoff: 8 significant bits, 2^-8
  // FP32 SIMT: operand rounding (2u) + FMA accumulation of r terms (r u).
  // Tensor cores: both operands rounded to BF16 (2 ub + ub^2 per product)
  // + an accumulation of K products whose additions are each charged 2u
  // (the tensor core's internal alignment/rounding is not IEEE
  // round-to-nearest).  The split form (hi + lo, lo*lo dropped) would leave
  // 3 ub^2 per product.
  if (prec == GMGM_FP32) return kf * (double(r) + 4.0) * u32;
  if (prec == GMGM_BF16) return kf * (2.0 * ub + ub * ub + 2.0 * (double(r) + 4.0) * u32);
  return kf * (3.0 * ub * ub + 2.0 * (3.0 * double(r) + 4.0) * u32);
}

void launch_rescore(cudaStream_t s, int64_t d, int r, const void* V, int v64, int64_t ldv, const double* psi, int k,
                    const int* rows, const int* count_dev, const int32_t* cidx, const float* cval,
                    const float* thr, int nl, int64_t lstride, int64_t m, const unsigned* colmax_bits, double u,
                    int32_t* idx, float* val, int64_t orow0, int* flag_list, int* flag_count, unsigned* err_bits) {
  // one warp per row; the grid covers at most m rows (grid-stride beyond)
  const unsigned blocks = unsigned(std::min<int64_t>((m * 32 + 255) / 256, 4096));
  const size_t smem = size_t(r) * (sizeof(dfl) + sizeof(float));  // <= 96 KB (r <= 8192)
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(rescore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  rescore_kernel<<<blocks, 256, smem, s>>>(d, r, V, v64, ldv, psi, k, rows, m, count_dev, cidx, cval, thr, nl, lstride,
                                        colmax_bits, u, idx, val, orow0, flag_list, flag_count, err_bits);
}

// Exact FP64 top-k of the listed rows, column-parallel: a row's columns are
// split into chunks (one CTA each), then merged.  Batched so the partial
// lists stay within kExactCap entries.
int run_exact_rows(gmgm_handle* h, int64_t d, int r, const void* V, int v64, int64_t ldv, const double* psi, int k,
                   const int* rows, int nrows, double* part_v, int* part_j, int32_t* idx, float* val, int64_t orow0) {
  if (nrows <= 0) return GMGM_OK;
  const int64_t chunk = std::max<int64_t>(8192, (d + 255) / 256);
  const int nchunks = int((d + chunk - 1) / chunk);
  const int per_batch = int(std::max<int64_t>(1, std::min<int64_t>(nrows, kExactCap / (int64_t(nchunks) * k))));
  const size_t smem = size_t(r) * 8 + size_t(kExThreads) * k * 12;
  const size_t msmem = size_t(nchunks) * k * 12;
  GMGM_CUDA_TRY(h, cudaFuncSetAttribute(exact_chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  GMGM_CUDA_TRY(h, cudaFuncSetAttribute(exact_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(msmem)));
  for (int row0 = 0; row0 < nrows; row0 += per_batch) {
    const int nb = std::min(per_batch, nrows - row0);
    const unsigned grid = unsigned(std::min<int64_t>(int64_t(nb) * nchunks, int64_t(h->num_sms) * 8));
    exact_chunk_kernel<<<grid, kExThreads, smem, h->stream>>>(d, r, V, v64, ldv, psi, k, rows, row0, nb, nchunks,
                                                             chunk, part_v, part_j);
    exact_merge_kernel<<<unsigned(nb), kExThreads, msmem, h->stream>>>(rows, row0, nchunks, k, part_v, part_j, idx,
                                                                      val, orow0);
    note_launch(2);
  }
  GMGM_CUDA_TRY(h, cudaGetLastError());
  return GMGM_OK;
}

size_t topk_scratch_bytes(int64_t d, int32_t r, int32_t /*k*/, gmgm_prec prec) {
  const int64_t rpad = ((r + kBK - 1) / kBK) * kBK;
  size_t b = 0;
  b += Carve::round(size_t(d) * rpad * 4) * 2;  // A, B
  b += Carve::round(size_t(r + 1) * 4);         // colmax + max row norm
  b += Carve::round(size_t(d) * kC * 8) * 2;    // candidates (up to two lists per row)
  b += Carve::round(size_t(d) * 8);             // thresholds (one per list)
  b += Carve::round(size_t(d) * 4) * 2;         // flag lists (first screen, repair)
  b += Carve::round(size_t(kExactCap) * 12) + 256;  // exact partial lists
  b += Carve::round(64);                        // counters
  b += Carve::round(topk_tc_scratch_bytes(d, r, prec));
  b += Carve::round(size_t(d) * 4);             // row list of a block of rows
  return b + 4096;
}

__global__ void iota_kernel(int* __restrict__ out, int64_t m, int64_t base) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = int(base + i);
}

int topk_run(gmgm_handle* h, int64_t d, int32_t r, const void* V, int v_fp64, int64_t ldv, const double* psi,
             int32_t k, gmgm_prec prec, int32_t* idx, float* val, void* scratch, gmgm_topk_stats* st, int64_t row0,
             int64_t m) {
  cudaStream_t s = h->stream;
  const int rpad = ((r + kBK - 1) / kBK) * kBK;
  Carve c(scratch);
  float* A = c.take<float>(size_t(d) * rpad);
  float* B = c.take<float>(size_t(d) * rpad);
  unsigned* colmax = c.take<unsigned>(r + 1);  // [r] = max row norm
  // candidate lists per row: one from the FP32 screen, two (one per column
  // half of a tile) from the tensor-core screen
  const int nl = prec == GMGM_FP32 ? 1 : 2;
  int32_t* cidx = c.take<int32_t>(size_t(d) * kC * 2);
  float* cval = c.take<float>(size_t(d) * kC * 2);
  float* thr = c.take<float>(size_t(d) * 2);
  int* flag1 = c.take<int>(d);
  int* flag2 = c.take<int>(d);
  double* part_v = c.take<double>(kExactCap);
  int* part_j = c.take<int>(kExactCap);
  int* counters = c.take<int>(16);
  void* tc_scratch = c.take<char>(topk_tc_scratch_bytes(d, r, prec));
  // a block of rows: its rows listed (screens, rescoring and the exact scan
  // take row lists; outputs are written m x k from row row0)
  const bool block = m >= 0;
  if (!block) m = d;
  int* rowlist = block ? c.take<int>(size_t(m)) : nullptr;
  if (block)
    iota_kernel<<<unsigned(std::min<int64_t>((m + 255) / 256, 4096)), 256, 0, s>>>(rowlist, m, row0);
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  if (st)
    for (auto& e : ev) cudaEventCreate(&e);
  GMGM_CUDA_TRY(h, cudaMemsetAsync(colmax, 0, size_t(r + 1) * 4, s));
  GMGM_CUDA_TRY(h, cudaMemsetAsync(counters, 0, 64, s));
  {
    if (prec == GMGM_FP32) {
      // FP32 screen operands (the tensor-core screen prepares its own)
      const int64_t total = d * rpad;
      const unsigned blocks = unsigned(std::min<int64_t>((total + 255) / 256, int64_t(h->num_sms) * 16));
      prep_ab_kernel<<<blocks, 256, 0, s>>>(V, v_fp64, ldv, psi, d, r, rpad, A, B);
    }
    const unsigned nb = unsigned(std::min<int64_t>((d + 255) / 256, int64_t(h->num_sms) * 8));
    bound_stats_kernel<<<nb, 256, size_t(r) * sizeof(unsigned), s>>>(V, v_fp64, ldv, d, r, colmax);
  }
  if (st) cudaEventRecord(ev[0], s);
  const size_t smem = size_t(kBK * (kBM + 1) + kBK * (kBN + 1) + kBM * (kBN + 1) + kBM * kC) * 4 + size_t(kBM * kC) * 4;
  GMGM_CUDA_TRY(h, cudaFuncSetAttribute(screen_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const unsigned sblocks = unsigned(std::min<int64_t>((d + kBM - 1) / kBM, int64_t(h->num_sms) * 2));
  if (prec == GMGM_FP32) {
    screen_fp32_kernel<<<sblocks, 256, smem, s>>>(A, B, d, rpad, rowlist, m, nullptr, cidx, cval, thr);
  } else {
    GMGM_CUDA_TRY(h, launch_screen_tc(h, d, r, V, v_fp64, ldv, psi, prec, cidx, cval, thr, tc_scratch,
                                      block ? row0 : 0, m, rowlist,
                                      reinterpret_cast<unsigned long long*>(counters + 8)));
  }
  if (st) cudaEventRecord(ev[1], s);
  launch_rescore(s, d, r, V, v_fp64, ldv, psi, k, rowlist, nullptr, cidx, cval, thr, nl, m, m, colmax,
                 screen_unit(prec, r), idx, val, block ? row0 : 0, flag1, counters + 0,
                 reinterpret_cast<unsigned*>(counters + 2));
  note_launch(prec == GMGM_FP32 ? 4 : 2);
  // rows the screen could not certify (the count is read back once to size
  // the work): after the BF16 screen, a 3xBF16 tensor-core screen of those
  // rows and a second certification; what remains, an exact FP64 scan
  int nflag = 0, nexact = 0;
  GMGM_CUDA_TRY(h, cudaMemcpyAsync(&nflag, counters, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
  const int* exact_rows = flag1;
  nexact = nflag;
  if (prec == GMGM_BF16 && nflag > 0) {
    const int ncs = screen_tc_slices(nflag, h->num_sms, d);
    GMGM_CUDA_TRY(h, launch_screen_tc_repair(h, d, r, V, v_fp64, ldv, psi, flag1, nflag, ncs, cidx, cval, thr,
                                             tc_scratch));
    launch_rescore(s, d, r, V, v_fp64, ldv, psi, k, flag1, nullptr, cidx, cval, thr, 2 * ncs, nflag, nflag, colmax,
                   screen_unit(GMGM_BF16X3, r), idx, val, block ? row0 : 0, flag2, counters + 4,
                   reinterpret_cast<unsigned*>(counters + 2));
    note_launch(1);
    GMGM_CUDA_TRY(h, cudaMemcpyAsync(&nexact, counters + 4, sizeof(int), cudaMemcpyDeviceToHost, s));
    GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
    exact_rows = flag2;
  }
  int rc = run_exact_rows(h, d, r, V, v_fp64, ldv, psi, k, exact_rows, nexact, part_v, part_j, idx, val,
                          block ? row0 : 0);
  if (rc) return rc;
  if (st) cudaEventRecord(ev[2], s);
  GMGM_CUDA_TRY(h, cudaGetLastError());
  if (st) {
    unsigned hc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    GMGM_CUDA_TRY(h, cudaMemcpyAsync(hc, counters, 40, cudaMemcpyDeviceToHost, s));
    GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
    float t1 = 0.f, t2 = 0.f;
    cudaEventElapsedTime(&t1, ev[0], ev[1]);
    cudaEventElapsedTime(&t2, ev[1], ev[2]);
    float e1;
    memcpy(&e1, &hc[2], 4);
    st->rows_uncertified = int64_t(hc[0]);
    st->rows_exact = int64_t(nexact);
    st->candidates = int64_t(kC) * nl;
    st->screen_ms = t1;
    st->rescore_ms = t2;
    st->screen_err_ratio = double(e1);
    unsigned long long nrun;
    memcpy(&nrun, &hc[8], 8);
    st->screen_tiles = prec == GMGM_BF16 ? int64_t(nrun) : 0;
    st->screen_tiles_dense = prec == GMGM_BF16 ? ((m + 127) / 128) * ((d + 255) / 256) : 0;
    for (auto& e : ev) cudaEventDestroy(e);
  }
  return GMGM_OK;
}


// ---- square orthonormal V: split off c I --------------------------------------

namespace {

// c = min psi; the columns with psi_q > c in order (cols, psi_q - c), their
// count in *count.  One block.
__global__ void ortho_compact_kernel(const double* __restrict__ psi, int r, double* __restrict__ psi_free,
                                     int* __restrict__ cols, int* __restrict__ count) {
  __shared__ double red[33];
  __shared__ int base;
  double m = 1.0e308;
  for (int q = threadIdx.x; q < r; q += blockDim.x) m = fmin(m, psi[q]);
  const double c = -block_max(-m, red);
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int q0 = 0; q0 < r; q0 += blockDim.x) {
    const int q = q0 + threadIdx.x;
    const bool keep = q < r && psi[q] > c;
    // order-preserving compaction: warp ballots, then warps in order
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    __shared__ int wcount[32];
    if (lane == 0) wcount[threadIdx.x >> 5] = __popc(bal);
    __syncthreads();
    int before = base;
    for (int w = 0; w < int(threadIdx.x >> 5); ++w) before += wcount[w];
    if (keep) {
      const int pos = before + __popc(bal & ((1u << lane) - 1u));
      cols[pos] = q;
      psi_free[pos] = psi[q] - c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) t += wcount[w];
      base += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

__global__ void gather_cols_kernel(const void* V, int v64, int64_t ldv, int64_t d, const int* __restrict__ cols,
                                   int rf, double* __restrict__ Vf) {
  const int64_t total = d * rf;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / rf;
    const int q = int(e - i * rf);
    Vf[e] = vload(V, v64, i * ldv + cols[q]);
  }
}

// Every off-diagonal entry is exactly zero: the k lowest columns j != i
// (the tie rule), value 0.
__global__ void tie_rows_kernel(int64_t d, int k, int32_t* __restrict__ idx, float* __restrict__ val) {
  const int64_t total = d * k;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / k;
    const int c = int(e - i * k);
    idx[e] = int32_t(c < i ? c : c + 1);
    val[e] = 0.f;
  }
}

}  // namespace

namespace {

// ascending eigenvalue indices of the kept columns: cols[] holds descending-
// order indices q (ascending q); j = d - 1 - q, listed in ascending j
__global__ void gram_vlist_kernel(const int* __restrict__ cols, const int* __restrict__ count, int d,
                                  int* __restrict__ vlist) {
  const int n = *count;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
    vlist[t] = d - 1 - cols[n - 1 - t];
}

}  // namespace

size_t topk_gram_scratch_bytes(int64_t d, int32_t k, gmgm_prec prec) {
  // compaction buffers, the formed vectors (at most d), the eigensolver and
  // the network on the formed columns
  return Carve::round(size_t(d) * 8) + Carve::round(size_t(d) * 4) * 2 + Carve::round(64) +
         Carve::round(size_t(d) * d * 8) + eig_scratch_bytes(d, 0, int32_t(d)) +
         topk_scratch_bytes(d, int32_t(d), k, prec) + 4096;
}

int topk_run_gram(gmgm_handle* h, int64_t d, const double* S, int64_t lds, const double* psi, int32_t k,
                  gmgm_prec prec, int32_t* idx, float* val, void* scratch, gmgm_topk_stats* st) {
  cudaStream_t s = h->stream;
  const int n = int(d);
  Carve c(scratch);
  double* psif = c.take<double>(d);
  int* cols = c.take<int>(d);
  int* vlist = c.take<int>(d);
  int* cnt = c.take<int>(16);
  double* Vf = c.take<double>(size_t(d) * d);
  void* eig = c.take<char>(eig_scratch_bytes(d, 0, n));
  void* rest = c.take<char>(topk_scratch_bytes(d, n, k, prec));  // BF16 includes the tensor planes
  ortho_compact_kernel<<<1, 1024, 0, s>>>(psi, n, psif, cols, cnt);
  note_launch(1);
  int rf = 0;
  GMGM_CUDA_TRY(h, cudaMemcpyAsync(&rf, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
  if (rf == 0) {
    const unsigned blocks = unsigned(std::min<int64_t>((d * k + 255) / 256, int64_t(h->num_sms) * 8));
    tie_rows_kernel<<<blocks, 256, 0, s>>>(d, k, idx, val);
    note_launch(1);
    GMGM_CUDA_TRY(h, cudaGetLastError());
    if (st) {
      GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
      *st = gmgm_topk_stats{0, 0, 0, 0.0, 0.0, 0.0};
    }
    return GMGM_OK;
  }
  gram_vlist_kernel<<<unsigned((rf + 255) / 256), 256, 0, s>>>(cols, cnt, n, vlist);
  note_launch(1);
  // vectors for the kept eigenvalues, column t <-> cols[t] (descending order)
  GMGM_CUDA_TRY(h, launch_eig(h, d, S, lds, 0, nullptr, vlist, rf, Vf, rf, eig));
  const gmgm_prec p2 = prec == GMGM_BF16 && rf > 64 ? GMGM_FP32 : prec;
  return topk_run(h, d, rf, Vf, 1, rf, psif, k, p2, idx, val, rest, st);
}

size_t topk_ortho_scratch_bytes(int64_t d, int32_t r, int32_t k, gmgm_prec prec) {
  return Carve::round(size_t(d) * r * 8) + Carve::round(size_t(r) * 8) + Carve::round(size_t(r) * 4) +
         Carve::round(64) + topk_scratch_bytes(d, r, k, prec) + 4096;
}

int topk_run_ortho(gmgm_handle* h, int64_t d, int32_t r, const void* V, int v_fp64, int64_t ldv, const double* psi,
                   int32_t k, gmgm_prec prec, int32_t* idx, float* val, void* scratch, gmgm_topk_stats* st) {
  cudaStream_t s = h->stream;
  Carve c(scratch);
  double* Vf = c.take<double>(size_t(d) * r);
  double* psif = c.take<double>(r);
  int* cols = c.take<int>(r);
  int* cnt = c.take<int>(16);
  void* rest = c.take<char>(topk_scratch_bytes(d, r, k, prec));  // BF16 includes the tensor planes
  ortho_compact_kernel<<<1, 1024, 0, s>>>(psi, r, psif, cols, cnt);
  note_launch(1);
  int rf = 0;
  GMGM_CUDA_TRY(h, cudaMemcpyAsync(&rf, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
  if (rf == 0) {
    const unsigned blocks = unsigned(std::min<int64_t>((d * k + 255) / 256, int64_t(h->num_sms) * 8));
    tie_rows_kernel<<<blocks, 256, 0, s>>>(d, k, idx, val);
    note_launch(1);
    GMGM_CUDA_TRY(h, cudaGetLastError());
    if (st) {
      GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
      *st = gmgm_topk_stats{0, 0, 0, 0.0, 0.0, 0.0};
    }
    return GMGM_OK;
  }
  {
    const unsigned blocks = unsigned(std::min<int64_t>((d * rf + 255) / 256, int64_t(h->num_sms) * 16));
    gather_cols_kernel<<<blocks, 256, 0, s>>>(V, v_fp64, ldv, d, cols, rf, Vf);
    note_launch(1);
  }
  const gmgm_prec p2 = prec == GMGM_BF16 && rf > 64 ? GMGM_FP32 : prec;
  return topk_run(h, d, rf, Vf, 1, rf, psif, k, p2, idx, val, rest, st);
}

}  // namespace gmgm
