// Global top-n edges from the per-row top-k lists (Algorithm 1's last loop
// with the global threshold thresh_{n_l}: the complexity appendix keeps the
// n_l strongest edges with a heap of size n_l).  The per-row lists hold each
// row's k strongest off-diagonal entries; their union, as unordered pairs,
// contains the global top-n whenever every row's k-th magnitude lies
// strictly below the n-th magnitude of the union (a row cannot then hide an
// edge that strong outside its own list) -- the certificate returned with
// the edges.
//
// Steps (all on the device):
//   1. one canonical copy per unordered pair: the copy in the list of the
//      lower row; the higher row's copy is dropped when the lower row's list
//      holds the pair (a scan of that list, k entries);
//   2. the n-th largest magnitude T by a two-pass radix select over the FP32
//      magnitude bits (2^16-bin histograms of the high, then the low half);
//   3. every pair with magnitude >= T compacted (fewer than n above T, the
//      ties at T with them);
//   4. those sorted by (magnitude descending, lower row, higher row) with a
//      bitonic network, the first n kept;
//   5. the certificate: the largest k-th magnitude of any row < T.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "device.cuh"
#include "internal.cuh"

namespace gmgm {
namespace {

constexpr int kBins = 1 << 16;

struct Edge {
  unsigned mag;  // FP32 bits of |value| (order-preserving for non-negative floats)
  int a, b;      // a < b
  float v;
};

__device__ __forceinline__ bool edge_before(const Edge& x, const Edge& y) {
  if (x.mag != y.mag) return x.mag > y.mag;
  if (x.a != y.a) return x.a < y.a;
  return x.b < y.b;
}

// mag[e] = |val| bits of a canonical list entry, 0xffffffff for a dropped or
// empty one.
__global__ void canon_kernel(int64_t d, int k, const int32_t* __restrict__ idx, const float* __restrict__ val,
                             unsigned* __restrict__ mag) {
  const int64_t total = d * k;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / k;
    const int j = idx[e];
    unsigned m = 0xffffffffu;
    if (j >= 0 && j < d && j != i) {
      bool keep = true;
      if (j < i)
        for (int s = 0; s < k; ++s)
          if (idx[int64_t(j) * k + s] == int(i)) keep = false;
      if (keep) m = __float_as_uint(fabsf(val[e]));
    }
    mag[e] = m;
  }
}

// Histogram of the high (shift 16) or, among entries whose high half is
// `hi_sel`, the low half of the magnitude bits.
__global__ void hist_kernel(const unsigned* __restrict__ mag, int64_t total, int shift, unsigned hi_sel,
                            unsigned* __restrict__ hist) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const unsigned m = mag[e];
    if (m == 0xffffffffu) continue;
    if (shift == 16)
      atomicAdd(hist + (m >> 16), 1u);
    else if ((m >> 16) == hi_sel)
      atomicAdd(hist + (m & 0xffffu), 1u);
  }
}

// One CTA: walking the bins from the top, the bin holding the `need`-th
// largest entry; out[0] = that bin, out[1] = entries in higher bins.
__global__ void select_bin_kernel(const unsigned* __restrict__ hist, unsigned long long need,
                                  unsigned long long* __restrict__ out) {
  __shared__ unsigned long long part[256];
  const int t = threadIdx.x;  // 256 threads, 256 bins each, thread t owns the t-th highest range
  const int hi_bin = kBins - 1 - t * 256;
  unsigned long long s = 0;
  for (int q = 0; q < 256; ++q) s += hist[hi_bin - q];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    unsigned long long acc = 0;
    int owner = -1;
    for (int u = 0; u < 256; ++u) {
      if (acc + part[u] >= need) {
        owner = u;
        break;
      }
      acc += part[u];
    }
    if (owner < 0) {  // fewer entries than need: the lowest bin, all above
      out[0] = 0;
      out[1] = acc;
      return;
    }
    const int top = kBins - 1 - owner * 256;
    for (int q = 0; q < 256; ++q) {
      const unsigned c = hist[top - q];
      if (acc + c >= need) {
        out[0] = unsigned(top - q);
        out[1] = acc;
        return;
      }
      acc += c;
    }
  }
}

// Compact the canonical entries with magnitude >= thr into `cand`.
__global__ void compact_kernel(int64_t d, int k, const int32_t* __restrict__ idx, const float* __restrict__ val,
                               const unsigned* __restrict__ mag, unsigned thr, Edge* __restrict__ cand,
                               unsigned long long* __restrict__ count, unsigned long long cap) {
  const int64_t total = d * k;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const unsigned m = mag[e];
    if (m == 0xffffffffu || m < thr) continue;
    const unsigned long long pos = atomicAdd(count, 1ull);
    if (pos >= cap) continue;
    const int i = int(e / k), j = idx[e];
    cand[pos] = Edge{m, min(i, j), max(i, j), val[e]};
  }
}

__global__ void pad_kernel(Edge* __restrict__ cand, unsigned long long from, unsigned long long to) {
  for (unsigned long long e = from + blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; e < to;
       e += uint64_t(gridDim.x) * blockDim.x)
    cand[e] = Edge{0u, INT_MAX, INT_MAX, 0.f};  // sorts after every real edge
}

// One compare-exchange step (size, stride) of a bitonic sort, ascending in
// edge_before order.
__global__ void bitonic_step_kernel(Edge* __restrict__ a, unsigned long long m, unsigned long long size,
                                    unsigned long long stride) {
  for (unsigned long long t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < m / 2;
       t += uint64_t(gridDim.x) * blockDim.x) {
    const unsigned long long lo = (t / stride) * 2 * stride + (t % stride);
    const unsigned long long hi = lo + stride;
    const bool up = (lo & size) == 0;
    Edge x = a[lo], y = a[hi];
    if (edge_before(y, x) == up) {
      a[lo] = y;
      a[hi] = x;
    }
  }
}

__global__ void emit_kernel(const Edge* __restrict__ cand, int64_t n, int32_t* __restrict__ io,
                            int32_t* __restrict__ jo, float* __restrict__ vo) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    io[e] = cand[e].a;
    jo[e] = cand[e].b;
    vo[e] = cand[e].v;
  }
}

// Largest k-th magnitude over the rows (FP32 bits).
__global__ void kth_max_kernel(int64_t d, int k, const float* __restrict__ val, unsigned* __restrict__ out) {
  unsigned m = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < d; i += int64_t(gridDim.x) * blockDim.x)
    m = max(m, __float_as_uint(fabsf(val[i * k + (k - 1)])));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Candidate capacity: room for 2n + 2 pairs, or (for ties at the n-th
// magnitude) for every entry of up to 2^22 list entries.
unsigned long long topn_cap(int64_t d, int32_t k, int64_t n) {
  const unsigned long long want =
      std::max<unsigned long long>(2ull * uint64_t(n) + 2, std::min<unsigned long long>(uint64_t(d) * k, 1ull << 22));
  unsigned long long m2 = 1;
  while (m2 < want) m2 <<= 1;
  return m2;
}

}  // namespace

size_t topn_scratch_bytes(int64_t d, int32_t k, int64_t n) {
  const unsigned long long m2 = topn_cap(d, k, n);
  return Carve::round(size_t(d) * k * 4) + Carve::round(size_t(kBins) * 4) + Carve::round(64) +
         Carve::round(size_t(m2) * sizeof(Edge)) + 4096;
}

int topn_run(gmgm_handle* h, int64_t d, int32_t k, const int32_t* idx, const float* val, int64_t n, int32_t* io,
             int32_t* jo, float* vo, int64_t* count_out, int* certified_out) {
  cudaStream_t s = h->stream;
  const int64_t total = d * k;
  Carve c(h->scratch);
  unsigned* mag = c.take<unsigned>(size_t(total));
  unsigned* hist = c.take<unsigned>(kBins);
  unsigned long long* misc = c.take<unsigned long long>(8);  // [0..1] select, [2] count, [3] kth
  // ties at the threshold beyond the capacity make the call fail loudly
  const unsigned long long cap = topn_cap(d, k, n);
  Edge* cand = c.take<Edge>(size_t(cap));
  const unsigned blocks = unsigned(std::min<int64_t>((total + 255) / 256, int64_t(h->num_sms) * 16));
  canon_kernel<<<blocks, 256, 0, s>>>(d, k, idx, val, mag);
  GMGM_CUDA_TRY(h, cudaMemsetAsync(hist, 0, kBins * 4, s));
  GMGM_CUDA_TRY(h, cudaMemsetAsync(misc, 0, 64, s));
  hist_kernel<<<blocks, 256, 0, s>>>(mag, total, 16, 0, hist);
  select_bin_kernel<<<1, 256, 0, s>>>(hist, uint64_t(n), misc);
  unsigned long long sel[2];
  GMGM_CUDA_TRY(h, cudaMemcpyAsync(sel, misc, 16, cudaMemcpyDeviceToHost, s));
  GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
  const unsigned hi = unsigned(sel[0]);
  GMGM_CUDA_TRY(h, cudaMemsetAsync(hist, 0, kBins * 4, s));
  hist_kernel<<<blocks, 256, 0, s>>>(mag, total, 0, hi, hist);
  // sel[1] < n entries lie in higher bins, so the n-th is the
  // (n - sel[1])-th of this one (or, with fewer than n entries, the last)
  select_bin_kernel<<<1, 256, 0, s>>>(hist, sel[1] < uint64_t(n) ? uint64_t(n) - sel[1] : 1ull, misc);
  GMGM_CUDA_TRY(h, cudaMemcpyAsync(sel, misc, 16, cudaMemcpyDeviceToHost, s));
  GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
  const unsigned thr = (hi << 16) | unsigned(sel[0]);
  compact_kernel<<<blocks, 256, 0, s>>>(d, k, idx, val, mag, thr, cand, misc + 2, cap);
  unsigned long long m = 0;
  GMGM_CUDA_TRY(h, cudaMemcpyAsync(&m, misc + 2, 8, cudaMemcpyDeviceToHost, s));
  GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
  if (m > cap)
    return fail(h, GMGM_E_CAND_OVERFLOW, "gmgm_topn_edges: too many pairs tie at the n-th magnitude");
  unsigned long long m2 = 1;
  while (m2 < m) m2 <<= 1;
  if (m2 > m) pad_kernel<<<unsigned(std::min<unsigned long long>((m2 - m + 255) / 256, 4096)), 256, 0, s>>>(cand, m, m2);
  const unsigned sb = unsigned(std::min<unsigned long long>((m2 / 2 + 255) / 256, uint64_t(h->num_sms) * 16));
  int launches = 0;
  for (unsigned long long size = 2; size <= m2; size <<= 1)
    for (unsigned long long stride = size >> 1; stride > 0; stride >>= 1, ++launches)
      bitonic_step_kernel<<<std::max(sb, 1u), 256, 0, s>>>(cand, m2, size, stride);
  const int64_t cnt = std::min<int64_t>(int64_t(m), n);
  if (cnt > 0) emit_kernel<<<unsigned(std::min<int64_t>((cnt + 255) / 256, 4096)), 256, 0, s>>>(cand, cnt, io, jo, vo);
  kth_max_kernel<<<unsigned(std::min<int64_t>((d + 255) / 256, int64_t(h->num_sms) * 4)), 256, 0, s>>>(
      d, k, val, reinterpret_cast<unsigned*>(misc + 3));
  unsigned kth = 0;
  GMGM_CUDA_TRY(h, cudaMemcpyAsync(&kth, misc + 3, 4, cudaMemcpyDeviceToHost, s));
  GMGM_CUDA_TRY(h, cudaStreamSynchronize(s));
  note_launch(8 + launches + (m2 > m ? 1 : 0));
  GMGM_CUDA_TRY(h, cudaGetLastError());
  *count_out = cnt;
  // certified: n distinct pairs and no row's list stops at or above the n-th
  // magnitude (or every list holds all d - 1 columns)
  *certified_out = cnt == n && (int64_t(k) == d - 1 || kth < thr) ? 1 : 0;
  return GMGM_OK;
}

}  // namespace gmgm
