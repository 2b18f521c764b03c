// FP64 symmetric eigendecomposition on the GPU (the small axis Gram, e.g.
// 2000 x 2000 genes).  Steps:
//   1. Householder tridiagonalisation Q^T S Q = T, one cooperative kernel with
//      two bounded grid barriers per reflector (matrix in L2, FP64 bound);
//   2. bisection with Sturm counts for the wanted eigenvalues of T (one
//      thread per eigenvalue);
//   3. inverse iteration on T - lambda I (tridiagonal LU with partial
//      pivoting, one thread per eigenvalue), then modified Gram-Schmidt inside
//      clusters of nearly equal eigenvalues;
//   4. back-transformation Z <- Q Z (one warp per eigenvector, reflectors
//      streamed from L2);
//   5. output: the r largest eigenvalues descending, vectors row-major d x r.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>

#include "device.cuh"
#include "internal.cuh"

namespace gmgm {
namespace {

constexpr int kTriThreads = 256;
constexpr int kSeg = 128;  // columns per update segment

__global__ void copy_sym_kernel(const double* __restrict__ S, int64_t lds, int n, double* __restrict__ A) {
  const int64_t i = int64_t(blockIdx.y) * blockDim.y + threadIdx.y;
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n || j >= n) return;
  // lower triangle is authoritative
  A[i * n + j] = i >= j ? S[i * lds + j] : S[j * lds + i];
}

__global__ void __launch_bounds__(kTriThreads) tridiag_kernel(double* A, int n, double* dv, double* ev,
                                                              double* Vh, double* tau, double* P,
                                                              unsigned* bar, int* status) {
  extern __shared__ double sm[];
  double* v = sm;
  double* w = sm + n;
  __shared__ double red[33];
  const unsigned nb = gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int gwarp = blockIdx.x * nwarps + warp, total_warps = nb * nwarps;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    const double* rowk = A + int64_t(k) * n + k + 1;
    double ss = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      double t = __ldcg(rowk + i);
      v[i] = t;
      if (i > 0) ss += t * t;
    }
    const double tail = block_sum(ss, red);  // syncs: v visible
    const double x0 = v[0];
    double tk = 0.0, beta = x0;
    if (tail > 0.0) {
      const double nrm = sqrt(x0 * x0 + tail);
      beta = x0 >= 0.0 ? -nrm : nrm;
      tk = (beta - x0) / beta;
      const double sc = 1.0 / (x0 - beta);
      for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) v[i] *= sc;
    }
    __syncthreads();
    if (threadIdx.x == 0) v[0] = 1.0;
    __syncthreads();
    if (blockIdx.x == 0) {
      if (threadIdx.x == 0) {
        dv[k] = __ldcg(A + int64_t(k) * n + k);
        ev[k] = beta;
        tau[k] = tk;
      }
      for (int i = threadIdx.x; i < m; i += blockDim.x) Vh[int64_t(k) * n + k + 1 + i] = v[i];
    }
    if (tk == 0.0) continue;  // identical decision in every CTA (same data)
    // p = tau * A_sub v, one warp per row
    for (int i = gwarp; i < m; i += total_warps) {
      const double* row = A + int64_t(k + 1 + i) * n + k + 1;
      double s = 0.0;
      for (int j = lane; j < m; j += 32) s += __ldcg(row + j) * v[j];
      s = warp_sum(s);
      if (lane == 0) P[i] = tk * s;
    }
    if (!grid_barrier(bar, nb, status)) return;
    double pv = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) pv += __ldcg(P + i) * v[i];
    pv = block_sum(pv, red);
    const double K = 0.5 * tk * pv;
    for (int i = threadIdx.x; i < m; i += blockDim.x) w[i] = __ldcg(P + i) - K * v[i];
    __syncthreads();
    // A_sub -= v w^T + w v^T over (row, 128-column segment) work items
    const int segs = (m + kSeg - 1) / kSeg;
    const int64_t items = int64_t(m) * segs;
    for (int64_t it = gwarp; it < items; it += total_warps) {
      const int i = int(it / segs), sg = int(it - int64_t(i) * segs);
      double* row = A + int64_t(k + 1 + i) * n + k + 1;
      const double vi = v[i], wi = w[i];
      const int j1 = min(m, (sg + 1) * kSeg);
      for (int j = sg * kSeg + lane; j < j1; j += 32) row[j] = __ldcg(row + j) - (vi * w[j] + wi * v[j]);
    }
    if (!grid_barrier(bar, nb, status)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (n >= 2) {
      dv[n - 2] = __ldcg(A + int64_t(n - 2) * n + n - 2);
      ev[n - 2] = __ldcg(A + int64_t(n - 2) * n + n - 1);
    }
    dv[n - 1] = __ldcg(A + int64_t(n - 1) * n + n - 1);
  }
}

__global__ void tiny_tridiag_kernel(const double* A, int n, double* dv, double* ev) {
  dv[0] = A[0];
  if (n == 2) {
    dv[1] = A[3];
    ev[0] = A[1];
  }
}

// Gershgorin interval, squared off-diagonals and the pivot floor.
// info[0] = gl, info[1] = gu, info[2] = pivmin, info[3] = ||T|| estimate.
__global__ void tri_info_kernel(const double* dv, const double* ev, int n, double* e2, double* info) {
  __shared__ double red[33];
  double lo = 1e308, hi = -1e308, emax = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double el = i > 0 ? fabs(ev[i - 1]) : 0.0;
    const double er = i + 1 < n ? fabs(ev[i]) : 0.0;
    lo = fmin(lo, dv[i] - el - er);
    hi = fmax(hi, dv[i] + el + er);
    if (i + 1 < n) {
      e2[i] = ev[i] * ev[i];
      emax = fmax(emax, e2[i]);
    }
  }
  const double glo = -block_max(-lo, red);
  const double ghi = block_max(hi, red);
  const double em = block_max(emax, red);
  if (threadIdx.x == 0) {
    const double nrm = fmax(fabs(glo), fabs(ghi));
    const double pad = 2.0 * DBL_EPSILON * nrm * n + 1e-300;
    info[0] = glo - pad;
    info[1] = ghi + pad;
    info[2] = DBL_MIN * fmax(1.0, em);
    info[3] = nrm;
  }
}

// number of eigenvalues of T strictly below x (Sturm count of the LDL^T pivots)
__device__ __forceinline__ int sturm_count(const double* dv, const double* e2, int n, double x,
                                           double pivmin) {
  double q = dv[0] - x;
  int cnt = q < 0.0;
  if (fabs(q) < pivmin) q = -pivmin;
  for (int i = 1; i < n; ++i) {
    q = dv[i] - x - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// Thread t finds the ascending eigenvalue of index j0 + t by bisection.
__global__ void bisect_kernel(const double* __restrict__ dv_g, const double* __restrict__ e2_g, int n,
                              int j0, int cnt, const double* __restrict__ info, double* __restrict__ lam) {
  extern __shared__ double sm[];
  double* dv = sm;
  double* e2 = sm + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    dv[i] = dv_g[i];
    if (i + 1 < n) e2[i] = e2_g[i];
  }
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int j = j0 + t;
  const double pivmin = info[2];
  double lo = info[0], hi = info[1];
  for (int it = 0; it < 256; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 4.0 * pivmin || mid == lo || mid == hi)
      break;
    if (sturm_count(dv, e2, n, mid, pivmin) <= j)
      lo = mid;
    else
      hi = mid;
  }
  lam[t] = 0.5 * (lo + hi);
}

__device__ __forceinline__ double hash_unit(uint32_t a, uint32_t b) {
  uint32_t x = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  x ^= x >> 15;
  x *= 0x2C1B3C6Du;
  x ^= x >> 12;
  x *= 0x297A2D39u;
  x ^= x >> 15;
  return double(x) * (2.0 / 4294967296.0) - 1.0;  // [-1, 1)
}

// Inverse iteration: thread t (eigenvalue lam[t]) solves (T - lam I) z = y
// three times from a pseudo-random start.  Work arrays are interleaved
// [i][t] (stride B) so that a warp's accesses coalesce; z ends in Z[i*B + t].
__global__ void inverse_iter_kernel(const double* __restrict__ dv, const double* __restrict__ ev, int n,
                                    const double* __restrict__ lam, int cnt, int B,
                                    const double* __restrict__ info, double* __restrict__ u0,
                                    double* __restrict__ u1, double* __restrict__ u2,
                                    double* __restrict__ Z, int seed_base) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const double lm = lam[t];
  const double nrm = fmax(info[3], DBL_MIN);
  const double tiny = DBL_EPSILON * nrm;
  for (int i = 0; i < n; ++i) Z[int64_t(i) * B + t] = hash_unit(uint32_t(seed_base + t), uint32_t(i));
  for (int iter = 0; iter < 3; ++iter) {
    // factor with partial pivoting while applying L^-1 to the right-hand side
    double a = dv[0] - lm, b = n > 1 ? ev[0] : 0.0;
    double y = Z[t];  // current y_i (after elimination of previous rows)
    for (int i = 0; i + 1 < n; ++i) {
      const double c = ev[i];
      const double na = dv[i + 1] - lm;
      const double nb = i + 2 < n ? ev[i + 1] : 0.0;
      const double ynext = Z[int64_t(i + 1) * B + t];
      double yi, ynew;
      if (fabs(a) >= fabs(c)) {
        const double piv = fabs(a) < tiny ? (a < 0.0 ? -tiny : tiny) : a;
        const double l = c / piv;
        u0[int64_t(i) * B + t] = piv;
        u1[int64_t(i) * B + t] = b;
        u2[int64_t(i) * B + t] = 0.0;
        yi = y;
        ynew = ynext - l * y;
        a = na - l * b;
        b = nb;
      } else {
        const double l = a / c;
        u0[int64_t(i) * B + t] = c;
        u1[int64_t(i) * B + t] = na;
        u2[int64_t(i) * B + t] = nb;
        yi = ynext;
        ynew = y - l * ynext;
        a = b - l * na;
        b = -l * nb;
      }
      Z[int64_t(i) * B + t] = yi;
      y = ynew;
    }
    const double last = fabs(a) < tiny ? (a < 0.0 ? -tiny : tiny) : a;
    // back substitution, tracking the largest magnitude for scaling
    double z2 = 0.0, z1 = y / last;
    Z[int64_t(n - 1) * B + t] = z1;
    double zmax = fabs(z1);
    for (int i = n - 2; i >= 0; --i) {
      const double zi = (Z[int64_t(i) * B + t] - u1[int64_t(i) * B + t] * z1 - u2[int64_t(i) * B + t] * z2) /
                        u0[int64_t(i) * B + t];
      Z[int64_t(i) * B + t] = zi;
      z2 = z1;
      z1 = zi;
      zmax = fmax(zmax, fabs(zi));
    }
    // scale (keeps the next solve in range) and, on the last pass, normalise
    double s = 1.0 / fmax(zmax, DBL_MIN);
    if (iter == 2) {
      double nn = 0.0;
      for (int i = 0; i < n; ++i) {
        const double zi = Z[int64_t(i) * B + t] * s;
        nn += zi * zi;
      }
      s = s / sqrt(nn);
    }
    for (int i = 0; i < n; ++i) Z[int64_t(i) * B + t] *= s;
  }
}

// Z interleaved [i][t] (stride B) -> Zc eigenvector-major [t][i].
__global__ void transpose_kernel(const double* __restrict__ Z, int n, int cnt, int B,
                                 double* __restrict__ Zc, int t_off) {
  __shared__ double tile[32][33];
  const int t0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, t = t0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < n && t < cnt) ? Z[int64_t(i) * B + t] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int t = t0 + r, i = i0 + threadIdx.x;
    if (t < cnt && i < n) Zc[int64_t(t_off + t) * n + i] = tile[threadIdx.x][r];
  }
}

// Modified Gram-Schmidt (twice) inside clusters of consecutive eigenvalues
// closer than ctol * ||T||.  One CTA per potential cluster start.
__global__ void cluster_mgs_kernel(const double* __restrict__ lam, int cnt, const double* __restrict__ info,
                                   double ctol, int n, double* __restrict__ Zc) {
  __shared__ double red[33];
  const int s = blockIdx.x;
  const double thr = ctol * fmax(info[3], DBL_MIN);
  if (s > 0 && lam[s] - lam[s - 1] <= thr) return;  // not a cluster start
  int e = s + 1;
  while (e < cnt && lam[e] - lam[e - 1] <= thr) ++e;
  if (e - s < 2) return;
  for (int m = s + 1; m < e; ++m) {
    double* zm = Zc + int64_t(m) * n;
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = s; q < m; ++q) {
        const double* zq = Zc + int64_t(q) * n;
        double d = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) d += zm[i] * zq[i];
        d = block_sum(d, red);
        for (int i = threadIdx.x; i < n; i += blockDim.x) zm[i] -= d * zq[i];
        __syncthreads();
      }
    }
    double nn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) nn += zm[i] * zm[i];
    nn = block_sum(nn, red);
    const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) zm[i] *= inv;
    __syncthreads();
  }
}

// Z <- H_0 H_1 ... H_{n-3} Z, H_k = I - tau_k v_k v_k^T; one warp per
// eigenvector, the vector held in shared memory.
__global__ void back_transform_kernel(const double* __restrict__ Vh, const double* __restrict__ tau, int n,
                                      int cnt, double* __restrict__ Zc) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int t = blockIdx.x * nwarps + warp;
  if (t >= cnt) return;
  double* z = sm + int64_t(warp) * n;
  double* zg = Zc + int64_t(t) * n;
  for (int i = lane; i < n; i += 32) z[i] = zg[i];
  __syncwarp();
  for (int k = n - 3; k >= 0; --k) {
    const double tk = tau[k];
    if (tk == 0.0) continue;
    const double* vk = Vh + int64_t(k) * n;
    double y = 0.0;
    for (int i = k + 1 + lane; i < n; i += 32) y += __ldg(vk + i) * z[i];
    y = warp_sum(y) * tk;
    for (int i = k + 1 + lane; i < n; i += 32) z[i] -= y * __ldg(vk + i);
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) zg[i] = z[i];
}

// evals[c] = lam[cnt-1-c]; evecs[i*ldv + c] = Zc[(cnt-1-c)*n + i]
__global__ void output_kernel(const double* __restrict__ lam, const double* __restrict__ Zc, int n, int cnt,
                              double* __restrict__ evals, double* __restrict__ evecs, int64_t ldv) {
  __shared__ double tile[32][33];
  const int c0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  if (blockIdx.y == 0 && threadIdx.y == 0 && c0 + int(threadIdx.x) < cnt)
    evals[c0 + threadIdx.x] = lam[cnt - 1 - (c0 + threadIdx.x)];
  if (!evecs) return;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int c = c0 + r, i = i0 + threadIdx.x;
    tile[r][threadIdx.x] = (c < cnt && i < n) ? Zc[int64_t(cnt - 1 - c) * n + i] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, c = c0 + threadIdx.x;
    if (i < n && c < cnt) evecs[int64_t(i) * ldv + c] = tile[threadIdx.x][r];
  }
}

constexpr int kInvBatch = 1024;

struct EigScratch {
  double *A, *Vh, *tau, *dv, *ev, *e2, *P, *info, *lam, *u0, *u1, *u2, *Z, *Zc;
  size_t bytes;
};

EigScratch carve_eig(void* base, int64_t d, int32_t r) {
  Carve c(base);
  EigScratch s;
  const int64_t B = std::min<int64_t>(r, kInvBatch);
  s.A = c.take<double>(d * d);
  s.Vh = c.take<double>(d * d);
  s.tau = c.take<double>(d);
  s.dv = c.take<double>(d);
  s.ev = c.take<double>(d);
  s.e2 = c.take<double>(d);
  s.P = c.take<double>(d);
  s.info = c.take<double>(8);
  s.lam = c.take<double>(r);
  s.u0 = c.take<double>(d * B);
  s.u1 = c.take<double>(d * B);
  s.u2 = c.take<double>(d * B);
  s.Z = c.take<double>(d * B);
  s.Zc = c.take<double>(d * r);
  s.bytes = c.off + 256;
  return s;
}

}  // namespace

size_t eig_scratch_bytes(int64_t d, int32_t r) { return carve_eig(nullptr, d, r).bytes; }

cudaError_t launch_eig(gmgm_handle* h, int64_t d64, const double* S, int64_t lds, int32_t r, double* evals,
                       double* evecs, int64_t ldv, void* scratch) {
  const int n = int(d64);
  cudaStream_t st = h->stream;
  EigScratch s = carve_eig(scratch, d64, r);
  cudaError_t e;
  {
    dim3 b(32, 8), g(unsigned((n + 31) / 32), unsigned((n + 7) / 8));
    copy_sym_kernel<<<g, b, 0, st>>>(S, lds, n, s.A);
  }
  if ((e = cudaMemsetAsync(s.Vh, 0, size_t(n) * n * sizeof(double), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(s.tau, 0, size_t(n) * sizeof(double), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(s.ev, 0, size_t(n) * sizeof(double), st)) != cudaSuccess) return e;
  if (n >= 3) {
    const size_t smem = size_t(2) * n * sizeof(double);
    if ((e = cudaFuncSetAttribute(tridiag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) !=
        cudaSuccess)
      return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_kernel, kTriThreads, smem)) !=
        cudaSuccess)
      return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    unsigned blocks = unsigned(h->num_sms) * unsigned(std::min(per_sm, 2));
    // small problems: fewer CTAs (cheaper barriers)
    const unsigned want = unsigned((int64_t(n) * n + 16383) / 16384);
    blocks = std::min(blocks, std::max(1u, want));
    if ((e = cudaMemsetAsync(h->d_barrier, 0, 64, st)) != cudaSuccess) return e;
    double* A = s.A;
    double *dv = s.dv, *ev = s.ev, *Vh = s.Vh, *tau = s.tau, *P = s.P;
    unsigned* bar = h->d_barrier;
    int* status = h->d_status;
    int nn = n;
    void* args[] = {&A, &nn, &dv, &ev, &Vh, &tau, &P, &bar, &status};
    if ((e = cudaLaunchCooperativeKernel((void*)tridiag_kernel, dim3(blocks), dim3(kTriThreads), args, smem,
                                         st)) != cudaSuccess)
      return e;
  } else {
    // n = 1 or 2: already tridiagonal
    tiny_tridiag_kernel<<<1, 1, 0, st>>>(s.A, n, s.dv, s.ev);
  }
  tri_info_kernel<<<1, 256, 0, st>>>(s.dv, s.ev, n, s.e2, s.info);
  const int j0 = n - r;
  {
    const size_t smem = size_t(2) * n * sizeof(double);
    if ((e = cudaFuncSetAttribute(bisect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) !=
        cudaSuccess)
      return e;
    const int tpb = 64;
    bisect_kernel<<<unsigned((r + tpb - 1) / tpb), tpb, smem, st>>>(s.dv, s.e2, n, j0, r, s.info, s.lam);
  }
  const int B = std::min(r, kInvBatch);
  for (int t0 = 0; t0 < r; t0 += B) {
    const int cnt = std::min(B, r - t0);
    inverse_iter_kernel<<<unsigned((cnt + 63) / 64), 64, 0, st>>>(s.dv, s.ev, n, s.lam + t0, cnt, B, s.info,
                                                                   s.u0, s.u1, s.u2, s.Z, t0);
    dim3 tb(32, 8), tg(unsigned((cnt + 31) / 32), unsigned((n + 31) / 32));
    transpose_kernel<<<tg, tb, 0, st>>>(s.Z, n, cnt, B, s.Zc, t0);
  }
  cluster_mgs_kernel<<<unsigned(r), 256, 0, st>>>(s.lam, r, s.info, 1e-7, n, s.Zc);
  if (evecs) {
    int wpb = int(std::min<int64_t>(8, std::max<int64_t>(1, (200 * 1024) / (int64_t(n) * 8))));
    const size_t smem = size_t(wpb) * n * sizeof(double);
    if ((e = cudaFuncSetAttribute(back_transform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(smem))) != cudaSuccess)
      return e;
    back_transform_kernel<<<unsigned((r + wpb - 1) / wpb), wpb * 32, smem, st>>>(s.Vh, s.tau, n, r, s.Zc);
  }
  {
    dim3 b(32, 8), g(unsigned((r + 31) / 32), unsigned((n + 31) / 32));
    output_kernel<<<g, b, 0, st>>>(s.lam, s.Zc, n, r, evals, evecs, ldv);
  }
  note_launch(6 + 2 * ((r + B - 1) / B) + (evecs ? 1 : 0));
  return cudaGetLastError();
}

}  // namespace gmgm
