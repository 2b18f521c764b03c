// Symmetric eigendecomposition of an FP64 matrix on the GPU (the small axis
// Gram, e.g. 2000 x 2000 genes), to about 1e-14 of its largest eigenvalue.
// Steps:
//   1. Householder tridiagonalisation Q^T S Q = T in double-float (FP32
//      pairs, the matrix scaled by a power of two), one cooperative kernel
//      with one bounded grid barrier per reflector (matrix in L2);
//   2. multisection with division-free double-float Sturm counts for the
//      wanted eigenvalues of T (sixteen lanes per eigenvalue);
//   3. inverse iteration on T - lambda I (tridiagonal LU with partial
//      pivoting, one thread per eigenvalue, double-float, work arrays in
//      shared memory when they fit), then modified
//      Gram-Schmidt inside clusters of nearly equal eigenvalues;
//   4. back-transformation Z <- Q Z in compact WY blocks of 32 reflectors
//      (one cooperative kernel over every SM, one grid barrier per block);
//   5. output: the r largest eigenvalues descending, vectors row-major d x r.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>

#include "device.cuh"
#include "df.cuh"
#include "internal.cuh"

namespace gmgm {
namespace {

constexpr int kTriThreads = 512;
constexpr int kBatch = 8;     // independent row loads per lane in flight
constexpr int kInvIters = 2;  // inverse-iteration solves (bisection eigenvalues are accurate to ~eps)

// max |S_ij| over the lower triangle, as the bits of a non-negative double
// (ordered like the values), into *amax (zeroed before).
__global__ void absmax_kernel(const double* __restrict__ S, int64_t lds, int n, unsigned long long* amax) {
  unsigned long long m = 0;
  const int64_t total = int64_t(n) * n;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    if (j <= i) m = max(m, static_cast<unsigned long long>(__double_as_longlong(fabs(S[i * lds + j]))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(amax, m);
}

// Exponent e with max |S| = f 2^e, f in [0.5, 1): the matrix is reduced as
// 2^-e S (exact), so the double-float entries stay far from the FP32
// overflow and underflow thresholds; 0 for a zero or non-finite maximum.
__device__ __forceinline__ int scale_exp(const unsigned long long* amax) {
  const double smax = __longlong_as_double(static_cast<long long>(*amax));
  if (!(smax > 0.0) || !isfinite(smax)) return 0;
  int e;
  frexp(smax, &e);
  return e;
}

__global__ void copy_sym_kernel(const double* __restrict__ S, int64_t lds, int n,
                                const unsigned long long* __restrict__ amax, dfl* __restrict__ A) {
  const int64_t i = int64_t(blockIdx.y) * blockDim.y + threadIdx.y;
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n || j >= n) return;
  const double sc = ldexp(1.0, -scale_exp(amax));
  // lower triangle is authoritative
  A[i * n + j] = df_from((i >= j ? S[i * lds + j] : S[j * lds + i]) * sc);
}

// Householder of x (length m, in smem): v (v[0] = 1) and tau with
// (I - tau v v^T) x = beta e_0.  Every CTA runs it on identical data, all
// in double-float: every warp evaluates the scalars, and on this part a
// warp's FP64 instruction costs dozens of FP32 ones.
__device__ __forceinline__ void householder(dfl* x, int m, dfl* red, dfl& tau, dfl& beta) {
  dfl ss = df_zero();
  for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) ss = df_fma(ss, x[i], x[i]);
  const dfl tail = df_block_sum(ss, red);
  const dfl x0 = x[0];
  tau = df_zero();
  beta = x0;
  if (tail.h > 0.f) {
    const dfl nrm = df_sqrt(df_fma(tail, x0, x0));
    beta = x0.h >= 0.f ? df_neg(nrm) : nrm;
    tau = df_div(df_add(beta, df_neg(x0)), beta);
    const dfl sc = df_div(dfl{1.f, 0.f}, df_add(x0, df_neg(beta)));
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) x[i] = df_mul(x[i], sc);
  }
  __syncthreads();
  if (threadIdx.x == 0) x[0] = dfl{1.f, 0.f};
  __syncthreads();
}

// The scalars of the Householder reflector of x = (x0, x1..): tau, beta and
// the scale sc of x1.. (v = (1, sc x1, ...)), from x0 and the squared tail
// sum_{i>=1} x_i^2.  False when the tail is zero (tau = 0, no scaling).
__device__ __forceinline__ bool reflector_scalars(dfl x0, dfl tail, dfl& tau, dfl& beta, dfl& sc) {
  tau = df_zero();
  beta = x0;
  sc = dfl{1.f, 0.f};
  if (!(tail.h > 0.f)) return false;
  const dfl nrm = df_sqrt(df_fma(tail, x0, x0));
  beta = x0.h >= 0.f ? df_neg(nrm) : nrm;
  tau = df_div(df_add(beta, df_neg(x0)), beta);
  sc = df_div(dfl{1.f, 0.f}, df_add(x0, df_neg(beta)));
  return true;
}

// acc += a b with the sum kept as an unnormalised pair (s, t): s the exact
// running sum of the high products (TwoSum), t the FP32 sum of every
// low-order term; renormalised once at the end (df_renorm(s, t)).  Six
// FP32 operations fewer than df_fma per term; with at most a few dozen
// terms per pair t stays within a few ulp(s), so the FP32 rounding of t is
// far below the double-float unit.
__device__ __forceinline__ void df_fma_acc(float& s, float& t, dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  float s2, t2;
  two_sum(s, p, s2, t2);
  s = s2;
  t = __fadd_rn(t, __fadd_rn(t2, e));
}

// Tridiagonalisation with one grid barrier per reflector: the rank-2 update
// of step k and the mat-vec of step k+1 share one pass over the trailing
// matrix.  Row k+1 of the updated matrix (which defines reflector k+1) is
// formed redundantly by every CTA from row k+1 of the old matrix.
//   v = reflector k (rows/cols k+1..n-1), u = reflector k+1 (k+2..n-1),
//   P = tau_{k+1} A_{k+1} u (written by row owners, read after the barrier;
//   double-buffered so a CTA still reading step k's P never sees step k+1's).
// The matrix, the reflectors and P are double-float (FP32 pipe); the
// reflectors' scalars are FP64.  Outputs: T's diagonal dv and off-diagonal
// ev (scaled back by 2^e, exact), tau, and the reflectors in Vh (FP64, the
// exact values of the double-float vectors the reduction applied).
__global__ void __launch_bounds__(kTriThreads) tridiag_kernel(dfl* A, int n, const unsigned long long* amax,
                                                              double* dv, double* ev, double* Vh, double* tau_out,
                                                              dfl* P, unsigned* bar, int* status) {
  extern __shared__ dfl tri_sm[];
  dfl* v = tri_sm;          // [n]
  dfl* w = tri_sm + n;      // [n]
  dfl* u = tri_sm + 2 * n;  // [n]
  __shared__ dfl red[33];
  const unsigned nb = gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // rows go to CTAs round-robin first (row i: CTA i mod nb), so every SM
  // streams its share of a short trailing block too
  const int gwarp = warp * int(nb) + blockIdx.x, total_warps = nb * nwarps;
  const int gthread = blockIdx.x * blockDim.x + threadIdx.x, total_threads = nb * blockDim.x;
  const double unscale = ldexp(1.0, scale_exp(amax));
  unsigned epoch = 0;  // grid barriers passed
  // prologue: reflector 0 from row 0, P = tau_0 A[1:,1:] v
  dfl tk, beta;
  {
    const int m = n - 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const float2 a = __ldcg(reinterpret_cast<const float2*>(A) + 1 + i);
      v[i] = dfl{a.x, a.y};
    }
    __syncthreads();
    householder(v, m, red, tk, beta);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const float2 a00 = __ldcg(reinterpret_cast<const float2*>(A));
      dv[0] = df_val(dfl{a00.x, a00.y}) * unscale;
      ev[0] = df_val(beta) * unscale;
      tau_out[0] = df_val(tk);
    }
    for (int i = gthread; i < m; i += total_threads) Vh[1 + i] = df_val(v[i]);
    const dfl td = tk;
    for (int i = gwarp; i < m; i += total_warps) {
      const float2* row = reinterpret_cast<const float2*>(A) + int64_t(1 + i) * n + 1;
      dfl acc[kBatch];
#pragma unroll
      for (int q = 0; q < kBatch; ++q) acc[q] = df_zero();
      for (int j0 = lane; j0 < m; j0 += 32 * kBatch) {
        float2 a[kBatch];
#pragma unroll
        for (int q = 0; q < kBatch; ++q) a[q] = j0 + 32 * q < m ? __ldcg(row + j0 + 32 * q) : make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < kBatch; ++q)
          if (j0 + 32 * q < m) acc[q] = df_fma(acc[q], dfl{a[q].x, a[q].y}, v[j0 + 32 * q]);
      }
#pragma unroll
      for (int q = 1; q < kBatch; ++q) acc[0] = df_add(acc[0], acc[q]);
      const dfl s = df_warp_sum(acc[0]);
      if (lane == 0) P[i] = df_mul(td, s);
    }
    if (!grid_barrier(bar, nb, epoch, status)) return;
  }
  // Reflector k lives at vb (vb[0] == 1); row k+1 and then reflector k+1 are
  // formed in the other buffer ub, so the next reflector is ub + 1 and the
  // buffer of the current one takes the next row: no copy.
  __shared__ dfl xs0;  // entry k+2 of the updated row k+1 (x0 of reflector k+1)
  dfl* vb = v;
  dfl* ub = u;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // size of the trailing block of step k
    const dfl* Pc = P + (k & 1) * int64_t(n);
    dfl* Pn = P + ((k + 1) & 1) * int64_t(n);
    const float2* rowk = reinterpret_cast<const float2*>(A) + int64_t(k + 1) * n + k + 1;
    // one round trip to L2: P into w, row k+1 of the old matrix into ub
    const float2 p0 = __ldcg(reinterpret_cast<const float2*>(Pc));
    dfl pv = df_zero();
#pragma unroll 4
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const float2 pc = __ldcg(reinterpret_cast<const float2*>(Pc) + i);
      const float2 a = __ldcg(rowk + i);
      w[i] = dfl{pc.x, pc.y};
      ub[i] = dfl{a.x, a.y};
      pv = df_fma(pv, w[i], vb[i]);
    }
    const bool live = tk.h != 0.f;  // reflector k is not the identity
    const dfl nK = df_mul(dfl{-0.5f * tk.h, -0.5f * tk.l}, df_block_sum(pv, red));  // -tau_k (P.v) / 2
    // w = P - K v, the updated row k+1 (u = row - v0 w - w0 v) and the
    // squared tail of reflector k+1's x = u[1..]; each thread touches its
    // own indices of w and ub
    const dfl v0 = vb[0];
    const dfl w0 = live ? df_fma(dfl{p0.x, p0.y}, nK, v0) : df_zero();
    dfl ss = df_zero();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const dfl wi = live ? df_fma(w[i], nK, vb[i]) : df_zero();
      w[i] = wi;
      const dfl ui = df_sub2(ub[i], v0, wi, w0, vb[i]);
      ub[i] = ui;
      if (i >= 2) ss = df_fma(ss, ui, ui);
      if (i == 1) xs0 = ui;
    }
    const dfl tail = df_block_sum(ss, red);  // ub, w and xs0 complete after its barriers
    const dfl dnext = ub[0];
    dfl tn = df_zero(), bn = xs0;
    const bool more = k + 3 < n;  // a reflector k+1 exists
    if (more) {
      dfl sc;
      if (reflector_scalars(xs0, tail, tn, bn, sc))
        for (int i = 2 + threadIdx.x; i < m; i += blockDim.x) ub[i] = df_mul(ub[i], sc);
      if (threadIdx.x == 0) ub[1] = dfl{1.f, 0.f};
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      dv[k + 1] = df_val(dnext) * unscale;
      ev[k + 1] = df_val(bn) * unscale;
      if (more) tau_out[k + 1] = df_val(tn);
    }
    __syncthreads();
    const dfl* uu = ub;  // u[1..]: reflector k+1
    if (more)
      for (int i = gthread; i < m - 1; i += total_threads) Vh[int64_t(k + 1) * n + k + 2 + i] = df_val(uu[1 + i]);
    // fused pass: rows i, cols j in k+2..n-1 (local index t = i - (k+1) >= 1)
    const bool upd = live;
    const dfl tnd = tn;
    for (int it = gwarp; it < (m - 1); it += total_warps) {
      const int t = 1 + it;
      float2* row = reinterpret_cast<float2*>(A) + int64_t(k + 1 + t) * n + k + 2;
      const dfl vi = vb[t], wi = w[t];
      const int mm = m - 1;
      float sh[kBatch], sl[kBatch];  // unnormalised partial sums of (row . u)
#pragma unroll
      for (int q = 0; q < kBatch; ++q) sh[q] = sl[q] = 0.f;
      // kBatch independent L2 loads per lane; the next batch's are issued
      // before this batch's update, so two batches are in flight
      float2 a[kBatch];
#pragma unroll
      for (int q = 0; q < kBatch; ++q) a[q] = lane + 32 * q < mm ? __ldcg(row + lane + 32 * q) : make_float2(0.f, 0.f);
      for (int j0 = lane; j0 < mm; j0 += 32 * kBatch) {
        float2 nx[kBatch];
#pragma unroll
        for (int q = 0; q < kBatch; ++q) {
          const int jj = j0 + 32 * (kBatch + q);
          nx[q] = jj < mm ? __ldcg(row + jj) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < kBatch; ++q) {
          const int jj = j0 + 32 * q;
          if (jj < mm) {
            dfl x{a[q].x, a[q].y};
            if (upd) {
              x = df_sub2(x, vi, w[1 + jj], wi, vb[1 + jj]);
              row[jj] = make_float2(x.h, x.l);
            }
            df_fma_acc(sh[q], sl[q], x, uu[1 + jj]);
          }
        }
#pragma unroll
        for (int q = 0; q < kBatch; ++q) a[q] = nx[q];
      }
      dfl acc = df_renorm(sh[0], sl[0]);
#pragma unroll
      for (int q = 1; q < kBatch; ++q) acc = df_add(acc, df_renorm(sh[q], sl[q]));
      const dfl s = df_warp_sum(acc);
      if (lane == 0 && more) Pn[it] = df_mul(tnd, s);
    }
    // the next reflector is ub + 1; the current one's buffer takes row k+2
    // (every read of vb, w and ub ends before the barrier's first sync)
    dfl* const base_v = vb == v || vb == v + 1 ? v : u;
    vb = ub + 1;
    ub = base_v;
    tk = tn;
    if (!grid_barrier(bar, nb, epoch, status)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const float2 a = __ldcg(reinterpret_cast<const float2*>(A) + int64_t(n - 1) * n + n - 1);
    dv[n - 1] = df_val(dfl{a.x, a.y}) * unscale;
  }
}

// n = 1 or 2: S is already tridiagonal (lower triangle authoritative).
__global__ void tiny_tridiag_kernel(const double* S, int64_t lds, int n, double* dv, double* ev) {
  dv[0] = S[0];
  if (n == 2) {
    dv[1] = S[lds + 1];
    ev[0] = S[lds];
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

// Number of eigenvalues of T strictly below x: sign changes of the Sturm
// sequence p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (the leading
// principal minors of T - x I; a zero takes the sign opposite to its
// predecessor's), division-free.  Double-float, on T scaled by a power of
// two c with ||c T|| about 1; p_i is rescaled by 2^-e whenever |p_i| leaves
// [2^-60, 2^60], so nothing leaves the FP32 range.  About 45 FP32 operations per step instead of six FP64
// ones, on a pipe that is two orders of magnitude wider.
__device__ __forceinline__ int sturm_count_df(const dfl* dv, const dfl* e2, int n, dfl x) {
  const dfl nx = df_neg(x);
  dfl pm{1.f, 0.f}, p = df_add(dv[0], nx);
  int sp = p.h <= 0.f;
  int cnt = sp;
  for (int i = 1; i < n; ++i) {
    dfl pn = df_mul(df_add(dv[i], nx), p);
    pn = df_fma(pn, df_neg(e2[i - 1]), pm);
    const int sn = pn.h < 0.f || (pn.h == 0.f && !sp);
    cnt += sn ^ sp;
    pm = p;
    p = pn;
    sp = sn;
    const float ap = fabsf(p.h);
    if (ap > 0x1p+60f || (ap < 0x1p-60f && ap != 0.f)) {
      const int e = ((__float_as_int(ap) >> 23) & 0xff) - 127;  // exponent of |p| (-127 when subnormal)
      const float f = __int_as_float((127 - e) << 23);          // 2^-e, exact
      p = dfl{__fmul_rn(p.h, f), __fmul_rn(p.l, f)};
      pm = dfl{__fmul_rn(pm.h, f), __fmul_rn(pm.l, f)};
    }
  }
  return cnt;
}

constexpr int kBisectLanes = 16;  // lanes per eigenvalue ((lanes + 1)-way multisection)

// Lanes in groups of kMS find the ascending eigenvalues j0 + group (or
// jlist[group]): each round evaluates kMS interior points of the current
// interval and keeps the sub-interval holding eigenvalue j (counts are
// monotone in x).
template <int kMS>
__global__ void bisect_kernel(const double* __restrict__ dv_g, const double* __restrict__ e2_g, int n, int j0,
                              const int* __restrict__ jlist, int cnt, const double* __restrict__ info,
                              double* __restrict__ lam) {
  extern __shared__ dfl bis_sm[];
  dfl* dv = bis_sm;      // c T's diagonal
  dfl* e2 = bis_sm + n;  // c^2 times the squared off-diagonal
  int ce = 0;            // c = 2^-ce
  {
    const double tn = info[3];
    if (tn > 0.0 && isfinite(tn)) frexp(tn, &ce);
  }
  const double c = ldexp(1.0, -ce), c2 = c * c;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    dv[i] = df_from(dv_g[i] * c);
    if (i + 1 < n) e2[i] = df_from(e2_g[i] * c2);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int sub = lane % kMS, gbase = lane - sub;
  const int group = (blockIdx.x * blockDim.x + threadIdx.x) / kMS;
  const bool active = group < cnt;
  const int gi = active ? group : cnt - 1;
  const int j = jlist ? jlist[gi] : j0 + gi;
  const double floor_abs = 4.0 * info[2];
  double lo = info[0], hi = info[1];
  for (int round = 0; round < 64; ++round) {
    const bool done = hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + floor_abs;
    if (!__any_sync(0xffffffffu, !done)) break;
    const double x = lo + (hi - lo) * double(sub + 1) / double(kMS + 1);
    const int cn = sturm_count_df(dv, e2, n, df_from(x * c));
    const unsigned bal = __ballot_sync(0xffffffffu, cn <= j);
    const unsigned gmask = kMS == 32 ? 0xffffffffu : ((1u << (kMS & 31)) - 1u);
    const int t = __popc((bal >> gbase) & gmask);  // points with count <= j (a prefix)
    const double xl = __shfl_sync(0xffffffffu, x, gbase + (t > 0 ? t - 1 : 0));
    const double xh = __shfl_sync(0xffffffffu, x, gbase + (t < kMS ? t : kMS - 1));
    if (!done) {
      if (t > 0) lo = xl;
      if (t < kMS) hi = xh;
    }
  }
  if (active && sub == 0) lam[group] = 0.5 * (lo + hi);
}

// Counter-based hash of (a, b) to [-1, 1], FP32 (the inverse-iteration start).
__device__ __forceinline__ float hash_unit_f(uint32_t a, uint32_t b) {
  uint32_t x = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  x ^= x >> 15;
  x *= 0x2C1B3C6Du;
  x ^= x >> 12;
  x *= 0x297A2D39u;
  x ^= x >> 15;
  return __fmaf_rn(__uint2float_rn(x), 0x1p-31f, -1.f);
}

// Inverse iteration for one eigenvalue: solves (T - lam I) z = y kInvIters
// times from a pseudo-random start, in double-float on c T (c a power of two
// with ||c T|| about 1; sd, se its diagonal and off-diagonal): each step's
// quotient and updates are a few dozen FP32 operations instead of an FP64
// division on a pipe that issues about one lane per clock.  Entry i of the
// work arrays Z, u0, u1, u2 sits at [i * st]; z ends, normalised, in
// out[i * ost] as FP64.
__device__ __forceinline__ void inverse_iter_one(const dfl* sd, const dfl* se, int n, dfl nlm, float tiny, uint32_t seed,
                                                 dfl* Z, dfl* u0, dfl* u1, dfl* u2, int64_t st, double* out,
                                                 int64_t ost) {
  for (int i = 0; i < n; ++i) Z[int64_t(i) * st] = dfl{hash_unit_f(seed, uint32_t(i)), 0.f};
  for (int iter = 0; iter < kInvIters; ++iter) {
    // factor with partial pivoting while applying L^-1 to the right-hand side
    dfl a = df_add(sd[0], nlm), b = se[0];
    dfl y = Z[0];  // current y_i (after elimination of previous rows)
    for (int i = 0; i + 1 < n; ++i) {
      const dfl c = se[i];
      const dfl na = df_add(sd[i + 1], nlm);
      const dfl nb = se[i + 1 < n ? i + 1 : i];
      const dfl nbv = i + 2 < n ? nb : df_zero();
      const dfl ynext = Z[int64_t(i + 1) * st];
      dfl yi, ynew;
      const int64_t o = int64_t(i) * st;
      if (fabsf(a.h) >= fabsf(c.h)) {
        const dfl piv = fabsf(a.h) < tiny ? dfl{a.h < 0.f ? -tiny : tiny, 0.f} : a;
        const dfl nl = df_neg(df_div(c, piv));
        u0[o] = piv;
        u1[o] = b;
        u2[o] = df_zero();
        yi = y;
        ynew = df_fma(ynext, nl, y);  // ynext - l y
        a = df_fma(na, nl, b);        // na - l b
        b = nbv;
      } else {
        const dfl nl = df_neg(df_div(a, c));
        u0[o] = c;
        u1[o] = na;
        u2[o] = nbv;
        yi = ynext;
        ynew = df_fma(y, nl, ynext);  // y - l ynext
        a = df_fma(b, nl, na);        // b - l na
        b = df_mul(nl, nbv);          // -l nb
      }
      Z[o] = yi;
      y = ynew;
    }
    const dfl last = fabsf(a.h) < tiny ? dfl{a.h < 0.f ? -tiny : tiny, 0.f} : a;
    // back substitution, tracking the largest magnitude for scaling
    dfl z2 = df_zero(), z1 = df_div(y, last);
    Z[int64_t(n - 1) * st] = z1;
    float zmax = fabsf(z1.h);
    for (int i = n - 2; i >= 0; --i) {
      const int64_t o = int64_t(i) * st;
      const dfl zi = df_div(df_sub2(Z[o], u1[o], z1, u2[o], z2), u0[o]);
      Z[o] = zi;
      z2 = z1;
      z1 = zi;
      zmax = fmaxf(zmax, fabsf(zi.h));
    }
    // scale (keeps the next solve in range); on the last pass normalise and
    // write FP64
    const dfl sc{1.f / fmaxf(zmax, FLT_MIN), 0.f};
    if (iter + 1 < kInvIters) {
      for (int i = 0; i < n; ++i) Z[int64_t(i) * st] = df_mul(Z[int64_t(i) * st], sc);
    } else {
      dfl nn = df_zero();
      for (int i = 0; i < n; ++i) {
        const dfl zi = df_mul(Z[int64_t(i) * st], sc);
        nn = df_fma(nn, zi, zi);
      }
      const dfl s2 = df_div(sc, df_sqrt(nn));
      for (int i = 0; i < n; ++i) out[int64_t(i) * ost] = df_val(df_mul(Z[int64_t(i) * st], s2));
    }
  }
}

// c T in double-float into shared memory (sd, se; se 0 past the end), and
// the power-of-two scale c.
__device__ __forceinline__ double load_scaled_tri(const double* __restrict__ dv, const double* __restrict__ ev, int n,
                                                  const double* __restrict__ info, dfl* sd, dfl* se) {
  int ce = 0;
  {
    const double tn = info[3];
    if (tn > 0.0 && isfinite(tn)) frexp(tn, &ce);
  }
  const double cs = ldexp(1.0, -ce);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sd[i] = df_from(dv[i] * cs);
    se[i] = i + 1 < n ? df_from(ev[i] * cs) : df_zero();
  }
  __syncthreads();
  return cs;
}

// Inverse iteration, one thread per eigenvalue lam[t], work arrays in global
// memory interleaved [i][t] (stride B) so that a warp's accesses coalesce;
// z ends in Zd[i*B + t] (the same 8 bytes that held the double-float
// iterate).  For tridiagonals too long for the shared-memory form below.
__global__ void inverse_iter_kernel(const double* __restrict__ dv, const double* __restrict__ ev, int n,
                                    const double* __restrict__ lam, int cnt, int B,
                                    const double* __restrict__ info, dfl* __restrict__ u0, dfl* __restrict__ u1,
                                    dfl* __restrict__ u2, double* __restrict__ Zd, int seed_base) {
  extern __shared__ dfl inv_sm[];
  dfl* sd = inv_sm;
  dfl* se = inv_sm + n;
  const double cs = load_scaled_tri(dv, ev, n, info, sd, se);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const dfl nlm = df_from(-lam[t] * cs);
  const float tiny = 0x1p-52f * float(fmax(info[3], DBL_MIN) * cs);
  inverse_iter_one(sd, se, n, nlm, tiny, uint32_t(seed_base + t), reinterpret_cast<dfl*>(Zd) + t, u0 + t, u1 + t,
                   u2 + t, B, Zd + t, B);
}

// The same solves with each thread's work arrays in shared memory (4n
// double-float per eigenvalue after the 2n of c T): every step of the two
// sequential sweeps reads and writes shared memory instead of waiting on
// an L2 round trip.  Output as inverse_iter_kernel (Zd[i*B + t], FP64).
__global__ void inverse_iter_smem_kernel(const double* __restrict__ dv, const double* __restrict__ ev, int n,
                                         const double* __restrict__ lam, int cnt, int B,
                                         const double* __restrict__ info, double* __restrict__ Zd, int seed_base) {
  extern __shared__ dfl inv_sm[];
  dfl* sd = inv_sm;
  dfl* se = inv_sm + n;
  const double cs = load_scaled_tri(dv, ev, n, info, sd, se);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  dfl* wk = inv_sm + 2 * n + int64_t(threadIdx.x) * 4 * n;  // Z, u0, u1, u2 of this thread
  const dfl nlm = df_from(-lam[t] * cs);
  const float tiny = 0x1p-52f * float(fmax(info[3], DBL_MIN) * cs);
  inverse_iter_one(sd, se, n, nlm, tiny, uint32_t(seed_base + t), wk, wk + n, wk + 2 * n, wk + 3 * n, 1, Zd + t, B);
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

// ---- blocked back-transformation (compact WY) ------------------------------
// Q = H_0 H_1 ... H_{n-3} = Q_0 Q_1 ... Q_{B-1}, Q_b = H_{32b} ... H_{32b+31}
// = I - V_b T_b V_b^T (T_b upper triangular, the forward recurrence
// T_jj = tau_j, T(0:j, j) = -tau_j T(0:j, 0:j) V_b(:, 0:j)^T v_j).  With
// U_b = V_b T_b, Z <- Q Z is Z <- Z - U_b (V_b^T Z) for b = B-1 down to 0.

constexpr int kWY = 32;    // reflectors per block
constexpr int kWYV = 64;   // eigenvectors per pass of the apply kernel

// One CTA per block: G = V_b^T V_b (rows in chunks of 64 through shared
// memory), T_b, then U_b (stored [b][j][i], rows contiguous).
__global__ void __launch_bounds__(256) wy_prep_kernel(const double* __restrict__ Vh, const double* __restrict__ tau,
                                                      int n, double* __restrict__ U) {
  __shared__ double Vs[kWY][65];
  __shared__ double G[kWY][kWY + 1];
  __shared__ double T[kWY][kWY + 1];
  const int b = blockIdx.x, k0 = b * kWY;
  const int nb = min(kWY, (n - 2) - k0);
  // the 528 pairs j <= j2, up to 3 per thread
  double acc[3] = {0.0, 0.0, 0.0};
  int pj[3], pk[3];
  for (int q = 0; q < 3; ++q) {
    int p = threadIdx.x + q * 256, j = 0;
    while (p >= kWY - j && j < kWY) p -= kWY - j, ++j;  // p-th pair of row j: (j, j + p)
    pj[q] = j < kWY ? j : -1;
    pk[q] = j < kWY ? j + p : -1;
  }
  for (int i0 = k0 + 1; i0 < n; i0 += 64) {
    for (int e = threadIdx.x; e < kWY * 64; e += blockDim.x) {
      const int j = e >> 6, r = e & 63;
      Vs[j][r] = (j < nb && i0 + r < n) ? Vh[int64_t(k0 + j) * n + i0 + r] : 0.0;
    }
    __syncthreads();
    for (int q = 0; q < 3; ++q) {
      if (pj[q] < 0) continue;
      double sacc = 0.0;
      for (int r = 0; r < 64; ++r) sacc += Vs[pj[q]][r] * Vs[pk[q]][r];
      acc[q] += sacc;
    }
    __syncthreads();
  }
  for (int q = 0; q < 3; ++q)
    if (pj[q] >= 0) G[pj[q]][pk[q]] = acc[q];
  for (int e = threadIdx.x; e < kWY * (kWY + 1); e += blockDim.x) T[e / (kWY + 1)][e % (kWY + 1)] = 0.0;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    const double tj = tau[k0 + j];
    double t = 0.0;
    const int i = threadIdx.x;
    if (i < j) {
      for (int l = i; l < j; ++l) t += T[i][l] * G[l][j];
    }
    __syncthreads();
    if (i < j) T[i][j] = -tj * t;
    if (i == j) T[j][j] = tj;
    __syncthreads();
  }
  // U_b[j][i] = sum_{l <= j} V[k0 + l][i] T[l][j], rows i > k0
  double* Ub = U + int64_t(b) * kWY * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v[kWY];
#pragma unroll
    for (int l = 0; l < kWY; ++l) v[l] = (l < nb && i > k0) ? Vh[int64_t(k0 + l) * n + i] : 0.0;
    // T is zero below its diagonal: the full sum over l is the triangular one
#pragma unroll 1
    for (int j = 0; j < kWY; ++j) {
      double u = 0.0;
#pragma unroll
      for (int l = 0; l < kWY; ++l) u += v[l] * T[l][j];
      Ub[int64_t(j) * n + i] = u;
    }
  }
}

// Z (cnt vectors, vector-major cnt x n) <- Q Z.  Cooperative: CTA p owns
// rows [r0, r1) of every vector and keeps them in shared memory across the
// blocks; per block it adds its rows' part of Y = V_b^T Z into Y_b (zeroed
// beforehand, one slot per (vector group, block)), one grid barrier, then
// updates its rows with U_b Y_b.
__global__ void __launch_bounds__(256) wy_apply_kernel(const double* __restrict__ Vh, const double* __restrict__ U,
                                                       int n, int nblk, int cnt, int chunk,
                                                       double* __restrict__ Z, double* __restrict__ Y,
                                                       unsigned* bar, int* status) {
  extern __shared__ double wsm[];
  double* Zs = wsm;                       // [kWYV][chunk]
  double* Vs = Zs + kWYV * chunk;         // [kWY][chunk]
  double* Us = Vs + kWY * chunk;          // [kWY][chunk]
  double* Ys = Us + kWY * chunk;          // [kWY][kWYV]
  const unsigned nb = gridDim.x;
  unsigned epoch = 0;  // grid barriers passed
  const int r0 = blockIdx.x * chunk, r1 = min(n, r0 + chunk);
  const int rows = max(0, r1 - r0);
  const int ngroups = (cnt + kWYV - 1) / kWYV;
  for (int g = 0; g < ngroups; ++g) {
    const int vg = g * kWYV, nv = min(kWYV, cnt - vg);
    for (int e = threadIdx.x; e < kWYV * chunk; e += blockDim.x) {
      const int c = e / chunk, ri = e - c * chunk;
      Zs[e] = (c < nv && ri < rows) ? Z[int64_t(vg + c) * n + r0 + ri] : 0.0;
    }
    for (int b = nblk - 1; b >= 0; --b) {
      const int k0 = b * kWY;
      const int nbr = min(kWY, (n - 2) - k0);  // reflectors in this block (rows k0 .. k0 + nbr - 1 of Vh)
      const int lo = max(0, k0 + 1 - r0);     // first local row with nonzero v (i > k0)
      double* Yb = Y + (int64_t(g) * nblk + b) * kWY * kWYV;
      __syncthreads();
      if (lo < rows) {
        for (int e = threadIdx.x; e < kWY * chunk; e += blockDim.x) {
          const int j = e / chunk, ri = e - j * chunk;
          const bool in = ri >= lo && ri < rows;
          Vs[e] = in && j < nbr ? __ldg(Vh + int64_t(k0 + j) * n + r0 + ri) : 0.0;
          Us[e] = in ? __ldg(U + (int64_t(b) * kWY + j) * n + r0 + ri) : 0.0;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kWY * nv; e += blockDim.x) {
          const int j = e / nv, c = e - j * nv;
          double s = 0.0;
          for (int ri = lo; ri < rows; ++ri) s += Vs[j * chunk + ri] * Zs[c * chunk + ri];
          atomicAdd(Yb + j * kWYV + c, s);
        }
      }
      if (!grid_barrier(bar, nb, epoch, status)) return;
      if (lo < rows) {
        for (int e = threadIdx.x; e < kWY * nv; e += blockDim.x) {
          const int j = e / nv, c = e - j * nv;
          Ys[j * kWYV + c] = __ldcg(Yb + j * kWYV + c);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nv * rows; e += blockDim.x) {
          const int c = e / rows, ri = e - c * rows;
          if (ri < lo) continue;
          double s = 0.0;
#pragma unroll 8
          for (int j = 0; j < kWY; ++j) s += Us[j * chunk + ri] * Ys[j * kWYV + c];
          Zs[c * chunk + ri] -= s;
        }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nv * chunk; e += blockDim.x) {
      const int c = e / chunk, ri = e - c * chunk;
      if (ri < rows) Z[int64_t(vg + c) * n + r0 + ri] = Zs[e];
    }
  }
}

// evals[c] = lam[cnt-1-c] (descending)
__global__ void values_kernel(const double* __restrict__ lam, int cnt, double* __restrict__ evals) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < cnt) evals[c] = lam[cnt - 1 - c];
}

// evecs[i*ldv + c] = Zc[(cnt-1-c)*n + i]
__global__ void output_kernel(const double* __restrict__ Zc, int n, int cnt, double* __restrict__ evecs,
                              int64_t ldv) {
  __shared__ double tile[32][33];
  const int c0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
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

constexpr int kInvBatch = 4096;

struct EigScratch {
  dfl *A, *P;  // the matrix being reduced and the mat-vec, double-float
  double *Vh, *tau, *dv, *ev, *e2, *info, *lam, *lamv, *u0, *u1, *u2, *Z, *Zc, *Uwy, *Ywy;
  unsigned long long* amax;
  size_t bytes;
};

int wy_blocks(int64_t d) { return d >= 3 ? int((d - 2 + kWY - 1) / kWY) : 0; }

EigScratch carve_eig(void* base, int64_t d, int32_t nval, int32_t nvec) {
  Carve c(base);
  EigScratch s;
  const int64_t B = std::max<int64_t>(1, std::min<int64_t>(nvec, kInvBatch));
  s.A = c.take<dfl>(d * d);
  s.Vh = c.take<double>(d * d);
  s.tau = c.take<double>(d);
  s.dv = c.take<double>(d);
  s.ev = c.take<double>(d);
  s.e2 = c.take<double>(d);
  s.P = c.take<dfl>(2 * d);
  s.amax = c.take<unsigned long long>(1);
  s.info = c.take<double>(8);
  s.lam = c.take<double>(std::max(nval, 1));
  s.lamv = c.take<double>(std::max(nvec, 1));
  s.u0 = c.take<double>(d * B);
  s.u1 = c.take<double>(d * B);
  s.u2 = c.take<double>(d * B);
  s.Z = c.take<double>(d * B);
  s.Zc = c.take<double>(d * std::max(nvec, 1));
  s.Uwy = c.take<double>(int64_t(wy_blocks(d)) * kWY * d);
  s.Ywy = c.take<double>(int64_t((std::max(nvec, 1) + kWYV - 1) / kWYV) * wy_blocks(d) * kWY * kWYV);
  s.bytes = c.off + 256;
  return s;
}

}  // namespace

size_t eig_scratch_bytes(int64_t d, int32_t nval, int32_t nvec) { return carve_eig(nullptr, d, nval, nvec).bytes; }

cudaError_t launch_eig(gmgm_handle* h, int64_t d64, const double* S, int64_t lds, int32_t nval, double* evals,
                       const int* vlist, int32_t nvec, double* evecs, int64_t ldv, void* scratch) {
  const int n = int(d64);
  cudaStream_t st = h->stream;
  EigScratch s = carve_eig(scratch, d64, nval, nvec);
  cudaError_t e;
  int launches = 0;
  if (n >= 3) {
    if ((e = cudaMemsetAsync(s.amax, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    const int64_t total = int64_t(n) * n;
    absmax_kernel<<<unsigned(std::min<int64_t>((total + 255) / 256, int64_t(h->num_sms) * 8)), 256, 0, st>>>(
        S, lds, n, s.amax);
    dim3 b(32, 8), g(unsigned((n + 31) / 32), unsigned((n + 7) / 8));
    copy_sym_kernel<<<g, b, 0, st>>>(S, lds, n, s.amax, s.A);
    launches += 2;
  }
  if ((e = cudaMemsetAsync(s.Vh, 0, size_t(n) * n * sizeof(double), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(s.tau, 0, size_t(n) * sizeof(double), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(s.ev, 0, size_t(n) * sizeof(double), st)) != cudaSuccess) return e;
  if (n >= 3) {
    const size_t smem = size_t(3) * n * sizeof(dfl);
    if ((e = cudaFuncSetAttribute(tridiag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) !=
        cudaSuccess)
      return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_kernel, kTriThreads, smem)) !=
        cudaSuccess)
      return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    unsigned blocks = unsigned(h->num_sms);
    // small problems: fewer CTAs (cheaper barriers)
    const unsigned want = unsigned((int64_t(n) * n + 16383) / 16384);
    blocks = std::min(blocks, std::max(1u, want));
    if ((e = cudaMemsetAsync(h->d_barrier, 0, 64, st)) != cudaSuccess) return e;
    dfl* A = s.A;
    dfl* P = s.P;
    const unsigned long long* amax = s.amax;
    double *dv = s.dv, *ev = s.ev, *Vh = s.Vh, *tau = s.tau;
    unsigned* bar = h->d_barrier;
    int* status = h->d_status;
    int nn = n;
    void* args[] = {&A, &nn, &amax, &dv, &ev, &Vh, &tau, &P, &bar, &status};
    if ((e = cudaLaunchCooperativeKernel((void*)tridiag_kernel, dim3(blocks), dim3(kTriThreads), args, smem,
                                         st)) != cudaSuccess)
      return e;
  } else {
    // n = 1 or 2: already tridiagonal
    tiny_tridiag_kernel<<<1, 1, 0, st>>>(S, lds, n, s.dv, s.ev);
  }
  tri_info_kernel<<<1, 256, 0, st>>>(s.dv, s.ev, n, s.e2, s.info);
  launches += 2;
  const size_t bsmem = size_t(2) * n * sizeof(dfl);
  if ((e = cudaFuncSetAttribute(bisect_kernel<kBisectLanes>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(bsmem))) != cudaSuccess)
    return e;
  const int tpb = kBisectLanes >= 8 ? 64 : 32;  // small blocks: the groups spread over every SM
  if (nval > 0) {
    // the nval largest eigenvalues, ascending in lam
    const int64_t threads = int64_t(nval) * kBisectLanes;
    bisect_kernel<kBisectLanes><<<unsigned((threads + tpb - 1) / tpb), tpb, bsmem, st>>>(s.dv, s.e2, n, n - nval, nullptr, nval,
                                                                          s.info, s.lam);
    values_kernel<<<unsigned((nval + 255) / 256), 256, 0, st>>>(s.lam, nval, evals);
    launches += 2;
  }
  if (nvec > 0) {
    // targets of the vectors: the nvec largest (reusing lam), or the listed
    // ascending indices
    const double* lamv = s.lam + (nval - nvec);
    if (vlist || nvec > nval) {
      const int64_t threads = int64_t(nvec) * kBisectLanes;
      bisect_kernel<kBisectLanes><<<unsigned((threads + tpb - 1) / tpb), tpb, bsmem, st>>>(s.dv, s.e2, n, n - nvec, vlist, nvec,
                                                                            s.info, s.lamv);
      lamv = s.lamv;
      ++launches;
    }
    const int B = std::min(nvec, kInvBatch);
    const size_t ismem = size_t(2) * n * sizeof(dfl);
    // eigenvalues per block with the work arrays in shared memory (0: too long)
    int smem_optin = 0;
    if ((e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device)) != cudaSuccess)
      return e;
    const size_t per_vec = size_t(4) * n * sizeof(dfl);
    const int vpb = size_t(smem_optin) > ismem ? int(std::min<size_t>(32, (size_t(smem_optin) - ismem) / per_vec)) : 0;
    if (vpb > 0) {
      if ((e = cudaFuncSetAttribute(inverse_iter_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    int(ismem + vpb * per_vec))) != cudaSuccess)
        return e;
    } else if ((e = cudaFuncSetAttribute(inverse_iter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(ismem))) != cudaSuccess) {
      return e;
    }
    for (int t0 = 0; t0 < nvec; t0 += B) {
      const int cnt = std::min(B, nvec - t0);
      if (vpb > 0)
        inverse_iter_smem_kernel<<<unsigned((cnt + vpb - 1) / vpb), unsigned(vpb), ismem + vpb * per_vec, st>>>(
            s.dv, s.ev, n, lamv + t0, cnt, B, s.info, s.Z, t0);
      else
        inverse_iter_kernel<<<unsigned((cnt + 31) / 32), 32, ismem, st>>>(
            s.dv, s.ev, n, lamv + t0, cnt, B, s.info, reinterpret_cast<dfl*>(s.u0), reinterpret_cast<dfl*>(s.u1),
            reinterpret_cast<dfl*>(s.u2), s.Z, t0);
      dim3 tb(32, 8), tg(unsigned((cnt + 31) / 32), unsigned((n + 31) / 32));
      transpose_kernel<<<tg, tb, 0, st>>>(s.Z, n, cnt, B, s.Zc, t0);
      launches += 2;
    }
    cluster_mgs_kernel<<<unsigned(nvec), 256, 0, st>>>(lamv, nvec, s.info, 1e-7, n, s.Zc);
    ++launches;
    const int nblk = wy_blocks(n);
    if (nblk > 0) {
      // back-transformation Z <- Q Z in compact WY blocks
      wy_prep_kernel<<<unsigned(nblk), 256, 0, st>>>(s.Vh, s.tau, n, s.Uwy);
      const int ngroups = (nvec + kWYV - 1) / kWYV;
      if ((e = cudaMemsetAsync(s.Ywy, 0, size_t(ngroups) * nblk * kWY * kWYV * sizeof(double), st)) != cudaSuccess)
        return e;
      if ((e = cudaMemsetAsync(h->d_barrier, 0, 64, st)) != cudaSuccess) return e;
      int chunk = (n + h->num_sms - 1) / h->num_sms;
      const int grid = (n + chunk - 1) / chunk;
      const size_t smem = (size_t(kWYV + 2 * kWY) * chunk + size_t(kWY) * kWYV) * sizeof(double);
      if ((e = cudaFuncSetAttribute(wy_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) !=
          cudaSuccess)
        return e;
      int per_sm = 0;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wy_apply_kernel, 256, smem)) != cudaSuccess)
        return e;
      if (per_sm < 1 || grid > per_sm * h->num_sms) return cudaErrorInvalidConfiguration;
      const double* Vh = s.Vh;
      const double* Uw = s.Uwy;
      double* Z = s.Zc;
      double* Y = s.Ywy;
      unsigned* bar = h->d_barrier;
      int* status = h->d_status;
      int nn = n, nbk = nblk, nc = nvec, ch = chunk;
      void* args[] = {&Vh, &Uw, &nn, &nbk, &nc, &ch, &Z, &Y, &bar, &status};
      if ((e = cudaLaunchCooperativeKernel((void*)wy_apply_kernel, dim3(grid), dim3(256), args, smem, st)) !=
          cudaSuccess)
        return e;
      launches += 2;
    }
    dim3 b(32, 8), g(unsigned((nvec + 31) / 32), unsigned((n + 31) / 32));
    output_kernel<<<g, b, 0, st>>>(s.Zc, n, nvec, evecs, ldv);
    ++launches;
  }
  note_launch(launches);
  return cudaGetLastError();
}

}  // namespace gmgm
