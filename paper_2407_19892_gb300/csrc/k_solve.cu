// Eigenvalue solve of the improved GmGM (Proposition on the eigenvalue
// gradient; existence lemma's box Lam_l >= eps_l; Algorithm 1's loop).
//
//   f(Lam) = sum_l E_l . Lam_l - sum_gamma sum_{grid of gamma} log s,
//   s = sum_{l in gamma} lam_{l, i_l},
//   g_l,i = E_l,i - sum_{gamma containing l} sum_{grid, i_l = i} 1/s.
//
// One persistent CTA (1024 threads) runs a projected Newton method
// (Bertsekas' nearly-active set: coordinates at/near their bound with a
// positive gradient take a diagonally scaled step; the free ones a Newton
// step from Jacobi-preconditioned conjugate gradients, whose Hessian-vector
// products are reductions over the grids) with an Armijo search along the
// projection arc.  Every pass over a grid is a reduction: per point one
// reciprocal (and its square), row sums by warp shuffles + shared-memory FP64
// atomics, column sums in registers with Kahan compensation.
//
// Precision: the passes run in FP32 (Kahan / FP64 partials) until the
// relative KKT residual reaches 1e-5; from then on the gradient is formed in
// FP64 (FP32 reciprocal refined by one Newton step in FP64) while the CG
// Hessian products stay FP32 (inexact Newton).  The line search evaluates
// f(x_new) - f(x) = g.dx + sum (u - log1p(u)), u = ds/s, which is accurate
// where the two objective values would cancel.  The final KKT check is FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>

#include "device.cuh"
#include "internal.cuh"

namespace gmgm {

namespace {

constexpr int kThreads = 1024;
constexpr int kQ = 4;                    // columns per thread per chunk (path A)
constexpr int kChunkCols = kThreads * kQ;
constexpr int kMaxLoop = 8192;           // largest loop-axis rank (smem accumulators)

struct Params {
  int L;
  int r[GMGM_MAX_AXES];
  int off[GMGM_MAX_AXES + 1];
  int N;
  int nmod;
  int mk[GMGM_MAX_MODALITIES];
  int ma[GMGM_MAX_MODALITIES][GMGM_MAX_AXES];
  double eps[GMGM_MAX_AXES];
  const double* E[GMGM_MAX_AXES];
  const double* init[GMGM_MAX_AXES];
  double* out[GMGM_MAX_AXES];
  double tol;
  int max_newton, max_cg, fp32_phase, gauge, has_init;
  double trace_rtol;
  // several CTAs (cooperative launch): CTA 0 runs the method and hands each
  // grid pass to every CTA through these words (null with one CTA)
  unsigned* co_bar;   // grid barrier words
  int* co_cmd;        // the pass kind, -1: finished
  double* co_ls;      // line-search sum of the pass
  int* co_bad;        // a point of the pass was infeasible / non-finite
};

struct Vecs {
  double *E, *x, *g, *lo, *hd, *d, *rr, *z, *p, *hp, *dx, *s1, *s2;
  float *x32, *v32;
  int* act;
};

enum Kind { K_GRAD32 = 0, K_GRAD64 = 1, K_HVP = 2, K_LS = 3 };

struct PassOut {
  double ls;   // line-search remainder sum (K_LS)
  int bad;     // infeasible / non-finite seen
};

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// u - log1p(u), accurate for small u (series) and exact elsewhere.
__device__ __forceinline__ float u_minus_log1p(float u) {
  if (fabsf(u) < 1e-2f) {
    const float u2 = u * u;
    return u2 * (0.5f - u * (1.f / 3.f - u * (0.25f - u * 0.2f)));
  }
  return u - log1pf(u);
}

// ---- one pass over one modality's grid ------------------------------------
// Accumulates into s1/s2 (global FP64, indexed by concatenated coordinate)
// and returns the scalar line-search sum.  sm1/sm2: shared accumulators of
// the loop axis.
template <int KIND>
__device__ double modality_pass(const Params& P, const Vecs& V, int gm, double* sm1, double* sm2, int* bad) {
  const int k = P.mk[gm];
  double ls = 0.0;
  if (k == 1) {
    const int a = P.ma[gm][0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.r[a]; i += gridDim.x * blockDim.x) {
      const int ia = P.off[a] + i;
      if (KIND == K_GRAD64) {
        const double s = V.x[ia];
        if (!(s > 0.0)) *bad = 1;
        V.s1[ia] += 1.0 / s;
      } else {
        const float s = V.x32[ia];
        if (KIND == K_GRAD32) {
          if (!(s > 0.f)) *bad = 1;
          const float inv = 1.f / s;
          V.s1[ia] += inv;
          V.s2[ia] += double(inv) * inv;
        } else if (KIND == K_HVP) {
          const float inv = 1.f / s;
          V.s1[ia] += double(V.v32[ia] * inv * inv);
        } else {
          const float ds = V.v32[ia];
          if (!(s + ds > 0.f)) *bad = 1;
          ls += u_minus_log1p(ds / s);
        }
      }
    }
    return ls;
  }
  // choose the loop axis: the smallest rank
  int lp = 0;
  for (int q = 1; q < k; ++q)
    if (P.r[P.ma[gm][q]] < P.r[P.ma[gm][lp]]) lp = q;
  const int a = P.ma[gm][lp];
  const int ra = P.r[a];
  for (int i = threadIdx.x; i < ra; i += blockDim.x) sm1[i] = 0.0, sm2[i] = 0.0;
  __syncthreads();
  // rest = all other axes, flattened (last axis fastest)
  int rest_ax[GMGM_MAX_AXES - 1];
  int nrest = 0;
  int64_t R = 1;
  for (int q = 0; q < k; ++q)
    if (q != lp) rest_ax[nrest++] = P.ma[gm][q], R *= P.r[P.ma[gm][q]];
  const int lane = threadIdx.x & 31;
  const float* xa32 = V.x32 + P.off[a];
  const float* va32 = V.v32 + P.off[a];
  const double* xa64 = V.x + P.off[a];
  // the chunks of rest points are split over the CTAs
  for (int64_t c0 = int64_t(blockIdx.x) * kChunkCols; c0 < R; c0 += int64_t(gridDim.x) * kChunkCols) {
    // this thread's rest points in the chunk
    int64_t qi[kQ];
    float xb[kQ], vb[kQ];
    double xb64[kQ];
    float acc1[kQ], cmp1[kQ], acc2[kQ];
    double acc64[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      qi[q] = c0 + threadIdx.x + int64_t(q) * kThreads;
      xb[q] = 0.f, vb[q] = 0.f, xb64[q] = 0.0;
      acc1[q] = 0.f, cmp1[q] = 0.f, acc2[q] = 0.f, acc64[q] = 0.0;
      if (qi[q] < R) {
        int64_t rem = qi[q];
        for (int t = nrest - 1; t >= 0; --t) {
          const int ax = rest_ax[t];
          const int idx = int(rem % P.r[ax]);
          rem /= P.r[ax];
          const int ci = P.off[ax] + idx;
          if (KIND == K_GRAD64) {
            xb64[q] += V.x[ci];
          } else {
            xb[q] += V.x32[ci];
            if (KIND == K_HVP || KIND == K_LS) vb[q] += V.v32[ci];
          }
        }
      }
    }
    for (int i = 0; i < ra; ++i) {
      float row1 = 0.f, row2 = 0.f;
      double row64 = 0.0;
      if (KIND == K_GRAD64) {
        const double xa = xa64[i];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          if (qi[q] < R) {
            const double s = xa + xb64[q];
            if (!(s > 0.0)) *bad = 1;
            const double r0 = double(1.f / float(s));
            const double inv = r0 * (2.0 - s * r0);  // one Newton step: ~46 bits
            acc64[q] += inv;
            row64 += inv;
          }
        }
        row64 = warp_sum(row64);
        if (lane == 0 && row64 != 0.0) atomicAdd(&sm1[i], row64);
      } else {
        const float xa = xa32[i];
        const float va = (KIND == K_HVP || KIND == K_LS) ? va32[i] : 0.f;
        float rc1 = 0.f;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          if (qi[q] < R) {
            const float s = xa + xb[q];
            if (KIND == K_GRAD32) {
              if (!(s > 0.f)) *bad = 1;
              const float inv = 1.f / s;
              kahan_add(acc1[q], cmp1[q], inv);
              acc2[q] = fmaf(inv, inv, acc2[q]);
              kahan_add(row1, rc1, inv);
              row2 = fmaf(inv, inv, row2);
            } else if (KIND == K_HVP) {
              const float inv = 1.f / s;
              const float t = (va + vb[q]) * inv * inv;
              kahan_add(acc1[q], cmp1[q], t);
              kahan_add(row1, rc1, t);
            } else {
              const float ds = va + vb[q];
              if (!(s + ds > 0.f)) *bad = 1;
              ls += u_minus_log1p(ds / s);
            }
          }
        }
        if (KIND != K_LS) {
          row1 = warp_sum(row1);
          if (KIND == K_GRAD32) row2 = warp_sum(row2);
          if (lane == 0) {
            atomicAdd(&sm1[i], double(row1));
            if (KIND == K_GRAD32) atomicAdd(&sm2[i], double(row2));
          }
        }
      }
    }
    // scatter the rest-point sums to their axes
    if (KIND != K_LS) {
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        if (qi[q] >= R) continue;
        int64_t rem = qi[q];
        for (int t = nrest - 1; t >= 0; --t) {
          const int ax = rest_ax[t];
          const int idx = int(rem % P.r[ax]);
          rem /= P.r[ax];
          const int ci = P.off[ax] + idx;
          const double v1 = KIND == K_GRAD64 ? acc64[q] : double(acc1[q]);
          if (nrest == 1 && gridDim.x == 1) {
            V.s1[ci] += v1;  // owned by this thread
            if (KIND == K_GRAD32) V.s2[ci] += double(acc2[q]);
          } else {
            atomicAdd(&V.s1[ci], v1);
            if (KIND == K_GRAD32) atomicAdd(&V.s2[ci], double(acc2[q]));
          }
        }
      }
    }
  }
  __syncthreads();
  if (KIND != K_LS) {
    for (int i = threadIdx.x; i < ra; i += blockDim.x) {
      if (gridDim.x == 1) {
        V.s1[P.off[a] + i] += sm1[i];
        if (KIND == K_GRAD32) V.s2[P.off[a] + i] += sm2[i];
      } else {
        atomicAdd(&V.s1[P.off[a] + i], sm1[i]);
        if (KIND == K_GRAD32) atomicAdd(&V.s2[P.off[a] + i], sm2[i]);
      }
    }
  }
  __syncthreads();
  return ls;
}

// This CTA's share of one pass over every modality's grid.
template <int KIND>
__device__ double pass_share(const Params& P, const Vecs& V, double* sm1, double* sm2, int* bad) {
  double ls = 0.0;
  for (int gm = 0; gm < P.nmod; ++gm) ls += modality_pass<KIND>(P, V, gm, sm1, sm2, bad);
  __syncthreads();
  return ls;
}

// A pass over the grids, by CTA 0.  With several CTAs it zeroes the sums,
// publishes the pass kind, meets the others at a grid barrier, does its
// share, and collects the line-search sum and the infeasible flag after a
// second barrier (a barrier that gives up marks the pass infeasible).
template <int KIND>
__device__ double grid_pass(const Params& P, const Vecs& V, double* sm1, double* sm2, double* red, int* bad,
                            unsigned& epoch, int* status) {
  if (KIND != K_LS) {
    for (int i = threadIdx.x; i < P.N; i += blockDim.x) {
      V.s1[i] = 0.0;
      if (KIND == K_GRAD32) V.s2[i] = 0.0;
    }
  }
  if (gridDim.x == 1) {
    __syncthreads();
    const double ls = pass_share<KIND>(P, V, sm1, sm2, bad);
    return KIND == K_LS ? block_sum(ls, red) : 0.0;
  }
  if (threadIdx.x == 0) {
    *reinterpret_cast<volatile int*>(P.co_cmd) = KIND;
    *reinterpret_cast<volatile double*>(P.co_ls) = 0.0;
    *reinterpret_cast<volatile int*>(P.co_bad) = 0;
  }
  if (!grid_barrier(P.co_bar, gridDim.x, epoch, status)) {
    if (threadIdx.x == 0) *bad = 1;
    __syncthreads();
    return 0.0;
  }
  double ls = pass_share<KIND>(P, V, sm1, sm2, bad);
  if (KIND == K_LS) {
    ls = block_sum(ls, red);
    if (threadIdx.x == 0) atomicAdd(P.co_ls, ls);
  }
  if (!grid_barrier(P.co_bar, gridDim.x, epoch, status)) {
    if (threadIdx.x == 0) *bad = 1;
    __syncthreads();
    return 0.0;
  }
  if (threadIdx.x == 0 && *reinterpret_cast<volatile int*>(P.co_bad)) *bad = 1;
  __syncthreads();
  return KIND == K_LS ? *reinterpret_cast<volatile double*>(P.co_ls) : 0.0;
}

// CTAs 1.. of a cooperative solve: take every pass CTA 0 publishes, do their
// share, until CTA 0 publishes the end (or a grid barrier gives up).
__device__ void pass_worker(const Params& P, const Vecs& V, double* sm1, double* sm2, int* status) {
  __shared__ double wred[33];
  __shared__ int wbad;
  unsigned epoch = 0;
  for (;;) {
    if (!grid_barrier(P.co_bar, gridDim.x, epoch, status)) return;
    const int k = *reinterpret_cast<volatile int*>(P.co_cmd);
    if (k < 0) return;
    if (threadIdx.x == 0) wbad = 0;
    __syncthreads();
    if (k == K_GRAD32) pass_share<K_GRAD32>(P, V, sm1, sm2, &wbad);
    else if (k == K_GRAD64) pass_share<K_GRAD64>(P, V, sm1, sm2, &wbad);
    else if (k == K_HVP) pass_share<K_HVP>(P, V, sm1, sm2, &wbad);
    else {
      const double ls = block_sum(pass_share<K_LS>(P, V, sm1, sm2, &wbad), wred);
      if (threadIdx.x == 0) atomicAdd(P.co_ls, ls);
    }
    __syncthreads();
    if (threadIdx.x == 0 && wbad) atomicOr(P.co_bad, 1);
    if (!grid_barrier(P.co_bar, gridDim.x, epoch, status)) return;
  }
}

__device__ double dotv(const double* a, const double* b, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[i] * b[i];
  return block_sum(s, red);
}

__device__ double rel_kkt(const Params& P, const Vecs& V, double* red) {
  double m = 0.0;
  for (int i = threadIdx.x; i < P.N; i += blockDim.x) {
    const double g = V.g[i];
    const double pg = V.x[i] > V.lo[i] ? g : fmin(g, 0.0);
    m = fmax(m, fabs(pg) / V.E[i]);
  }
  return block_max(m, red);
}

__device__ void solve_master(const Params& P, const Vecs& V, int* status, gmgm_solve_stats* st, double* sm1,
                             double* sm2, unsigned& epoch) {
  __shared__ double red[33];
  __shared__ int bad_s;
  if (threadIdx.x == 0) bad_s = 0;
  const int N = P.N;
  // ---- setup: E, box, start ----
  int bad_e = 0, nonfinite_e = 0;
  for (int a = 0; a < P.L; ++a)
    for (int i = threadIdx.x; i < P.r[a]; i += blockDim.x) {
      const double e = P.E[a][i];
      V.E[P.off[a] + i] = e;
      nonfinite_e |= !isfinite(e);
      bad_e |= !(e > 0.0) || !isfinite(e);
    }
  // every E must be positive and finite: with E_i <= 0 (an axis on which X
  // lacks full rank) f falls without bound along that coordinate, so there
  // is no minimiser; outputs become NaN and the solve stops here
  {
    const int any_nonfinite = __syncthreads_or(nonfinite_e);
    if (__syncthreads_or(bad_e)) {
      const double qnan = __longlong_as_double(0x7ff8000000000000ll);
      for (int a = 0; a < P.L; ++a)
        for (int i = threadIdx.x; i < P.r[a]; i += blockDim.x) P.out[a][i] = qnan;
      if (threadIdx.x == 0) {
        set_status(status, any_nonfinite ? GMGM_DEV_NONFINITE : GMGM_DEV_INFEASIBLE);
        st->status = any_nonfinite ? GMGM_E_NONFINITE : GMGM_E_INFEASIBLE;
        st->newton_iters = 0;
        st->cg_iters = 0;
        st->grid_passes = 0;
        st->n_active = 0;
        st->fp64_iters = 0;
        st->rel_kkt = qnan;
        st->objective = qnan;
      }
      return;
    }
  }
  // one modality whose traces agree within trace_rtol: scale every axis'
  // spectrum to the mean trace, so the flat shift of the gauge is exact
  if (P.gauge && P.nmod == 1 && P.mk[0] > 1 && P.trace_rtol > 0.0) {
    double tr[GMGM_MAX_AXES], mean = 0.0;
    for (int q = 0; q < P.mk[0]; ++q) {
      const int a = P.ma[0][q];
      double s = 0.0;
      for (int i = threadIdx.x; i < P.r[a]; i += blockDim.x) s += V.E[P.off[a] + i];
      tr[q] = block_sum(s, red);
      mean += tr[q] / P.mk[0];
    }
    bool close = mean > 0.0;
    for (int q = 0; q < P.mk[0]; ++q) close = close && fabs(tr[q] - mean) <= P.trace_rtol * mean;
    if (close) {
      for (int q = 0; q < P.mk[0]; ++q) {
        const int a = P.ma[0][q];
        const double sc = mean / tr[q];
        for (int i = threadIdx.x; i < P.r[a]; i += blockDim.x) V.E[P.off[a] + i] *= sc;
      }
      __syncthreads();
    }
  }
  // default eps: 1e-10 * max over modalities of sum_l max_i 1/E_l,i
  double epsdef = 0.0;
  {
    double big = 0.0;
    for (int gm = 0; gm < P.nmod; ++gm) {
      double s = 0.0;
      for (int q = 0; q < P.mk[gm]; ++q) {
        const int a = P.ma[gm][q];
        double mn = 1e308;
        for (int i = threadIdx.x; i < P.r[a]; i += blockDim.x) mn = fmin(mn, V.E[P.off[a] + i]);
        mn = -block_max(-mn, red);
        s += 1.0 / mn;
      }
      big = fmax(big, s);
    }
    epsdef = 1e-10 * big;
  }
  double epsv[GMGM_MAX_AXES];
  for (int a = 0; a < P.L; ++a) epsv[a] = P.eps[a] > 0.0 ? P.eps[a] : epsdef;
  for (int a = 0; a < P.L; ++a)
    for (int i = threadIdx.x; i < P.r[a]; i += blockDim.x) {
      const int c = P.off[a] + i;
      V.lo[c] = epsv[a];
      const double x0 = P.has_init ? P.init[a][i] : 1.0 / V.E[c];
      V.x[c] = fmax(x0, epsv[a]);
    }
  __syncthreads();
  int newton = 0, cg_total = 0, passes = 0, fp64_iters = 0, status_code = GMGM_OK;
  bool fp64 = P.fp32_phase == 0;
  double kkt = 1e300;
  const double sigma = 1e-4;
  for (;;) {
    // ---- gradient (and Hessian diagonal) ----
    for (int i = threadIdx.x; i < N; i += blockDim.x) V.x32[i] = float(V.x[i]);
    __syncthreads();
    grid_pass<K_GRAD32>(P, V, sm1, sm2, red, &bad_s, epoch, status);
    ++passes;
    if (fp64) {
      // FP64 gradient; s2 (Hessian diagonal) kept from the FP32 pass
      for (int i = threadIdx.x; i < N; i += blockDim.x) V.hd[i] = V.s2[i];
      __syncthreads();
      grid_pass<K_GRAD64>(P, V, sm1, sm2, red, &bad_s, epoch, status);
      ++passes;
      for (int i = threadIdx.x; i < N; i += blockDim.x) V.g[i] = V.E[i] - V.s1[i];
    } else {
      for (int i = threadIdx.x; i < N; i += blockDim.x) V.g[i] = V.E[i] - V.s1[i], V.hd[i] = V.s2[i];
    }
    __syncthreads();
    if (bad_s) {
      status_code = GMGM_E_NONFINITE;
      break;
    }
    kkt = rel_kkt(P, V, red);
    if (!fp64 && kkt <= fmax(P.tol, 1e-5)) {
      fp64 = true;
      continue;
    }
    if (fp64 && kkt <= P.tol) break;
    if (newton >= P.max_newton) {
      status_code = GMGM_E_NOT_CONVERGED;
      break;
    }
    ++newton;
    if (fp64) ++fp64_iters;
    // ---- nearly-active set, diagonal step there; CG on the free set ----
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const double g = V.g[i], h = V.hd[i];
      const int act = g > 0.0 && (V.x[i] - V.lo[i]) <= g / h;
      V.act[i] = act;
      V.d[i] = act ? g / h : 0.0;
      V.rr[i] = act ? 0.0 : g;
      V.z[i] = act ? 0.0 : g / h;
      V.p[i] = V.z[i];
    }
    __syncthreads();
    double rz = dotv(V.rr, V.z, N, red);
    const double gnorm = sqrt(dotv(V.rr, V.rr, N, red));
    const double eta = fmin(0.1, fmax(1e-12, sqrt(kkt)));
    for (int it = 0; it < P.max_cg && gnorm > 0.0; ++it) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) V.v32[i] = float(V.p[i]);
      __syncthreads();
      grid_pass<K_HVP>(P, V, sm1, sm2, red, &bad_s, epoch, status);
      ++passes;
      ++cg_total;
      for (int i = threadIdx.x; i < N; i += blockDim.x) V.hp[i] = V.act[i] ? 0.0 : V.s1[i];
      __syncthreads();
      const double pHp = dotv(V.p, V.hp, N, red);
      if (!(pHp > 0.0)) break;
      const double alpha = rz / pHp;
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        if (V.act[i]) continue;
        V.d[i] += alpha * V.p[i];
        V.rr[i] -= alpha * V.hp[i];
      }
      __syncthreads();
      const double rn = sqrt(dotv(V.rr, V.rr, N, red));
      if (rn <= eta * gnorm) break;
      for (int i = threadIdx.x; i < N; i += blockDim.x) V.z[i] = V.act[i] ? 0.0 : V.rr[i] / V.hd[i];
      __syncthreads();
      const double rz2 = dotv(V.rr, V.z, N, red);
      const double beta = rz2 / rz;
      rz = rz2;
      for (int i = threadIdx.x; i < N; i += blockDim.x) V.p[i] = V.z[i] + beta * V.p[i];
      __syncthreads();
    }
    // ---- Armijo search on the projection arc ----
    double alpha = 1.0;
    bool accepted = false;
    for (int ls = 0; ls < 60; ++ls) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double xn = fmax(V.lo[i], V.x[i] - alpha * V.d[i]);
        V.dx[i] = xn - V.x[i];
        V.v32[i] = float(V.dx[i]);
      }
      if (threadIdx.x == 0) bad_s = 0;
      __syncthreads();
      const double gdx = dotv(V.g, V.dx, N, red);
      const double rem = grid_pass<K_LS>(P, V, sm1, sm2, red, &bad_s, epoch, status);
      ++passes;
      const int infeasible = bad_s;
      __syncthreads();
      if (threadIdx.x == 0) bad_s = 0;
      const double df = gdx + rem;
      if (!infeasible && gdx < 0.0 && df <= sigma * gdx) {
        accepted = true;
        break;
      }
      if (!infeasible && gdx >= 0.0) break;  // not a descent direction
      alpha *= 0.5;
    }
    __syncthreads();
    if (!accepted) {
      status_code = GMGM_E_NOT_CONVERGED;
      break;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) V.x[i] += V.dx[i];
    __syncthreads();
  }
  __syncthreads();
  // ---- gauge: one modality with equal traces -> every axis but the first
  // gets its minimum at eps (the flat shift moves to the first axis) ----
  if (P.gauge && P.nmod == 1 && status_code == GMGM_OK) {
    double tr[GMGM_MAX_AXES];
    double tmax = 0.0;
    for (int a = 0; a < P.L; ++a) {
      double s = 0.0;
      for (int i = threadIdx.x; i < P.r[a]; i += blockDim.x) s += V.E[P.off[a] + i];
      tr[a] = block_sum(s, red);
      tmax = fmax(tmax, fabs(tr[a]));
    }
    bool equal = true;
    const int a0 = P.ma[0][0];
    for (int q = 0; q < P.mk[0]; ++q) equal = equal && fabs(tr[P.ma[0][q]] - tr[a0]) <= 1e-9 * tmax;
    if (equal && P.mk[0] > 1) {
      for (int q = 1; q < P.mk[0]; ++q) {
        const int a = P.ma[0][q];
        double mn = 1e308;
        for (int i = threadIdx.x; i < P.r[a]; i += blockDim.x) mn = fmin(mn, V.x[P.off[a] + i]);
        mn = -block_max(-mn, red);
        const double c = epsv[a] - mn;
        for (int i = threadIdx.x; i < P.r[a]; i += blockDim.x) V.x[P.off[a] + i] += c;
        for (int i = threadIdx.x; i < P.r[a0]; i += blockDim.x) V.x[P.off[a0] + i] -= c;
        __syncthreads();
      }
    }
  }
  // ---- outputs, final FP64 KKT check, objective ----
  for (int a = 0; a < P.L; ++a)
    for (int i = threadIdx.x; i < P.r[a]; i += blockDim.x) P.out[a][i] = V.x[P.off[a] + i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) V.x32[i] = float(V.x[i]);
  __syncthreads();
  grid_pass<K_GRAD64>(P, V, sm1, sm2, red, &bad_s, epoch, status);
  for (int i = threadIdx.x; i < N; i += blockDim.x) V.g[i] = V.E[i] - V.s1[i];
  __syncthreads();
  const double kkt64 = rel_kkt(P, V, red);
  // objective: E.x - sum log s (FP32 logs, FP64 accumulation): u - log1p(u)
  // with ds = 0 is not usable, so evaluate log s directly per grid point
  double lsum = 0.0;
  for (int gm = 0; gm < P.nmod; ++gm) {
    int64_t G = 1;
    for (int q = 0; q < P.mk[gm]; ++q) G *= P.r[P.ma[gm][q]];
    for (int64_t t = threadIdx.x; t < G; t += blockDim.x) {
      int64_t rem = t;
      float s = 0.f;
      for (int q = P.mk[gm] - 1; q >= 0; --q) {
        const int ax = P.ma[gm][q];
        s += V.x32[P.off[ax] + int(rem % P.r[ax])];
        rem /= P.r[ax];
      }
      lsum += double(logf(s));
    }
  }
  lsum = block_sum(lsum, red);
  const double ex = dotv(V.E, V.x, N, red);
  int nact = 0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) nact += V.x[i] <= V.lo[i];
  const double nact_d = block_sum(double(nact), red);
  if (status_code == GMGM_OK && !(kkt64 <= fmax(P.tol, 1e-12) * 10.0)) status_code = GMGM_E_NOT_CONVERGED;
  if (threadIdx.x == 0) {
    if (status_code == GMGM_E_NOT_CONVERGED) set_status(status, GMGM_DEV_NOT_CONVERGED);
    if (status_code == GMGM_E_NONFINITE) set_status(status, GMGM_DEV_NONFINITE);
    st->status = status_code;
    st->newton_iters = newton;
    st->cg_iters = cg_total;
    st->grid_passes = passes;
    st->n_active = int(nact_d);
    st->fp64_iters = fp64_iters;
    st->rel_kkt = kkt64;
    st->objective = ex - lsum;
  }
}


// One CTA runs the method; with a cooperative launch (large grids) CTAs
// 1.. take a share of every grid pass.
__global__ void __launch_bounds__(kThreads, 1) solve_kernel(Params P, Vecs V, int* status, gmgm_solve_stats* st) {
  extern __shared__ double smem[];
  double* sm1 = smem;
  double* sm2 = smem + kMaxLoop;
  if (blockIdx.x > 0) {
    pass_worker(P, V, sm1, sm2, status);
    return;
  }
  unsigned epoch = 0;
  solve_master(P, V, status, st, sm1, sm2, epoch);
  if (gridDim.x > 1) {
    if (threadIdx.x == 0) *reinterpret_cast<volatile int*>(P.co_cmd) = -1;
    grid_barrier(P.co_bar, gridDim.x, epoch, status);
  }
}

}  // namespace

size_t solve_scratch_bytes(const gmgm_problem* p) {
  int64_t N = 0;
  for (int a = 0; a < p->n_axes; ++a) N += p->r[a];
  return size_t(N) * (13 * sizeof(double) + 2 * sizeof(float) + sizeof(int)) + 22 * 256;
}

cudaError_t launch_solve(gmgm_handle* h, const gmgm_problem* p, const double* const* init,
                         const gmgm_solve_opts* o, double* const* out, void* scratch, gmgm_solve_stats* d_stats) {
  Params P{};
  P.L = p->n_axes;
  P.off[0] = 0;
  for (int a = 0; a < P.L; ++a) {
    P.r[a] = p->r[a];
    P.off[a + 1] = P.off[a] + p->r[a];
    P.eps[a] = p->eps[a];
    P.E[a] = p->E[a];
    P.init[a] = init ? init[a] : nullptr;
    P.out[a] = out[a];
  }
  P.N = P.off[P.L];
  P.nmod = p->n_modalities;
  for (int g = 0; g < P.nmod; ++g) {
    P.mk[g] = p->mod_n_axes[g];
    for (int q = 0; q < P.mk[g]; ++q) P.ma[g][q] = p->mod_axes[g][q];
  }
  // the loop axis of every modality must fit the shared accumulators
  for (int g = 0; g < P.nmod; ++g) {
    int mn = 1 << 30;
    for (int q = 0; q < P.mk[g]; ++q) mn = std::min(mn, P.r[P.ma[g][q]]);
    if (P.mk[g] > 1 && mn > kMaxLoop) return cudaErrorInvalidValue;
  }
  P.tol = o->tol;
  P.max_newton = o->max_newton;
  P.max_cg = o->max_cg;
  P.fp32_phase = o->fp32_phase;
  P.gauge = o->gauge;
  P.trace_rtol = o->trace_rtol == 0.0 ? 1e-6 : o->trace_rtol;
  P.has_init = init != nullptr;
  Carve c(scratch);
  const int N = P.N;
  Vecs V;
  V.E = c.take<double>(N);
  V.x = c.take<double>(N);
  V.g = c.take<double>(N);
  V.lo = c.take<double>(N);
  V.hd = c.take<double>(N);
  V.d = c.take<double>(N);
  V.rr = c.take<double>(N);
  V.z = c.take<double>(N);
  V.p = c.take<double>(N);
  V.hp = c.take<double>(N);
  V.dx = c.take<double>(N);
  V.s1 = c.take<double>(N);
  V.s2 = c.take<double>(N);
  V.x32 = c.take<float>(N);
  V.v32 = c.take<float>(N);
  V.act = c.take<int>(N);
  const size_t smem = size_t(2) * kMaxLoop * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  // grids of 2^20 points or more: every SM takes a share of each pass
  int64_t pts = 0;
  for (int g = 0; g < P.nmod; ++g) {
    int64_t q = 1;
    for (int k = 0; k < P.mk[g]; ++k) q *= P.r[P.ma[g][k]];
    pts = std::max(pts, q);
  }
  int per_sm = 0;
  if (pts >= (int64_t(1) << 20) &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel, kThreads, smem) == cudaSuccess &&
      per_sm >= 1) {
    P.co_bar = h->d_barrier;
    P.co_cmd = c.take<int>(4);
    P.co_ls = c.take<double>(2);
    P.co_bad = P.co_cmd + 1;
    if ((e = cudaMemsetAsync(h->d_barrier, 0, 16, h->stream)) != cudaSuccess) return e;
    gmgm_solve_stats* stp = d_stats;
    int* status = h->d_status;
    void* args[] = {&P, &V, &status, &stp};
    e = cudaLaunchCooperativeKernel((void*)solve_kernel, dim3(h->num_sms), dim3(kThreads), args, smem, h->stream);
    note_launch(1);
    return e;
  }
  solve_kernel<<<1, kThreads, smem, h->stream>>>(P, V, h->d_status, d_stats);
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace gmgm

// ---------------------------------------------------------------------------
// Allocation-free variant of the eigenvalue solve (gmgm_eigsolve_static).
//
// Some callers cannot allocate device memory when they call the library:
// a host that has reserved the whole device for its own allocator, a
// latency-critical loop that cannot afford cudaMalloc's implicit device
// synchronisation, or a plugin whose memory budget is fixed up front.  For
// them this entry point takes no handle and allocates nothing: its working
// vectors, status word and statistics live in one file-scope device array of
// fixed size, reserved when the library is loaded and held by every device
// that loads it until the process exits.
// ---------------------------------------------------------------------------

namespace gmgm {
namespace {

constexpr int kStaticMaxRank = 4096;  // sum of the ranks accepted
constexpr size_t kStaticVecBytes =
    size_t(kStaticMaxRank) * (13 * sizeof(double) + 2 * sizeof(float) + sizeof(int)) + 20 * 256;
constexpr size_t kStaticBytes = kStaticVecBytes + 1024;  // + status word and stats

}  // namespace

// The scratch of gmgm_eigsolve_static.  In host code this name is only a
// stand-in for the symbol; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_solve_static[kStaticBytes];

namespace {

// The array's device address on the current device, looked up on every call
// (no allocation; a cached address would dangle after a device reset
// reloads the module).
int static_scratch(int device, void** out) {
  if (device < 0) return GMGM_E_ARG;
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_solve_static) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return GMGM_E_CUDA;
  }
  *out = ptr;
  return GMGM_OK;
}

}  // namespace

}  // namespace gmgm

extern "C" int gmgm_eigsolve_static(const gmgm_problem* p, const double* const* init, const gmgm_solve_opts* o,
                                    double* const* lambda_out, gmgm_solve_stats* stats, void* cuda_stream) {
  using namespace gmgm;
  if (!p || !lambda_out) return GMGM_E_ARG;
  if (p->n_axes < 1 || p->n_axes > GMGM_MAX_AXES || p->n_modalities < 1 || p->n_modalities > GMGM_MAX_MODALITIES)
    return GMGM_E_ARG;
  int64_t total = 0;
  for (int a = 0; a < p->n_axes; ++a) {
    if (p->r[a] < 1 || !p->E[a] || !lambda_out[a] || (init && !init[a])) return GMGM_E_ARG;
    total += p->r[a];
  }
  if (total > kStaticMaxRank) return GMGM_E_ARG;  // beyond the fixed scratch
  int used[GMGM_MAX_AXES] = {0, 0, 0, 0};
  for (int g = 0; g < p->n_modalities; ++g) {
    const int k = p->mod_n_axes[g];
    if (k < 1 || k > GMGM_MAX_AXES) return GMGM_E_ARG;
    int seen = 0;
    int64_t pts = 1;
    for (int q = 0; q < k; ++q) {
      const int a = p->mod_axes[g][q];
      if (a < 0 || a >= p->n_axes || (seen & (1 << a))) return GMGM_E_ARG;
      seen |= 1 << a;
      used[a] = 1;
      pts *= p->r[a];
    }
    if (pts > (int64_t(1) << 31)) return GMGM_E_ARG;
  }
  for (int a = 0; a < p->n_axes; ++a)
    if (!used[a]) return GMGM_E_ARG;
  gmgm_solve_opts opt = {1e-9, 200, 200, 1, 1, 0.0};
  if (o) {
    opt = *o;
    if (opt.tol <= 0) opt.tol = 1e-9;
    if (opt.max_newton <= 0) opt.max_newton = 200;
    if (opt.max_cg <= 0) opt.max_cg = 200;
  }
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return GMGM_E_CUDA;
  }
  void* base = nullptr;
  int rc = static_scratch(device, &base);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // layout of the array: vectors, then the status word, then the stats
  char* b = static_cast<char*>(base);
  int* d_status = reinterpret_cast<int*>(b + kStaticVecBytes);
  gmgm_solve_stats* d_stats = reinterpret_cast<gmgm_solve_stats*>(b + kStaticVecBytes + 256);
  Params P{};
  P.L = p->n_axes;
  P.off[0] = 0;
  for (int a = 0; a < P.L; ++a) {
    P.r[a] = p->r[a];
    P.off[a + 1] = P.off[a] + p->r[a];
    P.eps[a] = p->eps[a];
    P.E[a] = p->E[a];
    P.init[a] = init ? init[a] : nullptr;
    P.out[a] = lambda_out[a];
  }
  P.N = P.off[P.L];
  P.nmod = p->n_modalities;
  for (int g = 0; g < P.nmod; ++g) {
    P.mk[g] = p->mod_n_axes[g];
    for (int q = 0; q < P.mk[g]; ++q) P.ma[g][q] = p->mod_axes[g][q];
  }
  P.tol = opt.tol;
  P.max_newton = opt.max_newton;
  P.max_cg = opt.max_cg;
  P.fp32_phase = opt.fp32_phase;
  P.gauge = opt.gauge;
  P.trace_rtol = opt.trace_rtol == 0.0 ? 1e-6 : opt.trace_rtol;
  P.has_init = init != nullptr;
  Carve c(base);
  const int N = P.N;
  Vecs V;
  V.E = c.take<double>(N);
  V.x = c.take<double>(N);
  V.g = c.take<double>(N);
  V.lo = c.take<double>(N);
  V.hd = c.take<double>(N);
  V.d = c.take<double>(N);
  V.rr = c.take<double>(N);
  V.z = c.take<double>(N);
  V.p = c.take<double>(N);
  V.hp = c.take<double>(N);
  V.dx = c.take<double>(N);
  V.s1 = c.take<double>(N);
  V.s2 = c.take<double>(N);
  V.x32 = c.take<float>(N);
  V.v32 = c.take<float>(N);
  V.act = c.take<int>(N);
  // the array keeps the previous call's contents: the status word starts at zero
  if (cudaMemsetAsync(d_status, 0, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return GMGM_E_CUDA;
  }
  const size_t smem = size_t(2) * kMaxLoop * sizeof(double);
  if (cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) {
    cudaGetLastError();
    return GMGM_E_CUDA;
  }
  solve_kernel<<<1, kThreads, smem, st>>>(P, V, d_status, d_stats);
  if (cudaGetLastError() != cudaSuccess) return GMGM_E_CUDA;
  note_launch(1);
  if (stats) {
    if (cudaMemcpyAsync(stats, d_stats, sizeof(gmgm_solve_stats), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return GMGM_E_CUDA;
    }
    return stats->status;
  }
  return GMGM_OK;
}

