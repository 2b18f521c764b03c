// Double-float arithmetic: a value is the unevaluated sum h + l of two FP32
// numbers (|l| about ulp(h)/2 or less), about 48 significant bits.  Built
// from the error-free transformations of one addition (Knuth's TwoSum) and
// one product (TwoProd through the fused multiply-add), as in Dekker's
// double-length arithmetic.  On GB300 the FP32 pipe issues 128 FMA per
// clock per SM and the FP64 pipe about one, so a double-float update of a
// few dozen FP32 operations is several times cheaper than three FP64 FMAs.
// Every operation goes through the _rn intrinsics: the compiler neither
// contracts a product into a later addition nor reorders, either of which
// would break the error-free transformations.
#pragma once

#include <cuda_runtime.h>

namespace gmgm {

struct __align__(8) dfl {
  float h, l;
};

// s + e = a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

__device__ __forceinline__ dfl df_renorm(float h, float l) {
  dfl r;
  two_sum(h, l, r.h, r.l);
  return r;
}

__device__ __forceinline__ dfl df_zero() { return dfl{0.f, 0.f}; }

// Nearest double-float of an FP64 value (FP64 pipe: use off the hot loops).
__device__ __forceinline__ dfl df_from(double x) {
  dfl r;
  r.h = __double2float_rn(x);
  r.l = __double2float_rn(x - double(r.h));
  return r;
}

// The exact FP64 value of a double-float (48 bits fit in 53).
__device__ __forceinline__ double df_val(dfl a) { return double(a.h) + double(a.l); }

// a + b: both high and both low parts added with TwoSum, the errors folded in.
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  float s, e, t, f;
  two_sum(a.h, b.h, s, e);
  two_sum(a.l, b.l, t, f);
  e = __fadd_rn(e, t);
  two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  return df_renorm(s, e);
}

__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.h, -a.l}; }

// a * b: exact product of the high parts, the cross terms added by FMA.
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_renorm(p, e);
}

// acc + a * b (one TwoSum of the high parts; the low-order terms in FP32).
__device__ __forceinline__ dfl df_fma(dfl acc, dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  float s, t;
  two_sum(acc.h, p, s, t);
  t = __fadd_rn(t, __fadd_rn(e, acc.l));
  return df_renorm(s, t);
}

// a - (x * y + z * w): the two products' high parts exact (TwoProd), both
// additions of high parts by TwoSum, every low-order term in FP32.  The
// error is a few units of 2^-48 of |a| + |x y| + |z w|.
__device__ __forceinline__ dfl df_sub2(dfl a, dfl x, dfl y, dfl z, dfl w) {
  const float p1 = __fmul_rn(-x.h, y.h);
  float e1 = __fmaf_rn(-x.h, y.h, -p1);
  e1 = __fmaf_rn(-x.h, y.l, e1);
  e1 = __fmaf_rn(-x.l, y.h, e1);
  const float p2 = __fmul_rn(-z.h, w.h);
  float e2 = __fmaf_rn(-z.h, w.h, -p2);
  e2 = __fmaf_rn(-z.h, w.l, e2);
  e2 = __fmaf_rn(-z.l, w.h, e2);
  float s1, t1, s2, t2;
  two_sum(a.h, p1, s1, t1);
  two_sum(s1, p2, s2, t2);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(a.l, e1), __fadd_rn(e2, t1)), t2);
  return df_renorm(s2, lo);
}

// a / b: FP32 quotient of the high parts, then one correction from the
// double-float remainder a - q b.
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const dfl r = df_fma(a, dfl{-q1, 0.f}, b);  // a - q1 b
  const float q2 = __fdiv_rn(r.h, b.h);
  return df_renorm(q1, q2);
}

// sqrt(a), a >= 0: FP32 root y of the high part, then one Newton step
// y + (a - y^2) / (2 y) with the remainder in double-float.
__device__ __forceinline__ dfl df_sqrt(dfl a) {
  if (!(a.h > 0.f)) return df_zero();
  const float y = __fsqrt_rn(a.h);
  const dfl r = df_fma(a, dfl{-y, 0.f}, dfl{y, 0.f});  // a - y^2
  return df_renorm(y, __fdiv_rn(r.h, __fmul_rn(2.f, y)));
}

__device__ __forceinline__ dfl df_shfl_xor(dfl a, int o) {
  return dfl{__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}

__device__ __forceinline__ dfl df_warp_sum(dfl a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_xor(a, o));
  return a;
}

// Block-wide sum (blockDim.x a multiple of 32); every thread gets the result.
// `red` is shared scratch of >= 33 entries.
__device__ __forceinline__ dfl df_block_sum(dfl a, dfl* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = df_warp_sum(a);
  __syncthreads();
  if (lane == 0) red[w] = a;
  __syncthreads();
  if (w == 0) {
    dfl t = lane < nw ? red[lane] : df_zero();
    t = df_warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

}  // namespace gmgm
