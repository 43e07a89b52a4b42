// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// float32 numbers with |lo| <= ulp(hi)/2, about 48 significand bits, computed
// on the float32 pipe (GB300 executes float64 at 1/64 of the float32 rate).
//
// Built from error-free transformations: TwoSum (Knuth, TAOCP vol. 2), Fast2Sum
// (Dekker 1971, |a| >= |b|) and TwoProd through a fused multiply-add; the
// double-float sum and product follow Dekker's double-length algorithms (1971),
// the dot-product accumulation the compensated Dot2 of Ogita, Rump and Oishi
// (2005).  Every float32 operation is written with an explicit rounding
// intrinsic so that the compiler can neither contract nor reorder it.
#pragma once

#include <cuda_runtime.h>

namespace ctaux {

struct df64 {
  float hi, lo;
};

__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}
__device__ __forceinline__ float fast_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}
__device__ __forceinline__ float two_prod(float a, float b, float& e) {
  const float p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
  return p;
}

__device__ __forceinline__ df64 df_from(double x) {
  df64 r;
  r.hi = __double2float_rn(x);
  r.lo = __double2float_rn(x - (double)r.hi);
  return r;
}
__device__ __forceinline__ double df_to(df64 a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df64 df_zero() { return df64{0.f, 0.f}; }
__device__ __forceinline__ df64 df_neg(df64 a) { return df64{-a.hi, -a.lo}; }

// a + b, both parts summed exactly, then renormalised (accurate in cancellation)
__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
  float e, f;
  float s = two_sum(a.hi, b.hi, e);
  const float t = two_sum(a.lo, b.lo, f);
  e = __fadd_rn(e, t);
  s = fast_two_sum(s, e, e);
  e = __fadd_rn(e, f);
  df64 r;
  r.hi = fast_two_sum(s, e, r.lo);
  return r;
}
__device__ __forceinline__ df64 df_sub(df64 a, df64 b) { return df_add(a, df_neg(b)); }

// a * b: exact product of the high parts plus the two cross terms
__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
  float e;
  const float p = two_prod(a.hi, b.hi, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df64 r;
  r.hi = fast_two_sum(p, e, r.lo);
  return r;
}

// 1 / a: float32 reciprocal refined by one Newton step in double-float,
// y = y0 + y0 (1 - a y0)
__device__ __forceinline__ df64 df_recip(df64 a) {
  const df64 y0{__frcp_rn(a.hi), 0.f};
  const df64 r = df_sub(df64{1.f, 0.f}, df_mul(a, y0));
  return df_add(y0, df_mul(y0, r));
}

// Compensated accumulation of sum_k x_k y_k (Dot2): the high products and
// their running sum are kept error-free, their rounding errors and the cross
// terms with the low parts are gathered in a float32 compensation.
struct DfDot {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(df64 x, df64 y) {
    float pe, se;
    const float p = two_prod(x.hi, y.hi, pe);
    const float cross = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, pe));
    s = two_sum(s, p, se);
    c = __fadd_rn(c, __fadd_rn(se, cross));
  }
  __device__ __forceinline__ df64 value() const {
    df64 r;
    r.hi = two_sum(s, c, r.lo);
    return r;
  }
};

}  // namespace ctaux
