// Double-float ("df") arithmetic for the outer defect correction of the
// mixed-precision path.
//
// A value x is held as the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2: a 48-bit significand, unit roundoff 2^-48 ~ 3.6e-15.
// Every operation is built from three error-free transformations:
//   two_sum(a, b)      (s, e) with s = fl(a + b) and s + e = a + b exactly,
//                      for any a, b (Knuth, TAOCP vol. 2, Section 4.2.2)
//   fast_two_sum(a, b) the same in three operations when |a| >= |b|
//                      (Dekker, Numer. Math. 18, 1971)
//   two_prod(a, b)     (p, e) with p = fl(a b) and p + e = a b exactly, e
//                      from one fused multiply-add
// Additions are the "sloppy" double-word sum: the hi parts are added exactly,
// the lo parts once, and the pair renormalised.  Its error is a few
// 2^-48 (|a| + |b|) in absolute terms, the accuracy that the residual
// S - N(u) of O(1) operands needs (its relative accuracy is lost only under
// cancellation, where the absolute bound is what matters).
//
// GB300 issues FP32 operations at about 60 times its FP64 rate, and converts
// between FP64 and FP32 only at the FP64 rate; these kernels therefore keep
// the mixed path's outer state in df pairs and never touch a double on the
// hot path.  Fields are stored as float2 {hi, lo} per cell (8 bytes, the
// size of a double).  Every step goes through the _rn intrinsics so that the
// compiler can neither contract a product into a sum nor reassociate.
#pragma once

#include <cuda_runtime.h>

namespace pfc {

struct df {
  float hi, lo;
};

// Host-side rounding of a double constant to a df pair.
inline df df_const(double x) {
  const float hi = (float)x;
  df r;
  r.hi = hi;
  r.lo = (float)(x - (double)hi);
  return r;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  const float t = __fadd_rn(a, b);
  const float bv = __fsub_rn(t, a);
  const float av = __fsub_rn(t, bv);
  e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
  s = t;
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  const float t = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(t, a));
  s = t;
}

__device__ __forceinline__ df df_make(float s, float e) {
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df df_neg(df a) {
  df r;
  r.hi = -a.hi;
  r.lo = -a.lo;
  return r;
}

__device__ __forceinline__ df df_add(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_make(s, e);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a + b for an FP32 b.
__device__ __forceinline__ df df_add_f(df a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e = __fadd_rn(e, a.lo);
  return df_make(s, e);
}

__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_make(p, e);
}

// a * b for an FP32 b.
__device__ __forceinline__ df df_mul_f(df a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return df_make(p, e);
}

__device__ __forceinline__ df df_sqr(df a) {
  const float p = __fmul_rn(a.hi, a.hi);
  float e = __fmaf_rn(a.hi, a.hi, -p);
  e = __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, e);
  return df_make(p, e);
}

// Exact scaling by a power of two.
__device__ __forceinline__ df df_scale2(df a, float pow2) {
  df r;
  r.hi = __fmul_rn(a.hi, pow2);
  r.lo = __fmul_rn(a.lo, pow2);
  return r;
}

// Sum of six values (a 7-point neighbour sum): the hi parts accumulate
// exactly through two_sum, their rounding errors and the lo parts in plain
// FP32, and a final two_sum renormalises (safe also when the sum cancels).
__device__ __forceinline__ df df_sum6(df v0, df v1, df v2, df v3, df v4, df v5) {
  float s = v0.hi, e = 0.f, l = v0.lo, t;
  two_sum(s, v1.hi, s, t);
  e = __fadd_rn(e, t);
  l = __fadd_rn(l, v1.lo);
  two_sum(s, v2.hi, s, t);
  e = __fadd_rn(e, t);
  l = __fadd_rn(l, v2.lo);
  two_sum(s, v3.hi, s, t);
  e = __fadd_rn(e, t);
  l = __fadd_rn(l, v3.lo);
  two_sum(s, v4.hi, s, t);
  e = __fadd_rn(e, t);
  l = __fadd_rn(l, v4.lo);
  two_sum(s, v5.hi, s, t);
  e = __fadd_rn(e, t);
  l = __fadd_rn(l, v5.lo);
  df r;
  two_sum(s, __fadd_rn(e, l), r.hi, r.lo);
  return r;
}

// Unnormalised double-float accumulator for sums that are rounded to FP32 at
// the end: hi collects the hi parts exactly (two_sum), lo collects their
// rounding errors and the lo parts in plain FP32.  The value hi + lo carries
// an absolute error of a few 2^-48 times the sum of the magnitudes added,
// like a chain of df_add, at 8 instead of 11 operations per term and without
// renormalising in between.
struct dacc {
  float hi, lo;
};

__device__ __forceinline__ dacc dacc_of(df a) {
  dacc r;
  r.hi = a.hi;
  r.lo = a.lo;
  return r;
}

__device__ __forceinline__ void dacc_add(dacc& a, float hi, float lo) {
  float s, e;
  two_sum(a.hi, hi, s, e);
  a.hi = s;
  a.lo = __fadd_rn(a.lo, __fadd_rn(e, lo));
}

__device__ __forceinline__ void dacc_add(dacc& a, df b) { dacc_add(a, b.hi, b.lo); }
__device__ __forceinline__ void dacc_sub(dacc& a, df b) { dacc_add(a, -b.hi, -b.lo); }

// k * a for a df constant k and an unnormalised pair a: hi = fl(k.hi a.hi),
// lo = its exact rounding error plus the cross terms (k.lo a.lo dropped).
__device__ __forceinline__ dacc dacc_mul(df k, dacc a) {
  dacc r;
  r.hi = __fmul_rn(k.hi, a.hi);
  r.lo = __fmaf_rn(k.lo, a.hi, __fmaf_rn(k.hi, a.lo, __fmaf_rn(k.hi, a.hi, -r.hi)));
  return r;
}

__device__ __forceinline__ float dacc_round(dacc a) { return __fadd_rn(a.hi, a.lo); }

// The value rounded to FP32.
__device__ __forceinline__ float df_round(df a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ df df_ld(const float2* __restrict__ p, int i) {
  const float2 v = __ldg(p + i);
  df r;
  r.hi = v.x;
  r.lo = v.y;
  return r;
}

__device__ __forceinline__ void df_st(float2* p, int i, df v) { p[i] = make_float2(v.hi, v.lo); }

// Conversions at the API boundary (these use the FP64 pipe).
__device__ __forceinline__ df df_from_double(double x) {
  df r;
  r.hi = __double2float_rn(x);
  r.lo = __double2float_rn(x - (double)r.hi);
  return r;
}

__device__ __forceinline__ double df_to_double(float2 v) { return (double)v.x + (double)v.y; }

}  // namespace pfc
