// df.cuh -- double-float ("df") arithmetic on the FP32 pipe.
//
// A df number is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significand bits.  On a GB300 the FP64 pipe issues ~0.5 T DFMA/s
// while the FP32 pipe issues ~35 T FFMA/s, so every hot kernel keeps its
// states in df form and does its arithmetic with error-free transformations:
//   * TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly, 6 flops;
//   * FastTwoSum (Dekker 1971): the same when |a| >= |b|, 3 flops;
//   * exact product with one fused multiply-add: p + e = a * b,
//     e = fma(a, b, -p) (the FMA form of Dekker's product).
// Products of df numbers keep the cross terms a.hi*b.lo + a.lo*b.hi and drop
// a.lo*b.lo (relative 2^-48); sums keep the low parts in a second float.
// All float operations use the _rn intrinsics so the compiler can neither
// contract nor reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace cvq {

struct df {
  float h, l;
};

// Complex amplitude stored as four floats (re.hi, re.lo, im.hi, im.lo): 16 B,
// the size of a complex128.
typedef float4 cdf;

__device__ __forceinline__ df df_make(float h, float l) { return {h, l}; }

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.h, b.h);
  s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }

__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}

// Accumulator for sums of df products: s = h + l is renormalised only by
// df_acc_get, the low part gathering rounding errors and cross terms.
struct dfacc {
  float h, l;
};

__device__ __forceinline__ void acc_zero(dfacc& s) { s.h = 0.f; s.l = 0.f; }

// s += a * b
__device__ __forceinline__ void acc_mac(dfacc& s, df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const df t = two_sum(s.h, p);
  s.h = t.h;
  s.l = __fadd_rn(s.l, __fadd_rn(t.l, e));
}

// s += a * b with b a plain float
__device__ __forceinline__ void acc_macf(dfacc& s, df a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = __fmaf_rn(a.h, b, -p);
  e = __fmaf_rn(a.l, b, e);
  const df t = two_sum(s.h, p);
  s.h = t.h;
  s.l = __fadd_rn(s.l, __fadd_rn(t.l, e));
}

// s += a
__device__ __forceinline__ void acc_add(dfacc& s, df a) {
  const df t = two_sum(s.h, a.h);
  s.h = t.h;
  s.l = __fadd_rn(s.l, __fadd_rn(t.l, a.l));
}

__device__ __forceinline__ df acc_get(const dfacc& s) { return fast_two_sum(s.h, s.l); }

// ------------------------------------------------------------ conversions

// Exact split of a double into hi + lo floats (lo carries the next 24 bits).
// Runs on the FP64 pipe: used only at the boundaries of a call.
__device__ __forceinline__ df df_from_double(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - (double)h);
  return {h, l};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ double acc_to_double(const dfacc& s) { return (double)s.h + (double)s.l; }

__device__ __forceinline__ df re_of(cdf v) { return {v.x, v.y}; }
__device__ __forceinline__ df im_of(cdf v) { return {v.z, v.w}; }
__device__ __forceinline__ cdf make_cdf(df re, df im) { return make_float4(re.h, re.l, im.h, im.l); }

}  // namespace cvq
