// Double-float arithmetic shared by the FP64 kernels (sweep, operator).
// Included by patch_kernels.cuh.
#pragma once
#include <cuda_runtime.h>

#include "df_convert.h"

namespace gmg {

// GB300 issues FP64 fused multiply-adds at about 1/74 of its FP32 rate, so
// the arithmetic of FP64 problems' sweep and level operator runs in
// double-float arithmetic on the FP32 pipe: a value is the unevaluated sum
// hi + lo of two floats (about 48 significant bits).  A product's rounding error is recovered
// exactly with one fmaf (TwoProd, after Dekker), a sum's with Knuth's
// TwoSum, and each output of a line transform accumulates its leading
// products exactly and its error terms in a second float (the Dot2 scheme
// of Ogita, Rump and Oishi).  Every operation uses the _rn intrinsics, so
// the compiler cannot contract or reassociate them.  Measured against FP64
// on whole 3D FD solves (k = 3..8): relative error below 2e-14.
struct dfv {
  float hi, lo;
};

__device__ __forceinline__ dfv df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// a + b exactly as s + e, valid when |a| >= |b| or a == 0
__device__ __forceinline__ dfv df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfv df_add(dfv a, dfv b) {
  const dfv s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfv df_neg(dfv a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfv df_mul(dfv a, dfv b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// conversions by integer operations on the bit patterns (df_convert.h): the
// F2F conversions to and from FP64 run at the FP64 rate
__device__ __forceinline__ dfv df_from_double(double x) {
  dfv r;
  dfconv::to_df(x, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ double df_to_double(dfv a) { return dfconv::from_df(a.hi, a.lo); }

// Dot2 accumulator: the exact sum of the leading products is s + (the
// rounding errors of the additions), collected with the products' errors in e
struct df_acc {
  float s, e;
};
// acc = c x (first term), c = ch + cl a constant
__device__ __forceinline__ df_acc df_acc_first(float ch, float cl, dfv x) {
  const float p = __fmul_rn(ch, x.hi);
  float e = __fmaf_rn(ch, x.hi, -p);
  e = __fmaf_rn(ch, x.lo, e);
  e = __fmaf_rn(cl, x.hi, e);
  return {p, e};
}
// acc += c x
__device__ __forceinline__ void df_acc_add(df_acc& a, float ch, float cl, dfv x) {
  const float p = __fmul_rn(ch, x.hi);
  float e = __fmaf_rn(ch, x.hi, -p);
  e = __fmaf_rn(ch, x.lo, e);
  e = __fmaf_rn(cl, x.hi, e);
  const dfv t = df_two_sum(a.s, p);
  a.s = t.hi;
  a.e = __fadd_rn(a.e, __fadd_rn(t.lo, e));
}
__device__ __forceinline__ dfv df_acc_value(df_acc a) { return df_two_sum(a.s, a.e); }

}  // namespace gmg
