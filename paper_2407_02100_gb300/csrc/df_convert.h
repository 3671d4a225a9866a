// Conversions between double and double-float (a value hi + lo of two
// floats) by integer operations on the IEEE-754 bit patterns.  GB300 runs
// FP64 instructions and the F2F conversions to and from FP64 at about 1/74
// of its FP32 rate, so the double-float sweep of FP64 problems converts its
// inputs and outputs with these integer forms instead.  Host and device
// compile the same code (it is checked on the host against exact
// arithmetic).
//
// to_df: hi is x truncated to 24 significant bits, lo the remaining 29 bits
//   rounded to 24 (|lo| < ulp(hi)), so hi + lo = x to 2^-47 relative.  Exact
//   integer path for 2^-74 <= |x| < 2^115; other magnitudes (zero aside) take
//   the rounded FP64 path; zero and FP64 subnormals give (0, 0).  The range
//   of double-float is that of float: below |x| = 2^-100 lo is a float
//   subnormal and the error becomes absolute (at most 2^-149); from 2^128 on
//   hi is infinite.
// from_df: hi + lo rounded to double (to 2^-52 relative; the bits of lo below
//   the double's last place are truncated) for normal hi and lo with
//   |lo| <= ulp(hi) and lo far below hi or zero; other cases use the FP64 sum.
#pragma once
#include <cstdint>
#include <cstring>

namespace gmg {
namespace dfconv {

#if defined(__CUDA_ARCH__)
#define GMG_DFC __device__ __forceinline__
// the FP64 fallbacks live in functions of their own, so that the compiler
// does not predicate their FP64 instructions into the common path
__device__ __noinline__ void to_df_rounded(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}
__device__ __noinline__ double from_df_fp64(float hi, float lo) { return (double)hi + (double)lo; }
__device__ __forceinline__ float u2f_rn(uint32_t v) { return __uint2float_rn(v); }
__device__ __forceinline__ float fmul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(uint64_t b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ uint32_t fbits(float x) { return __float_as_uint(x); }
__device__ __forceinline__ float bitsf(uint32_t b) { return __uint_as_float(b); }
#else
#define GMG_DFC inline
inline float u2f_rn(uint32_t v) { return (float)v; }
inline float fmul_rn(float a, float b) { return a * b; }
inline uint64_t dbits(double x) { uint64_t b; std::memcpy(&b, &x, 8); return b; }
inline double bitsd(uint64_t b) { double x; std::memcpy(&x, &b, 8); return x; }
inline uint32_t fbits(float x) { uint32_t b; std::memcpy(&b, &x, 4); return b; }
inline float bitsf(uint32_t b) { float x; std::memcpy(&x, &b, 4); return x; }
inline void to_df_rounded(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}
inline double from_df_fp64(float hi, float lo) { return (double)hi + (double)lo; }
#endif

GMG_DFC void to_df(double x, float& hi, float& lo) {
  const uint64_t b = dbits(x);
  const int e = (int)((b >> 52) & 0x7FF);  // biased exponent
  if (e == 0) {                            // zero or FP64 subnormal (below the float range)
    hi = 0.f;
    lo = 0.f;
    return;
  }
  if (e < 949 || e > 1137) {  // outside the exact integer path: rounded conversions
    to_df_rounded(x, hi, lo);
    return;
  }
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;  // 52 explicit significand bits
  hi = bitsf(sign | ((uint32_t)(e - 896) << 23) | (uint32_t)(m >> 29));
  // x - hi = (low 29 bits) * 2^(e - 1075), with the sign of x; e >= 949 keeps
  // the scale 2^(e - 1075) a normal float
  const float r = fmul_rn(u2f_rn((uint32_t)(m & 0x1FFFFFFFu)), bitsf((uint32_t)(e - 948) << 23));
  lo = sign ? -r : r;
}

GMG_DFC double from_df(float hi, float lo) {
  const uint32_t hb = fbits(hi), lb = fbits(lo);
  const int eh = (int)((hb >> 23) & 0xFF), el = (int)((lb >> 23) & 0xFF);
  if (eh == 0 || eh == 255 || el == 255 || (el == 0 && (lb & 0x7FFFFFFFu) != 0) || el > eh - 24)
    return from_df_fp64(hi, lo);  // zero or subnormal hi, inf/nan, subnormal or large lo
  const uint64_t sgn = (uint64_t)(hb & 0x80000000u) << 32;
  int64_t S = (int64_t)((hb & 0x7FFFFFu) | 0x800000u) << 29;  // 53 bits, units 2^(eh - 127 - 52)
  int ex = eh - 127 + 1023;
  if (el != 0) {
    const int64_t L = (int64_t)((lb & 0x7FFFFFu) | 0x800000u);  // units 2^(el - 127 - 23)
    const int d = eh - el - 29;                                  // L in units of S: L * 2^-d, d >= -5
    const int64_t Ls = d >= 63 ? 0 : d >= 0 ? (L >> d) : (L << -d);
    S = ((hb ^ lb) & 0x80000000u) ? S - Ls : S + Ls;
    if (S >= ((int64_t)1 << 53)) {
      S >>= 1;
      ++ex;
    } else if (S < ((int64_t)1 << 52)) {
      S <<= 1;
      --ex;
    }
  }
  return bitsd(sgn | ((uint64_t)ex << 52) | ((uint64_t)S & 0xFFFFFFFFFFFFFull));
}

#undef GMG_DFC

}  // namespace dfconv
}  // namespace gmg
