// Double-float arithmetic on the FP32 pipes (GB300's FP64 rate is a small
// fraction of its FP32 rate): FP64 values split into FP32 hi + lo, products
// formed by TwoProd (an exact FMA residual, Dekker 1971) plus cross terms,
// sums kept as a (sum, compensation) pair by Knuth's TwoSum (TAOCP vol. 2,
// Sec. 4.2.2).  __fadd_rn / __fsub_rn / __fmul_rn keep the compiler from
// fusing the steps.
#pragma once

#include <cuda_runtime.h>

namespace pcx {
namespace dfloat {

// v = hi + lo up to 2^-47 |v| for 2^-126 <= |v| < 2^128, with integer
// operations only: hi = the leading 24 significand bits, lo = the remainder
// rounded to 24 bits.  Magnitudes below 2^-126 give 0, at or above 2^128 NaN.
__device__ __forceinline__ void split(double v, float& hi, float& lo) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned sign = static_cast<unsigned>(b >> 63) << 31;
  const int ex = static_cast<int>((b >> 52) & 0x7FF);
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  const int fe = ex - 1023 + 127;
  if (fe <= 0) {   // zero, FP64 subnormal or below the FP32 normal range
    hi = lo = 0.f;
    return;
  }
  if (fe >= 255) {   // outside the FP32 range, Inf or NaN
    hi = lo = __uint_as_float(0x7fc00000u);
    return;
  }
  hi = __uint_as_float(sign | (static_cast<unsigned>(fe) << 23) | static_cast<unsigned>(mant >> 29));
  // remainder: low 29 significand bits, weight 2^(ex - 1075)
  const unsigned rem = static_cast<unsigned>(mant & 0x1FFFFFFFull);
  const int le = ex - 1075 + 127;
  const float scale = le > 0 ? __uint_as_float(static_cast<unsigned>(le) << 23) : 0.f;
  const float l = __fmul_rn(__uint2float_rn(rem), scale);
  lo = sign ? -l : l;
}

struct DF {
  float s, c;
};

// acc += p + e where p is the leading part (TwoSum) and e a small term
__device__ __forceinline__ void add(DF& acc, float p, float e) {
  const float s = __fadd_rn(acc.s, p);
  const float bb = __fsub_rn(s, acc.s);
  const float err = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.s = s;
  acc.c = __fadd_rn(acc.c, __fadd_rn(err, e));
}

// acc += (xh + xl) * y   (NEG: acc -= ...), error-free up to the lo*y rounding
template <bool NEG>
__device__ __forceinline__ void mac1(DF& acc, float xh, float xl, float y) {
  const float p = __fmul_rn(xh, y);
  float e = fmaf(xh, y, -p);   // p + e == xh * y exactly
  e = fmaf(xl, y, e);
  if (NEG) add(acc, -p, -e);
  else add(acc, p, e);
}

// acc += (xh + xl) * (yh + yl)   (NEG: acc -= ...)
template <bool NEG>
__device__ __forceinline__ void mac2(DF& acc, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  float e = fmaf(xh, yh, -p);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  e = fmaf(xl, yl, e);
  if (NEG) add(acc, -p, -e);
  else add(acc, p, e);
}

// (s, c) <- (s + c, the rounding error of that sum): the compensation stays at
// half an ulp of s (Fast2Sum; |c| <= |s| or s = 0 here).
__device__ __forceinline__ void renorm(DF& a) {
  const float s = __fadd_rn(a.s, a.c);
  a.c = __fsub_rn(a.c, __fsub_rn(s, a.s));
  a.s = s;
}

}  // namespace dfloat
}  // namespace pcx
