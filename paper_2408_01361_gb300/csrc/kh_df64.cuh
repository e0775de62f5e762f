// Double-float arithmetic for the mixed-precision update (host+device).
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits, computed on the FP32 pipe.
// GB300 issues FP64 arithmetic, FP64 compares and every conversion to or
// from FP64 at 1/64 of the FP32 rate, so the parts of the mixed update that
// need more than FP32 (the conserved variables entering the inversion, the
// inversion's invariants and residuals, the recovered primitives) run here
// instead, and FP64 values cross into and out of this form by integer
// operations on their bit patterns, not by conversion instructions.
//
// Error-free transformations: two-sum (Knuth, TAOCP vol. 2, 4.2.2: s + e =
// a + b for any a, b), fast two-sum (Dekker 1971: the same when |a| >= |b|)
// and the exact product p + e = a b with e from one fused multiply-add. The
// operations on pairs are the "sloppy" addition and the multiplication of
// Dekker (1971) as used in the double-double/quad-double library of Hida, Li
// and Bailey (2001); division and square root take one Newton correction of
// an FP32 quotient / root. Range: FP32's; the mixed update applies them to
// quantities scaled by powers of two to order unity.
#pragma once

#include <math.h>
#include <stdint.h>
#ifndef __CUDA_ARCH__
#include <string.h>
#endif

#include "kh_geom_math.h"

namespace kh {

KH_HD uint32_t f32_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  memcpy(&u, &x, 4);
  return u;
#endif
}
KH_HD float f32_of_bits(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, 4);
  return x;
#endif
}
KH_HD uint64_t f64_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
#endif
}
KH_HD double f64_of_bits(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}
// IEEE round-to-nearest FP32 reciprocal
KH_HD float frcp(float x) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(x);
#else
  return 1.0f / x;
#endif
}
// Rounded FP32 add / subtract / multiply that the compiler may not fuse into
// a multiply-add (the error-free transformations depend on each rounding).
KH_HD float fadd(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
KH_HD float fsub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
KH_HD float fmul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
KH_HD float u32_to_f32(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint2float_rn(u);
#else
  return (float)u;
#endif
}

struct df64 {
  float hi, lo;
};

KH_HD df64 mkdf(float hi, float lo) {
  df64 r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// s + e = a + b exactly, any a, b (Knuth's two-sum)
KH_HD df64 two_sum(float a, float b) {
  const float s = fadd(a, b);
  const float bb = fsub(s, a);
  return mkdf(s, fadd(fsub(a, fsub(s, bb)), fsub(b, bb)));
}
// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker's fast two-sum)
KH_HD df64 fast_two_sum(float a, float b) {
  const float s = fadd(a, b);
  return mkdf(s, fsub(b, fsub(s, a)));
}
// p + e = a b exactly (barring underflow)
KH_HD df64 two_prod(float a, float b) {
  const float p = fmul(a, b);
  return mkdf(p, fmaf(a, b, -p));
}

KH_HD df64 operator-(df64 a) { return mkdf(-a.hi, -a.lo); }
KH_HD df64 operator+(df64 a, df64 b) {
  const df64 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, fadd(s.lo, fadd(a.lo, b.lo)));
}
KH_HD df64 operator+(df64 a, float b) {
  const df64 s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, fadd(s.lo, a.lo));
}
KH_HD df64 operator+(float a, df64 b) { return b + a; }
KH_HD df64 operator-(df64 a, df64 b) { return a + (-b); }
KH_HD df64 operator-(df64 a, float b) { return a + (-b); }
KH_HD df64 operator-(float a, df64 b) { return (-b) + a; }
KH_HD df64 operator*(df64 a, df64 b) {
  const df64 p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}
KH_HD df64 operator*(df64 a, float b) {
  const df64 p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
KH_HD df64 operator*(float a, df64 b) { return b * a; }
// exact scaling by a power of two
KH_HD df64 scale2(df64 a, float pow2) { return mkdf(a.hi * pow2, a.lo * pow2); }
// a / b: FP32 quotient q, then q + (a - q b) / b
KH_HD df64 operator/(df64 a, df64 b) {
  const float rb = frcp(b.hi);
  const float q = a.hi * rb;
  const df64 r = a - b * q;
  return fast_two_sum(q, r.hi * rb);
}
KH_HD df64 rcp(df64 b) {
  const float rb = frcp(b.hi);
  const df64 r = mkdf(1.0f, 0.0f) - b * rb;
  return fast_two_sum(rb, r.hi * rb);
}
// square root (a >= 0): FP32 root s, then s + (a - s^2) / (2 s)
KH_HD df64 dfsqrt(df64 a) {
  if (!(a.hi > 0.0f)) return mkdf(0.0f, 0.0f);
  const float s = sqrtf(a.hi);
  const df64 s2 = two_prod(s, s);
  const float r = fadd(fsub(fsub(a.hi, s2.hi), s2.lo), a.lo);
  return fast_two_sum(s, r * (0.5f * frcp(s)));
}
KH_HD df64 dfabs(df64 a) { return a.hi < 0.0f ? -a : a; }
KH_HD df64 dfmax(df64 a, df64 b) { return (a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo)) ? a : b; }
KH_HD bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
KH_HD bool operator>(df64 a, df64 b) { return b < a; }

// FP64 -> double-float by bit operations: hi takes the top 24 bits of the
// significand, lo the next 29 rounded to FP32, then the pair is normalised.
// |x| below 2^-126 (FP32's normal range) maps to zero; beyond FP32's range to
// infinity; NaN to NaN.
KH_HD df64 df_of_f64(double x) {
  const uint64_t b = f64_bits(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const int ef = e - 896;  // FP32 biased exponent of the same power of two
  if (ef <= 0) return mkdf(f32_of_bits(sign), 0.0f);
  if (ef >= 255) {
    const bool nan = e == 2047 && (b & 0xFFFFFFFFFFFFFull) != 0;
    return mkdf(f32_of_bits(sign | (nan ? 0x7fc00000u : 0x7f800000u)), 0.0f);
  }
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;
  const float hi = f32_of_bits(sign | ((uint32_t)ef << 23) | (uint32_t)(m >> 29));
  // the remaining 29 bits weigh 2^(e - 1075) = 2^(ef - 179)
  float lo = u32_to_f32((uint32_t)(m & 0x1FFFFFFFu));
  if (ef > 52) {
    lo *= f32_of_bits((uint32_t)(ef - 52) << 23);
  } else {
    lo *= f32_of_bits((uint32_t)(ef + 12) << 23);  // 2^(ef - 115), then 2^-64 (may round)
    lo *= f32_of_bits((uint32_t)(127 - 64) << 23);
  }
  if (sign) lo = -lo;
  return fast_two_sum(hi, lo);
}
KH_HD int clz32(uint32_t v) {
#ifdef __CUDA_ARCH__
  return __clz((int)v);
#else
  int n = 0;
  while (n < 32 && !(v & (0x80000000u >> n))) ++n;
  return n;
#endif
}
// FP64 -> FP32 rounded to nearest (ties to even) by bit operations; results
// below FP32's normal range map to zero, beyond it to infinity.
KH_HD float f32_of_f64(double x) {
  const uint64_t b = f64_bits(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const int ef = e - 896;
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;
  if (e == 2047) return f32_of_bits(sign | (m ? 0x7fc00000u : 0x7f800000u));
  if (ef <= 0) return f32_of_bits(sign);
  if (ef >= 255) return f32_of_bits(sign | 0x7f800000u);
  uint32_t r = ((uint32_t)ef << 23) | (uint32_t)(m >> 29);
  const uint32_t rem = (uint32_t)(m & 0x1FFFFFFFu);
  r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;  // a carry moves into the exponent
  return f32_of_bits(sign | r);
}
// FP32 -> FP64 exactly by bit operations (subnormals included)
KH_HD double f64_of_f32(float x) {
  const uint32_t u = f32_bits(x);
  const uint32_t ef = (u >> 23) & 0xffu;
  const uint32_t m = u & 0x7fffffu;
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  if (ef == 0) {
    if (m == 0) return f64_of_bits(sign);
    // m 2^-149 with the leading one of m at bit q: 2^(q - 149) (1 + ...)
    const int q = 31 - clz32(m);
    const uint64_t mm = ((uint64_t)m << (52 - q)) & 0xFFFFFFFFFFFFFull;
    return f64_of_bits(sign | ((uint64_t)(q - 149 + 1023) << 52) | mm);
  }
  const uint64_t e = ef == 255 ? 2047 : ef + 896;
  return f64_of_bits(sign | (e << 52) | ((uint64_t)m << 29));
}
// double-float -> FP64 (hi and lo are exact in FP64; their sum rounds once)
KH_HD double f64_of_df(df64 a) { return f64_of_f32(a.hi) + f64_of_f32(a.lo); }

}  // namespace kh
