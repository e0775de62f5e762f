// Host check of the double-float arithmetic of the mixed-precision update
// (kh_df64.cuh) against FP64/long double references: the error-free
// transformations are exact, the conversions FP64 <-> double-float lose at
// most 2^-48 (relative), FP32 -> FP64 is exact, and +, -, *, /, reciprocal and
// square root on pairs stay within small multiples of 2^-48 of the exact
// result of the represented operands; FP64 -> FP32 by bits rounds as the
// conversion does. Prints the largest errors found, each
// in units of 2^-48 relative (for + and -: relative to |a| + |b|).
#include <cmath>
#include <cstdio>
#include <random>

#include "kh_df64.cuh"

using kh::df64;

static long double val(df64 a) { return (long double)a.hi + (long double)a.lo; }

int main() {
  std::mt19937_64 rng(11);
  std::uniform_real_distribution<double> u(0.0, 1.0);
  auto rnd = [&](double lo_exp, double hi_exp) {
    const double e = lo_exp + (hi_exp - lo_exp) * u(rng);
    return (u(rng) < 0.5 ? -1.0 : 1.0) * std::exp2(e) * (1.0 + u(rng));
  };
  const long double ulp48 = std::ldexp(1.0L, -48);
  long double e_sum = 0, e_prod = 0, e_conv = 0, e_back = 0, e_add = 0, e_mul = 0, e_div = 0, e_rcp = 0, e_sqrt = 0;
  long double e_mulf = 0, e_addf = 0;
  long bad_norm = 0, bad_f32 = 0;
  for (int n = 0; n < 2000000; ++n) {
    const float a = (float)rnd(-40, 40), b = (float)rnd(-40, 40);
    const kh::df64 s = kh::two_sum(a, b), p = kh::two_prod(a, b);
    e_sum = std::fmax(e_sum, std::fabs(val(s) - ((long double)a + b)));
    e_prod = std::fmax(e_prod, std::fabs(val(p) - (long double)a * b) / std::fabs((long double)a * b));
    // conversions over FP32's normal range; arithmetic on operands whose
    // results stay in it
    const double xc = rnd(-90, 120);
    const kh::df64 XC = kh::df_of_f64(xc);
    e_conv = std::fmax(e_conv, std::fabs(val(XC) - xc) / std::fabs(xc) / ulp48);
    e_back = std::fmax(e_back, std::fabs((long double)kh::f64_of_df(XC) - val(XC)) / std::fabs(val(XC)) / ulp48);
    const double x = rnd(-40, 40), y = rnd(-40, 40);
    const kh::df64 X = kh::df_of_f64(x), Y = kh::df_of_f64(y);
    if (std::fabs(X.lo) > 0.5f * std::fabs(std::nextafter(X.hi, INFINITY) - X.hi) * 1.0000001f) ++bad_norm;
    const float fa = (float)rnd(-40, 40);
    const double xr = rnd(-120, 120);
    if (kh::f32_of_f64(xr) != (float)xr) ++bad_f32;
    const float fs = std::ldexp((float)(1 + (rng() % 8388607)), -149 + (int)(rng() % 23));  // subnormal
    if ((long double)kh::f64_of_f32(fs) != (long double)fs) ++bad_f32;
    if ((long double)kh::f64_of_f32(fa) != (long double)fa) ++bad_f32;
    const long double vx = val(X), vy = val(Y);
    e_add = std::fmax(e_add, std::fabs(val(X + Y) - (vx + vy)) / (std::fabs(vx) + std::fabs(vy)) / ulp48);
    e_addf = std::fmax(e_addf, std::fabs(val(X + fa) - (vx + fa)) / (std::fabs(vx) + std::fabs((long double)fa)) / ulp48);
    e_mul = std::fmax(e_mul, std::fabs(val(X * Y) - vx * vy) / std::fabs(vx * vy) / ulp48);
    e_mulf = std::fmax(e_mulf, std::fabs(val(X * fa) - vx * fa) / std::fabs(vx * fa) / ulp48);
    e_div = std::fmax(e_div, std::fabs(val(X / Y) - vx / vy) / std::fabs(vx / vy) / ulp48);
    e_rcp = std::fmax(e_rcp, std::fabs(val(kh::rcp(Y)) - 1.0L / vy) * std::fabs(vy) / ulp48);
    const kh::df64 Z = kh::dfabs(X);
    e_sqrt = std::fmax(e_sqrt, std::fabs(val(kh::dfsqrt(Z)) - std::sqrt(std::fabs(vx))) / std::sqrt(std::fabs(vx)) / ulp48);
  }
  // FP32 -> FP64 at the edges of every branch: signed zeros, the smallest and
  // largest subnormals and normals, exponent boundaries, infinities (bit for
  // bit) and NaN
  {
    const uint32_t edge[] = {0x00000000u, 0x00000001u, 0x007fffffu, 0x00800000u, 0x00800001u, 0x3f7fffffu,
                             0x3f800000u, 0x3f800001u, 0x7effffffu, 0x7f000000u, 0x7f7fffffu, 0x7f800000u};
    for (uint32_t e : edge)
      for (uint32_t sg : {0u, 0x80000000u}) {
        const float f = kh::f32_of_bits(e | sg);
        if (kh::f64_bits(kh::f64_of_f32(f)) != kh::f64_bits((double)f)) ++bad_f32;
      }
    if (!std::isnan(kh::f64_of_f32(kh::f32_of_bits(0x7fc00000u)))) ++bad_f32;
    for (uint32_t q = 0; q < 4000000u; ++q) {  // every exponent, random significands
      const uint32_t bits = (uint32_t)(rng() & 0xffffffffu);
      const float f = kh::f32_of_bits(bits);
      if (std::isnan(f)) continue;
      if (kh::f64_bits(kh::f64_of_f32(f)) != kh::f64_bits((double)f)) ++bad_f32;
    }
  }
  std::printf("%.3Le %.3Le %.3Le %.3Le %.3Le %.3Le %.3Le %.3Le %.3Le %.3Le %.3Le %ld %ld\n", e_sum, e_prod, e_conv, e_back,
              e_add, e_addf, e_mul, e_mulf, e_div, e_rcp, e_sqrt, bad_norm, bad_f32);
  return 0;
}
