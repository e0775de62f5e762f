// Forward-mode dual numbers with N tangent directions, for the local
// Jacobians of the adjoint step (reconstruction, face physics, sources and
// the conserved-from-primitive map). Every operation carries the value and
// N directional derivatives. Branches follow the value (the branch the
// forward pass took); fmax/fmin pass the derivative of the larger/smaller
// argument, the first one on ties; |x| and sqrt take the + branch at 0 and
// sqrt a zero derivative there.
#pragma once

#include <math.h>

#include "kh_physics.cuh"

namespace kh {

// keep the plain-double overloads visible next to the dual ones
using ::fabs;
using ::fmax;
using ::fmin;
using ::isfinite;
using ::sqrt;

template <int N> struct Dn {
  double v;
  double d[N];
  KH_HD Dn() {}
  KH_HD Dn(double x) : v(x) {
#pragma unroll
    for (int q = 0; q < N; ++q) d[q] = 0.0;
  }
  // the independent variable number q with value x
  KH_HD static Dn var(double x, int q) {
    Dn r(x);
    r.d[q] = 1.0;
    return r;
  }
};

template <int N> KH_HD Dn<N> operator-(const Dn<N>& a) {
  Dn<N> r;
  r.v = -a.v;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = -a.d[q];
  return r;
}
template <int N> KH_HD Dn<N> operator+(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = a.d[q] + b.d[q];
  return r;
}
template <int N> KH_HD Dn<N> operator-(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = a.d[q] - b.d[q];
  return r;
}
template <int N> KH_HD Dn<N> operator*(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = a.d[q] * b.v + a.v * b.d[q];
  return r;
}
template <int N> KH_HD Dn<N> operator/(const Dn<N>& a, const Dn<N>& b) {
  const double ib = 1.0 / b.v;
  Dn<N> r;
  r.v = a.v * ib;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = (a.d[q] - r.v * b.d[q]) * ib;
  return r;
}
template <int N> KH_HD Dn<N> operator+(const Dn<N>& a, double b) {
  Dn<N> r = a;
  r.v += b;
  return r;
}
template <int N> KH_HD Dn<N> operator+(double a, const Dn<N>& b) { return b + a; }
template <int N> KH_HD Dn<N> operator-(const Dn<N>& a, double b) {
  Dn<N> r = a;
  r.v -= b;
  return r;
}
template <int N> KH_HD Dn<N> operator-(double a, const Dn<N>& b) {
  Dn<N> r = -b;
  r.v += a;
  return r;
}
template <int N> KH_HD Dn<N> operator*(const Dn<N>& a, double b) {
  Dn<N> r;
  r.v = a.v * b;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = a.d[q] * b;
  return r;
}
template <int N> KH_HD Dn<N> operator*(double a, const Dn<N>& b) { return b * a; }
template <int N> KH_HD Dn<N> operator/(const Dn<N>& a, double b) { return a * (1.0 / b); }
template <int N> KH_HD Dn<N> operator/(double a, const Dn<N>& b) {
  const double ib = 1.0 / b.v;
  Dn<N> r;
  r.v = a * ib;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = -r.v * b.d[q] * ib;
  return r;
}
template <int N> KH_HD Dn<N>& operator+=(Dn<N>& a, const Dn<N>& b) { return a = a + b; }
template <int N> KH_HD Dn<N>& operator-=(Dn<N>& a, const Dn<N>& b) { return a = a - b; }
template <int N> KH_HD Dn<N>& operator*=(Dn<N>& a, const Dn<N>& b) { return a = a * b; }
template <int N> KH_HD Dn<N>& operator*=(Dn<N>& a, double b) { return a = a * b; }

#define KH_DN_CMP(OP)                                                                              \
  template <int N> KH_HD bool operator OP(const Dn<N>& a, const Dn<N>& b) { return a.v OP b.v; } \
  template <int N> KH_HD bool operator OP(const Dn<N>& a, double b) { return a.v OP b; }         \
  template <int N> KH_HD bool operator OP(double a, const Dn<N>& b) { return a OP b.v; }
KH_DN_CMP(<)
KH_DN_CMP(>)
KH_DN_CMP(<=)
KH_DN_CMP(>=)
#undef KH_DN_CMP

template <int N> KH_HD Dn<N> sqrt(const Dn<N>& a) {
  Dn<N> r;
  r.v = ::sqrt(a.v);
  const double f = r.v > 0.0 ? 0.5 / r.v : 0.0;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = a.d[q] * f;
  return r;
}
template <int N> KH_HD Dn<N> krsqrt(const Dn<N>& a) {
  Dn<N> r;
  r.v = 1.0 / ::sqrt(a.v);
  const double f = -0.5 * r.v / a.v;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = a.d[q] * f;
  return r;
}
template <int N> KH_HD Dn<N> kdiv(const Dn<N>& a, const Dn<N>& b) { return a / b; }
template <int N> KH_HD Dn<N> kdiv(const Dn<N>& a, double b) { return a / b; }
template <int N> KH_HD Dn<N> kdiv(double a, const Dn<N>& b) { return a / b; }
template <int N> KH_HD Dn<N> fabs(const Dn<N>& a) { return a.v < 0.0 ? -a : a; }
template <int N> KH_HD Dn<N> fmax(const Dn<N>& a, const Dn<N>& b) { return a.v >= b.v ? a : b; }
template <int N> KH_HD Dn<N> fmax(double a, const Dn<N>& b) { return a >= b.v ? Dn<N>(a) : b; }
template <int N> KH_HD Dn<N> fmax(const Dn<N>& a, double b) { return a.v >= b ? a : Dn<N>(b); }
template <int N> KH_HD Dn<N> fmin(const Dn<N>& a, const Dn<N>& b) { return a.v <= b.v ? a : b; }
template <int N> KH_HD bool isfinite(const Dn<N>& a) { return ::isfinite(a.v); }

}  // namespace kh
