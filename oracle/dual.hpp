// Forward-mode dual numbers for the oracle (test infrastructure only).
//
// A Dual<T> carries a value and one directional derivative. Nesting
// (Dual<Dual<double>>) gives exact second derivatives, which the oracle uses
// for the connection coefficients of the native-coordinate metric: the metric
// itself contains first derivatives of the coordinate map.
#pragma once
#include <cmath>

namespace oracle {

template <class T> struct Dual {
  T v;  // value
  T d;  // derivative along the seeded direction
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}
  Dual(const T& x, const T& dx, int) : v(x), d(dx) {}
};

inline double val(double x) { return x; }
template <class T> inline double val(const Dual<T>& x) { return val(x.v); }

template <class T> inline Dual<T> mk(const T& x, const T& dx) { return Dual<T>(x, dx, 0); }

template <class T> inline Dual<T> operator+(const Dual<T>& a, const Dual<T>& b) { return mk<T>(a.v + b.v, a.d + b.d); }
template <class T> inline Dual<T> operator-(const Dual<T>& a, const Dual<T>& b) { return mk<T>(a.v - b.v, a.d - b.d); }
template <class T> inline Dual<T> operator*(const Dual<T>& a, const Dual<T>& b) { return mk<T>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <class T> inline Dual<T> operator/(const Dual<T>& a, const Dual<T>& b) {
  T q = a.v / b.v;
  return mk<T>(q, (a.d - q * b.d) / b.v);
}
template <class T> inline Dual<T> operator-(const Dual<T>& a) { return mk<T>(-a.v, -a.d); }
template <class T> inline Dual<T> operator+(const Dual<T>& a, double b) { return mk<T>(a.v + b, a.d); }
template <class T> inline Dual<T> operator+(double b, const Dual<T>& a) { return mk<T>(a.v + b, a.d); }
template <class T> inline Dual<T> operator-(const Dual<T>& a, double b) { return mk<T>(a.v - b, a.d); }
template <class T> inline Dual<T> operator-(double b, const Dual<T>& a) { return mk<T>(b - a.v, -a.d); }
template <class T> inline Dual<T> operator*(const Dual<T>& a, double b) { return mk<T>(a.v * b, a.d * b); }
template <class T> inline Dual<T> operator*(double b, const Dual<T>& a) { return mk<T>(a.v * b, a.d * b); }
template <class T> inline Dual<T> operator/(const Dual<T>& a, double b) { return mk<T>(a.v / b, a.d / b); }
template <class T> inline Dual<T> operator/(double b, const Dual<T>& a) { return Dual<T>(b) / a; }
template <class T> inline Dual<T>& operator+=(Dual<T>& a, const Dual<T>& b) { a = a + b; return a; }
template <class T> inline Dual<T>& operator-=(Dual<T>& a, const Dual<T>& b) { a = a - b; return a; }
template <class T> inline Dual<T>& operator*=(Dual<T>& a, const Dual<T>& b) { a = a * b; return a; }
template <class T> inline Dual<T>& operator+=(Dual<T>& a, double b) { a = a + b; return a; }
template <class T> inline Dual<T>& operator*=(Dual<T>& a, double b) { a = a * b; return a; }

template <class T> inline bool operator<(const Dual<T>& a, const Dual<T>& b) { return val(a) < val(b); }
template <class T> inline bool operator>(const Dual<T>& a, const Dual<T>& b) { return val(a) > val(b); }
template <class T> inline bool operator<=(const Dual<T>& a, const Dual<T>& b) { return val(a) <= val(b); }
template <class T> inline bool operator>=(const Dual<T>& a, const Dual<T>& b) { return val(a) >= val(b); }
template <class T> inline bool operator<(const Dual<T>& a, double b) { return val(a) < b; }
template <class T> inline bool operator>(const Dual<T>& a, double b) { return val(a) > b; }
template <class T> inline bool operator<=(const Dual<T>& a, double b) { return val(a) <= b; }
template <class T> inline bool operator>=(const Dual<T>& a, double b) { return val(a) >= b; }
template <class T> inline bool operator<(double a, const Dual<T>& b) { return a < val(b); }
template <class T> inline bool operator>(double a, const Dual<T>& b) { return a > val(b); }
template <class T> inline bool operator==(const Dual<T>& a, double b) { return val(a) == b; }
template <class T> inline bool operator!=(const Dual<T>& a, double b) { return val(a) != b; }

// Elementary functions: chain rule on each.
// At 0 the square root takes a zero derivative (the value of a clamped
// argument, e.g. a discriminant held at 0, carries no tangent).
template <class T> inline Dual<T> sqrt(const Dual<T>& a) {
  using std::sqrt;
  T s = sqrt(a.v);
  if (val(s) == 0.0) return mk<T>(s, T(0.0));
  return mk<T>(s, a.d / (2.0 * s));
}
template <class T> inline Dual<T> sin(const Dual<T>& a) {
  using std::sin; using std::cos;
  return mk<T>(sin(a.v), a.d * cos(a.v));
}
template <class T> inline Dual<T> cos(const Dual<T>& a) {
  using std::sin; using std::cos;
  return mk<T>(cos(a.v), -(a.d * sin(a.v)));
}
template <class T> inline Dual<T> exp(const Dual<T>& a) {
  using std::exp;
  T e = exp(a.v);
  return mk<T>(e, a.d * e);
}
template <class T> inline Dual<T> log(const Dual<T>& a) {
  using std::log;
  return mk<T>(log(a.v), a.d / a.v);
}
// x^p for a constant real exponent p (x > 0 unless p is an integer).
template <class T> inline Dual<T> pow(const Dual<T>& a, double p) {
  using std::pow;
  T y = pow(a.v, p);
  return mk<T>(y, a.d * (p * pow(a.v, p - 1.0)));
}
template <class T> inline Dual<T> fabs(const Dual<T>& a) { return val(a) < 0.0 ? -a : a; }

}  // namespace oracle
