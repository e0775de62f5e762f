// Floating-point operation counting for the oracle (test infrastructure only).
//
// Cnt carries a double value; every +, -, *, / and square root on it (or
// between it and a plain double) adds one to the counter of its kind, so the
// oracle's templated point physics instantiated on Cnt reports how many
// floating-point operations a formula takes. pow(x, 2) counts as one
// multiplication (it is x * x); negation, |x| and comparisons count nothing.
#pragma once
#include <cmath>

namespace oracle {

struct OpCounts {
  long long add = 0, mul = 0, div = 0, sqrt = 0;
  long long total() const { return add + mul + div + sqrt; }
};
inline OpCounts& op_counts() {
  static thread_local OpCounts c;
  return c;
}

struct Cnt {
  double v;
  Cnt() : v(0.0) {}
  Cnt(double x) : v(x) {}
};
inline double val(const Cnt& x) { return x.v; }

inline Cnt operator+(Cnt a, Cnt b) { ++op_counts().add; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++op_counts().add; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++op_counts().mul; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++op_counts().div; return Cnt(a.v / b.v); }
inline Cnt operator+(Cnt a, double b) { return a + Cnt(b); }
inline Cnt operator+(double a, Cnt b) { return Cnt(a) + b; }
inline Cnt operator-(Cnt a, double b) { return a - Cnt(b); }
inline Cnt operator-(double a, Cnt b) { return Cnt(a) - b; }
inline Cnt operator*(Cnt a, double b) { return a * Cnt(b); }
inline Cnt operator*(double a, Cnt b) { return Cnt(a) * b; }
inline Cnt operator/(Cnt a, double b) { return a / Cnt(b); }
inline Cnt operator/(double a, Cnt b) { return Cnt(a) / b; }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { return a = a + b; }
inline Cnt& operator-=(Cnt& a, Cnt b) { return a = a - b; }
inline Cnt& operator*=(Cnt& a, Cnt b) { return a = a * b; }
inline Cnt& operator+=(Cnt& a, double b) { return a = a + b; }
inline Cnt& operator*=(Cnt& a, double b) { return a = a * b; }
inline bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
inline bool operator<=(Cnt a, Cnt b) { return a.v <= b.v; }
inline bool operator>=(Cnt a, Cnt b) { return a.v >= b.v; }
inline bool operator<(Cnt a, double b) { return a.v < b; }
inline bool operator>(Cnt a, double b) { return a.v > b; }
inline bool operator<=(Cnt a, double b) { return a.v <= b; }
inline bool operator>=(Cnt a, double b) { return a.v >= b; }
inline Cnt sqrt(Cnt a) { ++op_counts().sqrt; return Cnt(std::sqrt(a.v)); }
inline Cnt fabs(Cnt a) { return Cnt(std::fabs(a.v)); }
inline Cnt pow(Cnt a, double p) {
  if (p == 2.0) return a * a;
  ++op_counts().mul;  // other powers are not used on counted paths
  return Cnt(std::pow(a.v, p));
}

}  // namespace oracle
