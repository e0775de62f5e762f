// Packed FP32 pairs for the mixed path's face physics (host+device).
//
// The left and right states of a face go through the same arithmetic, so the
// face kernels carry them as one pair value and issue sm_100-family paired
// FP32 instructions (two FP32 operations per lane per instruction:
// __ffma2_rn, __fadd2_rn, __fmul2_rn), halving the issue slots of that part;
// the FP32 face kernels are issue-bound. A product of two pairs is kept
// unevaluated until it meets an addition, which then becomes one paired fused
// multiply-add (the rounding of a contracted a*b + c). Per component the
// results are those of the scalar FP32 operations (round to nearest).
#pragma once

#include "kh_physics.cuh"

namespace kh {

using ::sqrt;  // keep the scalar overloads visible beside the pair one

struct P2 {
  float2 v;
  KH_HD P2() {}
  KH_HD P2(float a) { v.x = a; v.y = a; }  // both components
  KH_HD P2(float a, float b) { v.x = a; v.y = b; }
  KH_HD static P2 of(float2 x) {
    P2 r;
    r.v = x;
    return r;
  }
};

KH_HD P2 pmul(P2 a, P2 b) {
#ifdef __CUDA_ARCH__
  return P2::of(__fmul2_rn(a.v, b.v));
#else
  return P2(a.v.x * b.v.x, a.v.y * b.v.y);
#endif
}
KH_HD P2 padd(P2 a, P2 b) {
#ifdef __CUDA_ARCH__
  return P2::of(__fadd2_rn(a.v, b.v));
#else
  return P2(a.v.x + b.v.x, a.v.y + b.v.y);
#endif
}
KH_HD P2 pfma(P2 a, P2 b, P2 c) {
#ifdef __CUDA_ARCH__
  return P2::of(__ffma2_rn(a.v, b.v, c.v));
#else
  return P2(fmaf(a.v.x, b.v.x, c.v.x), fmaf(a.v.y, b.v.y, c.v.y));
#endif
}
KH_HD P2 operator-(P2 a) { return P2(-a.v.x, -a.v.y); }

// a * b, not yet rounded
struct P2Prod {
  P2 a, b;
  KH_HD operator P2() const { return pmul(a, b); }
};
KH_HD P2Prod operator*(P2 a, P2 b) { return P2Prod{a, b}; }
KH_HD P2Prod operator*(float a, P2 b) { return P2Prod{P2(a), b}; }
KH_HD P2Prod operator*(P2 a, float b) { return P2Prod{a, P2(b)}; }
KH_HD P2Prod operator*(P2Prod a, P2 b) { return P2Prod{pmul(a.a, a.b), b}; }
KH_HD P2Prod operator*(P2 a, P2Prod b) { return P2Prod{a, pmul(b.a, b.b)}; }
KH_HD P2Prod operator*(P2Prod a, P2Prod b) { return P2Prod{pmul(a.a, a.b), pmul(b.a, b.b)}; }
KH_HD P2Prod operator*(P2Prod a, float b) { return P2Prod{pmul(a.a, a.b), P2(b)}; }
KH_HD P2Prod operator*(float a, P2Prod b) { return P2Prod{P2(a), pmul(b.a, b.b)}; }
KH_HD P2Prod operator-(P2Prod a) { return P2Prod{-a.a, a.b}; }

KH_HD P2 operator+(P2 a, P2 b) { return padd(a, b); }
KH_HD P2 operator-(P2 a, P2 b) { return padd(a, -b); }
KH_HD P2 operator+(P2Prod p, P2 c) { return pfma(p.a, p.b, c); }
KH_HD P2 operator+(P2 c, P2Prod p) { return pfma(p.a, p.b, c); }
KH_HD P2 operator-(P2 c, P2Prod p) { return pfma(-p.a, p.b, c); }
KH_HD P2 operator-(P2Prod p, P2 c) { return pfma(p.a, p.b, -c); }
KH_HD P2 operator+(P2Prod p, P2Prod q) { return pfma(p.a, p.b, pmul(q.a, q.b)); }
KH_HD P2 operator-(P2Prod p, P2Prod q) { return pfma(p.a, p.b, pmul(-q.a, q.b)); }
KH_HD P2 operator+(P2 a, float b) { return padd(a, P2(b)); }
KH_HD P2 operator+(float a, P2 b) { return padd(P2(a), b); }
KH_HD P2 operator-(P2 a, float b) { return padd(a, P2(-b)); }
KH_HD P2 operator-(float a, P2 b) { return padd(P2(a), -b); }
KH_HD P2 operator+(P2Prod p, float c) { return pfma(p.a, p.b, P2(c)); }
KH_HD P2 operator-(P2Prod p, float c) { return pfma(p.a, p.b, P2(-c)); }
KH_HD P2 operator+(float c, P2Prod p) { return pfma(p.a, p.b, P2(c)); }
KH_HD P2 operator-(float c, P2Prod p) { return pfma(-p.a, p.b, P2(c)); }
KH_HD P2& operator+=(P2& a, P2 b) { return a = a + b; }
KH_HD P2& operator+=(P2& a, P2Prod b) { return a = a + b; }

// element-wise functions (one scalar instruction per component)
KH_HD P2 krsqrt(P2 a) { return P2(krsqrt(a.v.x), krsqrt(a.v.y)); }
KH_HD P2 sqrt(P2 a) { return P2(sqrtf(a.v.x), sqrtf(a.v.y)); }
KH_HD P2 kdiv(P2 a, P2 b) { return P2(kdiv(a.v.x, b.v.x), kdiv(a.v.y, b.v.y)); }
KH_HD P2 kdiv(P2 a, float b) { return P2(kdiv(a.v.x, b), kdiv(a.v.y, b)); }
KH_HD P2 kdiv(P2Prod a, P2 b) { return kdiv(P2(a), b); }
KH_HD P2 kdiv(P2 a, P2Prod b) { return kdiv(a, P2(b)); }
KH_HD P2 kclamp01(P2 a) { return P2(kclamp01(a.v.x), kclamp01(a.v.y)); }
KH_HD P2 kmax0(P2 a) { return P2(kmax0(a.v.x), kmax0(a.v.y)); }
// the FP32 scale-free WENO5 value at x = +1/2 (weno5_plus(float...)) of two
// stencils at once
KH_HD P2 weno5_plus(P2 a, P2 b, P2 c, P2 d, P2 e) {
  const P2 p0 = P2(0.375f) * a + (P2(-1.25f) * b + P2(1.875f) * c);
  const P2 p1 = P2(-0.125f) * b + (P2(0.75f) * c + P2(0.375f) * d);
  const P2 p2 = P2(0.375f) * c + (P2(0.75f) * d + P2(-0.125f) * e);
  const P2 k(13.0f / 12.0f), q4(0.25f);
  const P2 t0 = P2(-2.0f) * b + (a + c), u0 = P2(3.0f) * c + (a - P2(4.0f) * b);
  const P2 t1 = P2(-2.0f) * c + (b + d), u1 = b - d;
  const P2 t2 = P2(-2.0f) * d + (c + e), u2 = P2(3.0f) * c + (e - P2(4.0f) * d);
  const P2 b0 = (k * t0) * t0 + (q4 * u0) * u0;
  const P2 b1 = (k * t1) * t1 + (q4 * u1) * u1;
  const P2 b2 = (k * t2) * t2 + (q4 * u2) * u2;
  const P2 sum = b0 + b1 + b2 + 1e-37f;
#ifdef __CUDA_ARCH__
  const P2 in(__frcp_rn(sum.v.x), __frcp_rn(sum.v.y));
#else
  const P2 in(1.0f / sum.v.x, 1.0f / sum.v.y);
#endif
  const P2 eps(1e-12f);
  const P2 s0 = b0 * in + eps, s1 = b1 * in + eps, s2 = b2 * in + eps;
  const P2 sm(fminf(s0.v.x, fminf(s1.v.x, s2.v.x)), fminf(s0.v.y, fminf(s1.v.y, s2.v.y)));
  const P2 r0 = kdiv(sm, s0), r1 = kdiv(sm, s1), r2 = kdiv(sm, s2);
  const P2 w0 = (P2(0.0625f) * r0) * r0, w1 = (P2(0.625f) * r1) * r1, w2 = (P2(0.3125f) * r2) * r2;
  return kdiv(w0 * p0 + (w1 * p1 + w2 * p2), w0 + w1 + w2);
}

KH_HD void kminmax(P2 a, P2 b, P2& mx, P2& mn) {
  kminmax(a.v.x, b.v.x, mx.v.x, mn.v.x);
  kminmax(a.v.y, b.v.y, mx.v.y, mn.v.y);
}

}  // namespace kh
