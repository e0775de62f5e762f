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
KH_HD void kminmax(P2 a, P2 b, P2& mx, P2& mn) {
  kminmax(a.v.x, b.v.x, mx.v.x, mn.v.x);
  kminmax(a.v.y, b.v.y, mx.v.y, mn.v.y);
}

}  // namespace kh
