// Mixed-precision inversion without the FP64 pipe: the Noble et al. (2006)
// two-unknown (W, v^2) equations of noble2d, with
//   * the invariants D, Q.n, Q~^2, B^2, (Q.B)^2 formed in double-float
//     arithmetic from the double-float conserved variables and metric, on the
//     problem scaled by S = 4^k ~ W (fluid conserved variables times 1/S, the
//     field times 1/sqrt(S): every term of the momentum residual then scales
//     as S^2 and of the energy residual as S, exactly);
//   * Newton's iterations in FP32 on the scaled invariants (their hi parts),
//     started from the stage input's (W, v^2);
//   * refinement steps with both residuals in double-float and the FP32
//     Jacobian (its FP32 error multiplies a step of ~1e-7), until a step is
//     below 1e-5 (at most three) -- the iterate then lies in Newton's
//     quadratic regime, its error ~ the step squared (one step from a
//     converged FP32 root; more where FP32 rounding stalled the FP32 phase);
//   * the primitives recovered in double-float.
// A zone whose FP32 phase or refinement does not meet these conditions is
// reported (C2P_NEED_FP64) and the caller runs the FP64 inversion for it.
#pragma once

#include "kh_df64.cuh"
#include "kh_physics.cuh"

namespace kh {

constexpr int C2P_NEED_FP64 = -1;

// Double-float (hi, lo FP32 pair) copies of the cell-centre quantities the
// mixed update's inversion and floors use, per (i, j): planes [NDF][n2s][n1s]
// of (hi, lo) float pairs, so that one 8-byte load brings both halves.
// DF_GCON0: g^{0m} (m = 0..3); DF_GSP: gamma^{ij} = g^{ij} - g^{0i} g^{0j} / g^{00},
// the inverse of the spatial metric (11 12 13 22 23 33), formed in FP64 at
// setup; DF_GCOV: g_ij (same order).
enum { DF_GCON0 = 0, DF_GSP = 4, DF_GCOV = 10, DF_ALPHA = 16, DF_IG = 17, DF_RHOFL = 18, DF_UFL = 19, NDF = 20 };

// FP32 and double-float constants of the mixed update (host: set_mixed()).
struct MixedConsts {
  float gfac_hi, gfac_lo;  // (gam - 1) / gam as a double-float pair
  float igam_hi, igam_lo;  // 1 / gam
  float gam;
  float ibsq_rho_max, ibsq_u_max, u_rho_max, g2max;  // floors: 1/(b^2/rho)max, 1/(b^2/u)max, (u/rho)max, gamma_max^2
};

// Host: the constants from the FP64 adiabatic index and floors (hi = the
// nearest FP32, lo = the rest).
inline MixedConsts mixed_consts(double gam, const FloorParams& fl) {
  auto split = [](double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  };
  MixedConsts k;
  split((gam - 1.0) / gam, k.gfac_hi, k.gfac_lo);
  split(1.0 / gam, k.igam_hi, k.igam_lo);
  k.gam = (float)gam;
  k.ibsq_rho_max = (float)fl.ibsq_rho_max;
  k.ibsq_u_max = (float)fl.ibsq_u_max;
  k.u_rho_max = (float)fl.u_rho_max;
  const double g2 = fl.gamma_max * fl.gamma_max;
  k.g2max = g2 < 3.0e38 ? (float)g2 : 3.0e38f;
  return k;
}

struct MetDF {
  df64 gcon0[4];  // g^{0m}
  df64 gsp[6];    // gamma^{ij}: 11 12 13 22 23 33
  df64 gcov[6];   // g_ij: 11 12 13 22 23 33
  df64 alpha, ig, rho_fl, u_fl;
};

#ifdef __CUDACC__
__device__ __forceinline__ MetDF load_metdf(const float* df, long long gplane, long long p) {
  const float2* d2 = reinterpret_cast<const float2*>(df);  // (hi, lo) pairs: one 8-byte load each
  auto ld = [&](int q) {
    const float2 v = __ldg(d2 + q * gplane + p);
    return mkdf(v.x, v.y);
  };
  MetDF m;
#pragma unroll
  for (int q = 0; q < 4; ++q) m.gcon0[q] = ld(DF_GCON0 + q);
#pragma unroll
  for (int q = 0; q < 6; ++q) m.gsp[q] = ld(DF_GSP + q);
#pragma unroll
  for (int q = 0; q < 6; ++q) m.gcov[q] = ld(DF_GCOV + q);
  m.alpha = ld(DF_ALPHA);
  m.ig = ld(DF_IG);
  m.rho_fl = ld(DF_RHOFL);
  m.u_fl = ld(DF_UFL);
  return m;
}
#endif

// g_ij x^i x^j for a spatial vector (double-float)
KH_HD df64 spatial_sq(const MetDF& m, df64 a, df64 b, df64 c) {
  const df64 d = m.gcov[0] * (a * a) + m.gcov[3] * (b * b) + m.gcov[5] * (c * c);
  const df64 o = m.gcov[1] * (a * b) + m.gcov[2] * (a * c) + m.gcov[4] * (b * c);
  return d + scale2(o, 2.0f);
}

// FP32 quantities the floors decide on, from the leading parts of the
// primitives P (double-float) and of the metric: u_i = g_ij u~^j (the spatial
// part of u_mu), the Lorentz factor squared gamma^2 = 1 + u~^i u_i, and
// b^2 = alpha^2 (g_ij B^i B^j + (b^t)^2) / gamma^2 with b^t = B^i u_i (that is
// (B^i B_i + (b^t)^2) / (u^t)^2, u^t = gamma / alpha).
struct FloorF32 {
  float ucov[3];  // u_1, u_2, u_3
  float g2, bsq;
};
// a0 b0 + a1 b1 + a2 b2 with every rounding explicit (a product, then two
// fused multiply-adds), so that every kernel inlining this rounds alike
KH_HD float dot3f(float a0, float b0, float a1, float b1, float a2, float b2) {
  return fmaf(a2, b2, fmaf(a1, b1, fmul(a0, b0)));
}
KH_HD FloorF32 floor_f32(const MetDF& m, const df64* P) {
  const float g11 = m.gcov[0].hi, g12 = m.gcov[1].hi, g13 = m.gcov[2].hi;
  const float g22 = m.gcov[3].hi, g23 = m.gcov[4].hi, g33 = m.gcov[5].hi;
  const float v1 = P[V_U1].hi, v2 = P[V_U2].hi, v3 = P[V_U3].hi;
  const float B1 = P[V_B1].hi, B2 = P[V_B2].hi, B3 = P[V_B3].hi;
  FloorF32 f;
  f.ucov[0] = dot3f(g11, v1, g12, v2, g13, v3);
  f.ucov[1] = dot3f(g12, v1, g22, v2, g23, v3);
  f.ucov[2] = dot3f(g13, v1, g23, v2, g33, v3);
  f.g2 = fadd(1.0f, dot3f(f.ucov[0], v1, f.ucov[1], v2, f.ucov[2], v3));
  const float bt = dot3f(f.ucov[0], B1, f.ucov[1], B2, f.ucov[2], B3);
  const float BB = dot3f(dot3f(g11, B1, g12, B2, g13, B3), B1, dot3f(g12, B1, g22, B2, g23, B3), B2,
                         dot3f(g13, B1, g23, B2, g33, B3), B3);
  const float a = m.alpha.hi;
  f.bsq = kdiv(fmul(fmul(a, a), fmaf(bt, bt, BB)), f.g2);
  return f;
}

// u^t and u_t of the same state: u^t = gamma / alpha, u_t = -alpha gamma +
// beta_i u~^i with the shift beta_i = alpha^2 g_ij g^{0j}, i.e. alpha^2 g^{0j} u_j.
KH_HD void floor_ut(const MetDF& m, const FloorF32& f, float& ut, float& u_t) {
  const float a = m.alpha.hi, gl = sqrtf(f.g2);
  ut = kdiv(gl, a);
  u_t = fmul(a, fsub(fmul(a, dot3f(m.gcon0[1].hi, f.ucov[0], m.gcon0[2].hi, f.ucov[1], m.gcon0[3].hi, f.ucov[2])), gl));
}

// U: conserved variables of the zone (double-float, densitised); W0, vsq0:
// initial guess (FP32, unscaled). On success P[0..4] holds the fluid
// primitives (B^i = U_B / sqrt(-g) is left to the caller). Returns 0, a
// noble2d failure code (2 v^2 >= 1, 3 W <= 0, 4 rho <= 0, 5 u < 0) or
// C2P_NEED_FP64.
KH_HD int noble2d_df(const df64* U, const MetDF& m, const MixedConsts& k, float W0, float vsq0, df64* P) {
  const uint32_t wb = f32_bits(W0);
  const int ew = (int)((wb >> 23) & 0xffu);
  if (!(W0 > 0.0f) || ew == 0 || ew == 255) return C2P_NEED_FP64;
  const int e2 = (ew - 127) >> 1;                    // S = 4^e2 = 2^(2 e2)
  const float S = f32_of_bits((uint32_t)(127 + 2 * e2) << 23);
  const float iS = f32_of_bits((uint32_t)(127 - 2 * e2) << 23);
  const float iSb = f32_of_bits((uint32_t)(127 - e2) << 23);  // 1 / sqrt(S)
  const df64 aig = m.alpha * m.ig;
  const df64 as = scale2(aig, iS), ab = scale2(aig, iSb);
  const df64 D = as * U[V_RHO];
  const df64 Qc[4] = {as * (U[V_U] - U[V_RHO]), as * U[V_U1], as * U[V_U2], as * U[V_U3]};
  // Q.n = -alpha Q^t (n_mu = (-alpha, 0, 0, 0))
  const df64 Qdn = -(m.alpha * (m.gcon0[0] * Qc[0] + m.gcon0[1] * Qc[1] + m.gcon0[2] * Qc[2] + m.gcon0[3] * Qc[3]));
  // Q~^i = gamma^{ij} Q_j: the part of Q^mu orthogonal to n (its time component
  // vanishes, since gamma^{i0} = g^{i0} + n^i n^0 = 0), and Q~^2 = Q~^i Q_i =
  // Q^mu Q_mu + (Q.n)^2
  const df64 Qt[3] = {m.gsp[0] * Qc[1] + m.gsp[1] * Qc[2] + m.gsp[2] * Qc[3],
                      m.gsp[1] * Qc[1] + m.gsp[3] * Qc[2] + m.gsp[4] * Qc[3],
                      m.gsp[2] * Qc[1] + m.gsp[4] * Qc[2] + m.gsp[5] * Qc[3]};
  const df64 Qtsq = dfmax(Qt[0] * Qc[1] + Qt[1] * Qc[2] + Qt[2] * Qc[3], mkdf(0.0f, 0.0f));
  const df64 Bc[3] = {ab * U[V_B1], ab * U[V_B2], ab * U[V_B3]};
  const df64 Bsq = spatial_sq(m, Bc[0], Bc[1], Bc[2]);
  const df64 QdB = Qc[1] * Bc[0] + Qc[2] * Bc[1] + Qc[3] * Bc[2];
  const df64 QdB2 = QdB * QdB;
  const df64 gf = mkdf(k.gfac_hi, k.gfac_lo);

  // FP32 phase on the scaled invariants
  float Wf = W0 * iS, vf = vsq0, ef = 1.0f;
  if (!(vf >= 0.0f)) vf = 0.0f;
  if (vf > 1.0f - 1e-7f) vf = 1.0f - 1e-7f;
  const float Df = D.hi, Bf = Bsq.hi, QBf = QdB2.hi, gff = k.gfac_hi;
  newton_wv<float>(Df, Qdn.hi, Qtsq.hi, Bf, QBf, gff, 10, 3e-6f, Wf, vf, ef);
  // an FP32 phase that stalled on FP32 rounding still hands over a close root
  if (!(Wf > 0.0f) || !kfinite(Wf) || !(vf >= 0.0f && vf < 1.0f - 1e-6f) || !(ef < 1e-2f)) return C2P_NEED_FP64;

  // refinement: double-float residuals, FP32 Jacobian at the current iterate;
  // done after a step below 1e-5 (at most three steps)
  df64 W = mkdf(Wf, 0.0f), vsq = mkdf(vf, 0.0f);
  bool done = false;
  for (int r = 0; r < 3 && !done; ++r) {
    const float wf = W.hi, vv = vsq.hi;
    const df64 x = 1.0f - vsq;
    const df64 sg = dfsqrt(x);
    const df64 iW = rcp(W);
    const df64 iW2 = iW * iW;
    const df64 BW = Bsq + W;
    const df64 p = gf * (W * x - D * sg);
    const df64 r1 = Qtsq - vsq * (BW * BW) + QdB2 * (Bsq + scale2(W, 2.0f)) * iW2;
    const df64 r2 = Qdn + W - p + scale2(Bsq * (1.0f + vsq), 0.5f) - scale2(QdB2 * iW2, 0.5f);
    const float xg = 1.0f - vv, BWf = Bf + wf, iWf = kdiv(1.0f, wf), iW3f = iWf * iWf * iWf;
    const float j11 = -2.0f * vv * BWf - 2.0f * QBf * BWf * iW3f;
    const float j12 = -BWf * BWf;
    const float j21 = 1.0f - gff * xg + QBf * iW3f;
    const float j22 = 0.5f * Bf - gff * (-wf + 0.5f * Df * krsqrt(xg));
    const float idet = kdiv(1.0f, j11 * j22 - j12 * j21);
    const float dW = (j22 * r1.hi - j12 * r2.hi) * idet;
    const float dv = (-j21 * r1.hi + j11 * r2.hi) * idet;
    const df64 Wn = W - dW;
    df64 vn = vsq - dv;
    if (vn.hi < 0.0f) vn = mkdf(0.0f, 0.0f);  // a fluid at rest in the normal frame: v^2 = 0 up to rounding
    if (!(Wn.hi > 0.0f && vn.hi < 1.0f - 1e-7f)) return C2P_NEED_FP64;
    done = fabsf(dW) * iWf + fabsf(dv) < 1e-5f;
    W = Wn;
    vsq = vn;
  }
  if (!done) return C2P_NEED_FP64;

  // primitives (scaled rho, u times S; u~ is scale free)
  const df64 x = 1.0f - vsq;
  const df64 sg = dfsqrt(x);  // 1 / Lorentz factor
  const df64 gamma = rcp(sg);
  const df64 rho = D * sg;
  const df64 uint = (W * x - rho) * mkdf(k.igam_hi, k.igam_lo);
  if (!(rho.hi > 0.0f)) return 4;
  if (!(uint.hi >= 0.0f)) return 5;
  P[V_RHO] = scale2(rho, S);
  P[V_U] = scale2(uint, S);
  const df64 BW = W + Bsq;
  const df64 inv = rcp(W * BW);
  const df64 f = gamma * W * inv;
  const df64 iWb = BW * inv;
#pragma unroll
  for (int i = 0; i < 3; ++i) P[V_U1 + i] = f * (Qt[i] + QdB * Bc[i] * iWb);
  return 0;
}

}  // namespace kh
