// Per-point physics of the CUDA path (host+device), templated on the
// arithmetic type R so the same formulas serve the FP64 path.
//
// arXiv 2408.01361: the ideal-MHD stress-energy tensor
// T^{mu nu} = (rho + u + P + b^2) u^mu u^nu + (P + b^2/2) g^{mu nu} - b^mu b^nu
// ("Extended GRMHD" section); HARM's conserved variables, fluxes, signal
// speeds and the LLF flux ("Algorithm" section, Gammie et al. 2003); the
// normal-observer primitive velocity (McKinney & Gammie 2004); the Noble et
// al. (2006) two-unknown (W, v^2) Newton inversion; MC (van Leer 1977) and
// WENO5 (Liu et al. 1994) reconstruction; floors ("Algorithm" section).
#pragma once

#include "kh_geom_math.h"

namespace kh {

enum { V_RHO = 0, V_U = 1, V_U1 = 2, V_U2 = 3, V_U3 = 4, V_B1 = 5, V_B2 = 6, V_B3 = 7, NV = 8 };

// Symmetric-pair index of (m, n): 00 01 02 03 11 12 13 22 23 33.
KH_HD int sym_index(int m, int n) {
  if (m > n) { int t = m; m = n; n = t; }
  return m == 0 ? n : (m == 1 ? 3 + n : (m == 2 ? 5 + n : 9));
}

// 1/sqrt(x) (CUDA's rsqrt on the device; it gives sqrt(x) = x rsqrt(x) and its
// reciprocal from one operation).
KH_HD double krsqrt(double x) {
#ifdef __CUDA_ARCH__
  return rsqrt(x);
#else
  return 1.0 / sqrt(x);
#endif
}
KH_HD float krsqrt(float x) {
#ifdef __CUDA_ARCH__
  return rsqrtf(x);
#else
  return 1.0f / sqrtf(x);
#endif
}
// |x| and finiteness without promotion to FP64 for FP32 arguments (an FP64
// operation issues at 1/64 of the FP32 rate on GB300): x - x is 0 exactly
// when x is finite.
KH_HD float kabs(float x) { return fabsf(x); }
KH_HD double kabs(double x) { return fabs(x); }
KH_HD bool kfinite(float x) { return x - x == 0.0f; }
KH_HD bool kfinite(double x) { return isfinite(x); }
template <class R> KH_HD R kabs(const R& x) { return fabs(x); }  // other number types (duals)
// x clamped to [0, 1]; x clamped below at 0; the larger and smaller of a, b
// (a NaN passes through the clamps; other number types overload these)
template <class R> KH_HD R kclamp01(const R& x) { return x < R(0) ? R(0) : (x > R(1) ? R(1) : x); }
template <class R> KH_HD R kmax0(const R& x) { return x < R(0) ? R(0) : x; }
template <class R> KH_HD void kminmax(const R& a, const R& b, R& mx, R& mn) {
  mx = a > b ? a : b;
  mn = a > b ? b : a;
}
// a / b: IEEE division in FP64; in FP32 (the mixed path's stencil physics)
// CUDA's fast division, for divisors of modest magnitude (|b| < 2^126).
KH_HD double kdiv(double a, double b) { return a / b; }
KH_HD float kdiv(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}

// Metric at one point: full 4x4 covariant and contravariant, sqrt(-g), lapse.
template <class R> struct Met {
  R gcov[4][4];
  R gcon[4][4];
  R gdet;
  R alpha;
};

// Fluid 4-vectors at one point.
template <class R> struct FState {
  R ucon[4], ucov[4], bcon[4], bcov[4], bsq;
};

// u^t = gamma / alpha, u^i = u~^i - gamma alpha g^{ti}, gamma^2 = 1 + g_ij u~^i u~^j;
// b^t = B^i u_i, b^i = (B^i + b^t u^i) / u^t.
template <class R, class M> KH_HD void fluid_state(const R* P, const Met<M>& m, FState<R>& s) {
  const R v1 = P[V_U1], v2 = P[V_U2], v3 = P[V_U3];
  const R q = m.gcov[1][1] * v1 * v1 + m.gcov[2][2] * v2 * v2 + m.gcov[3][3] * v3 * v3 +
              R(2) * (m.gcov[1][2] * v1 * v2 + m.gcov[1][3] * v1 * v3 + m.gcov[2][3] * v2 * v3);
  const R opq = R(1) + q;
  const R rg = krsqrt(opq);  // 1 / gamma
  const R gam = opq * rg;
  const R ga = gam * m.alpha;
  s.ucon[0] = kdiv(gam, m.alpha);
  s.ucon[1] = v1 - ga * m.gcon[0][1];
  s.ucon[2] = v2 - ga * m.gcon[0][2];
  s.ucon[3] = v3 - ga * m.gcon[0][3];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
    s.ucov[mu] = m.gcov[mu][0] * s.ucon[0] + m.gcov[mu][1] * s.ucon[1] + m.gcov[mu][2] * s.ucon[2] +
                 m.gcov[mu][3] * s.ucon[3];
  const R bt = P[V_B1] * s.ucov[1] + P[V_B2] * s.ucov[2] + P[V_B3] * s.ucov[3];
  s.bcon[0] = bt;
  const R iut = m.alpha * rg;  // 1 / u^t
  s.bcon[1] = (P[V_B1] + bt * s.ucon[1]) * iut;
  s.bcon[2] = (P[V_B2] + bt * s.ucon[2]) * iut;
  s.bcon[3] = (P[V_B3] + bt * s.ucon[3]) * iut;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
    s.bcov[mu] = m.gcov[mu][0] * s.bcon[0] + m.gcov[mu][1] * s.bcon[1] + m.gcov[mu][2] * s.bcon[2] +
                 m.gcov[mu][3] * s.bcon[3];
  s.bsq = s.bcon[0] * s.bcov[0] + s.bcon[1] * s.bcov[1] + s.bcon[2] * s.bcov[2] + s.bcon[3] * s.bcov[3];
}

// Flux through an x^d face (d = 1..3) and the conserved vector of one state:
// F = sqrt(-g) (rho u^d, T^d_t + rho u^d, T^d_i, b^i u^d - b^d u^i),
// U = sqrt(-g) (rho u^t, T^t_t + rho u^t, T^t_i, B^i).
template <class R, class M>
KH_HD void flux_cons(const R* P, const FState<R>& s, const Met<M>& m, R gam, int d, R* F, R* U) {
  const R p = (gam - R(1)) * P[V_U];
  const R eta = P[V_RHO] + P[V_U] + p + s.bsq;
  const R ptot = p + R(0.5) * s.bsq;
  const R g = m.gdet;
  const R ud = s.ucon[d], bd = s.bcon[d];
  const R mf = P[V_RHO] * ud;
  F[V_RHO] = g * mf;
  F[V_U] = g * (eta * ud * s.ucov[0] - bd * s.bcov[0] + mf);
#pragma unroll
  for (int i = 1; i < 4; ++i) {
    R t = eta * ud * s.ucov[i] - bd * s.bcov[i];
    if (i == d) t += ptot;
    F[V_U1 + i - 1] = g * t;
    F[V_B1 + i - 1] = g * (s.bcon[i] * ud - bd * s.ucon[i]);
  }
  const R ut = s.ucon[0], bt = s.bcon[0];
  const R mt = P[V_RHO] * ut;
  U[V_RHO] = g * mt;
  U[V_U] = g * (eta * ut * s.ucov[0] - bt * s.bcov[0] + ptot + mt);
#pragma unroll
  for (int i = 1; i < 4; ++i) {
    U[V_U1 + i - 1] = g * (eta * ut * s.ucov[i] - bt * s.bcov[i]);
    U[V_B1 + i - 1] = g * P[V_B1 + i - 1];
  }
}

// Conserved vector only.
template <class R, class M> KH_HD void cons_only(const R* P, const FState<R>& s, const Met<M>& m, R gam, R* U) {
  const R p = (gam - R(1)) * P[V_U];
  const R eta = P[V_RHO] + P[V_U] + p + s.bsq;
  const R ptot = p + R(0.5) * s.bsq;
  const R g = m.gdet;
  const R ut = s.ucon[0], bt = s.bcon[0];
  const R mt = P[V_RHO] * ut;
  U[V_RHO] = g * mt;
  U[V_U] = g * (eta * ut * s.ucov[0] - bt * s.bcov[0] + ptot + mt);
#pragma unroll
  for (int i = 1; i < 4; ++i) {
    U[V_U1 + i - 1] = g * (eta * ut * s.ucov[i] - bt * s.bcov[i]);
    U[V_B1 + i - 1] = g * P[V_B1 + i - 1];
  }
}

// Signal speeds dx^d/dt: with the isotropic fast speed
// c_ms^2 = c_s^2 + v_A^2 - c_s^2 v_A^2 = (gam p + b^2) / (w + b^2)
// (c_s^2 = gam p / w, v_A^2 = b^2 / (w + b^2); clamped to [0, 1]) a covariant
// wave vector (-v, delta^d) obeys (k_mu u^mu)^2 = c_ms^2 (k_mu k^mu + (k_mu u^mu)^2),
// i.e. A v^2 - Bq v + C = 0.
template <class R, class M>
KH_HD void signal_speeds(const R* P, const FState<R>& s, const Met<M>& m, R gam, int d, R& cmax, R& cmin) {
  const R p = (gam - R(1)) * P[V_U];
  const R w = P[V_RHO] + P[V_U] + p;
  const R cms2 = kclamp01(R(kdiv(gam * p + s.bsq, w + s.bsq)));
  const R Au = s.ucon[d], Bu = s.ucon[0];
  const R A = Bu * Bu - (m.gcon[0][0] + Bu * Bu) * cms2;
  const R Bq = R(2) * (Au * Bu - (m.gcon[0][d] + Au * Bu) * cms2);
  const R C = Au * Au - (m.gcon[d][d] + Au * Au) * cms2;
  const R disc = kmax0(R(Bq * Bq - R(4) * A * C));
  const R sd = sqrt(disc);
  const R i2a = kdiv(R(1), R(2) * A);
  const R vp = (Bq + sd) * i2a;
  const R vm = (Bq - sd) * i2a;
  kminmax(vp, vm, cmax, cmin);
}

// ---------------------------------------------------------------------------
// Reconstruction of one variable.
// ---------------------------------------------------------------------------
// Monotonized central: zero slope unless both one-sided differences share a
// sign; otherwise the smallest-magnitude of 2 dL, 2 dR, (dL + dR)/2.
template <class R> KH_HD void recon_mc(R qm, R q0, R qp, R& lo, R& hi) {
  const R dl = q0 - qm, dr = qp - q0;
  R s = R(0);
  if (dl * dr > R(0)) {
    const R a = R(2) * dl, b = R(2) * dr, c = R(0.5) * (dl + dr);
    s = a;
    if (kabs(b) < kabs(s)) s = b;
    if (kabs(c) < kabs(s)) s = c;
  }
  lo = q0 - R(0.5) * s;
  hi = q0 + R(0.5) * s;
}

// WENO5 point value at x = +1/2 of the centre cell of (a, b, c, d, e):
// quadratic candidates at +1/2, linear weights (1/16, 5/8, 5/16), Jiang-Shu
// smoothness indicators, nonlinear weights d_k / (eps + beta_k)^2.
// FP64: eps = 1e-26 (absolute). The three weights share one division by
// multiplying each through by (s0 s1 s2)^2, s_k = eps + beta_k.
// (Templated for the adjoint's dual numbers; the double instance is the FP64
// path's.)
template <class R> KH_HD R weno5_plus_t(R a, R b, R c, R d, R e) {
  const R p0 = 0.375 * a - 1.25 * b + 1.875 * c;
  const R p1 = -0.125 * b + 0.75 * c + 0.375 * d;
  const R p2 = 0.375 * c + 0.75 * d - 0.125 * e;
  const double k = 13.0 / 12.0;
  const R t0 = a - 2.0 * b + c, u0 = a - 4.0 * b + 3.0 * c;
  const R t1 = b - 2.0 * c + d, u1 = b - d;
  const R t2 = c - 2.0 * d + e, u2 = 3.0 * c - 4.0 * d + e;
  const R s0 = k * t0 * t0 + 0.25 * u0 * u0 + 1e-26;
  const R s1 = k * t1 * t1 + 0.25 * u1 * u1 + 1e-26;
  const R s2 = k * t2 * t2 + 0.25 * u2 * u2 + 1e-26;
  const R q0 = s1 * s2, q1 = s0 * s2, q2 = s0 * s1;
  const R w0 = 0.0625 * q0 * q0, w1 = 0.625 * q1 * q1, w2 = 0.3125 * q2 * q2;
  return (w0 * p0 + w1 * p1 + w2 * p2) / (w0 + w1 + w2);
}
KH_HD double weno5_plus(double a, double b, double c, double d, double e) { return weno5_plus_t<double>(a, b, c, d, e); }

// FP32 (mixed path): the same weights, written scale-free so that nothing
// underflows in FP32: the indicators are normalised by their sum, eps = 1e-12
// relative to it, and each weight is d_k (s_min / s_k)^2 with s_min the
// smallest s_k (a common factor). A stencil whose indicator is many orders
// above the smoothest one gets a weight that vanishes, as it does in FP64.
KH_HD float weno5_plus(float a, float b, float c, float d, float e) {
  const float p0 = 0.375f * a - 1.25f * b + 1.875f * c;
  const float p1 = -0.125f * b + 0.75f * c + 0.375f * d;
  const float p2 = 0.375f * c + 0.75f * d - 0.125f * e;
  const float k = 13.0f / 12.0f;
  const float t0 = a - 2.0f * b + c, u0 = a - 4.0f * b + 3.0f * c;
  const float t1 = b - 2.0f * c + d, u1 = b - d;
  const float t2 = c - 2.0f * d + e, u2 = 3.0f * c - 4.0f * d + e;
  const float b0 = k * t0 * t0 + 0.25f * u0 * u0;
  const float b1 = k * t1 * t1 + 0.25f * u1 * u1;
  const float b2 = k * t2 * t2 + 0.25f * u2 * u2;
#ifdef __CUDA_ARCH__
  const float in = __frcp_rn(b0 + b1 + b2 + 1e-37f);  // any magnitude
#else
  const float in = 1.0f / (b0 + b1 + b2 + 1e-37f);
#endif
  const float s0 = b0 * in + 1e-12f, s1 = b1 * in + 1e-12f, s2 = b2 * in + 1e-12f;
  const float sm = fminf(s0, fminf(s1, s2));
  // s_k in [1e-12, 1 + 3e-12] and the weights' sum in [1/16, 1]: fast divisions
  const float r0 = kdiv(sm, s0), r1 = kdiv(sm, s1), r2 = kdiv(sm, s2);
  const float w0 = 0.0625f * r0 * r0, w1 = 0.625f * r1 * r1, w2 = 0.3125f * r2 * r2;
  return kdiv(w0 * p0 + w1 * p1 + w2 * p2, w0 + w1 + w2);
}

// ---------------------------------------------------------------------------
// Primitive recovery, FP64. Shared notation (Noble et al. 2006):
//   D = alpha rho u^t; Q_mu = alpha T^t_mu; B^mu = alpha (0, B^i);
//   n_mu = (-alpha, 0, 0, 0); Q~^mu = Q^mu + n^mu (Q.n);
//   W = (rho + u + p) gamma^2, v^2 = 1 - 1/gamma^2,
//   p = (gam - 1)/gam (W (1 - v^2) - D sqrt(1 - v^2)).
// The root satisfies
//   f1 = Q~^2 - v^2 (B^2 + W)^2 + (Q.B)^2 (B^2 + 2W) / W^2 = 0
//   f2 = Q.n + W - p(W, v^2) + B^2 (1 + v^2)/2 - (Q.B)^2 / (2 W^2) = 0.
// Three solvers find it (C2POpts::method): Noble's two-unknown Newton
// iteration on (W, v^2); Noble's one-unknown scheme on W (v^2 from f1 in
// closed form, Newton on f2, "1D_W"); and the scheme of Kastaun, Kalinani &
// Ciolfi (2021; the paper's "Algorithm" section) on mu = 1/(h gamma). Each
// returns 0 or a failure code (1 no convergence, 2 v^2 >= 1, 3 W <= 0,
// 4 rho <= 0, 5 u < 0); P (fluid slots) is written only on success.
// ---------------------------------------------------------------------------
enum { C2P_NOBLE2D = 0, C2P_1DW = 1, C2P_KASTAUN = 2 };

struct C2POpts {
  int max_iter;
  double tol;
  int method;  // C2P_NOBLE2D | C2P_1DW | C2P_KASTAUN
};

// The frame invariants of one zone's conserved variables.
struct C2PInv {
  double D, Qdn, Qtsq, Bsq, QdB, QdB2;
  double Qu[4], nu[4], Bc[3];
};

KH_HD void c2p_invariants(const double* U, const Met<double>& m, double ig, C2PInv& I) {
  const double a = m.alpha;
  I.D = a * U[V_RHO] * ig;
  const double Qc[4] = {a * (U[V_U] - U[V_RHO]) * ig, a * U[V_U1] * ig, a * U[V_U2] * ig, a * U[V_U3] * ig};
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
    I.Qu[mu] = m.gcon[mu][0] * Qc[0] + m.gcon[mu][1] * Qc[1] + m.gcon[mu][2] * Qc[2] + m.gcon[mu][3] * Qc[3];
  // n^mu = -alpha g^{mu t}
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) I.nu[mu] = -a * m.gcon[mu][0];
  I.Qdn = Qc[0] * I.nu[0] + Qc[1] * I.nu[1] + Qc[2] * I.nu[2] + Qc[3] * I.nu[3];
  const double Qsq = Qc[0] * I.Qu[0] + Qc[1] * I.Qu[1] + Qc[2] * I.Qu[2] + Qc[3] * I.Qu[3];
  // square of the spacelike projected momentum: >= 0 (rounding can make the
  // difference slightly negative for a fluid at rest in the normal frame)
  I.Qtsq = fmax(Qsq + I.Qdn * I.Qdn, 0.0);
  I.Bc[0] = a * U[V_B1] * ig;
  I.Bc[1] = a * U[V_B2] * ig;
  I.Bc[2] = a * U[V_B3] * ig;
  const double Bc1 = I.Bc[0], Bc2 = I.Bc[1], Bc3 = I.Bc[2];
  I.Bsq = m.gcov[1][1] * Bc1 * Bc1 + m.gcov[2][2] * Bc2 * Bc2 + m.gcov[3][3] * Bc3 * Bc3 +
          2.0 * (m.gcov[1][2] * Bc1 * Bc2 + m.gcov[1][3] * Bc1 * Bc3 + m.gcov[2][3] * Bc2 * Bc3);
  I.QdB = Qc[1] * Bc1 + Qc[2] * Bc2 + Qc[3] * Bc3;
  I.QdB2 = I.QdB * I.QdB;
}

// Primitives from a root (W, v^2): rho = D / gamma, u = (W (1 - v^2) - rho) / gam,
// u~^i = gamma (Q~^i + (Q.B) B^i / W) / (W + B^2).
KH_HD int c2p_output(const C2PInv& I, double W, double vsq, double igam, double* P) {
  if (!(W > 0.0)) return 3;
  if (!(vsq < 1.0) || vsq < 0.0) return 2;
  const double gamma = krsqrt(1.0 - vsq);
  const double rho = I.D * ((1.0 - vsq) * gamma);
  const double uint = (W * (1.0 - vsq) - rho) * igam;
  if (!(rho > 0.0)) return 4;
  if (!(uint >= 0.0)) return 5;
  P[V_RHO] = rho;
  P[V_U] = uint;
  const double BW = W + I.Bsq;
  const double inv = 1.0 / (W * BW);  // one division for 1/W and gamma/(W + B^2)
  const double f = gamma * W * inv;
  const double iW = BW * inv;
  P[V_U1] = f * (I.Qu[1] + I.nu[1] * I.Qdn + I.QdB * I.Bc[0] * iW);
  P[V_U2] = f * (I.Qu[2] + I.nu[2] * I.Qdn + I.QdB * I.Bc[1] * iW);
  P[V_U3] = f * (I.Qu[3] + I.nu[3] * I.Qdn + I.QdB * I.Bc[2] * iW);
  return 0;
}

// Initial guess (W, v^2) from the primitives in P at this metric.
KH_HD void c2p_guess(const double* P, const Met<double>& m, double gam, const C2PInv& I, double& W, double& vsq) {
  const double v1 = P[V_U1], v2 = P[V_U2], v3 = P[V_U3];
  const double q = m.gcov[1][1] * v1 * v1 + m.gcov[2][2] * v2 * v2 + m.gcov[3][3] * v3 * v3 +
                   2.0 * (m.gcov[1][2] * v1 * v2 + m.gcov[1][3] * v1 * v3 + m.gcov[2][3] * v2 * v3);
  const double g2 = 1.0 + q;
  W = (P[V_RHO] + gam * P[V_U]) * g2;
  vsq = q / g2;
  if (!(W > 0.0) || !isfinite(W)) W = fabs(I.Qdn) + 1e-300;
  const double vmax = 1.0 - 1e-16;
  if (!(vsq >= 0.0)) vsq = 0.0;
  if (vsq > vmax) vsq = vmax;
}

// Noble's two-unknown Newton iteration on (W, v^2).
KH_HD int noble2d(const double* U, const Met<double>& m, double ig, double gam, double igam, double gf,
                  const C2POpts& o, double* P) {
  C2PInv I;
  c2p_invariants(U, m, ig, I);
  const double D = I.D, Qdn = I.Qdn, Qtsq = I.Qtsq, Bsq = I.Bsq, QdB2 = I.QdB2;
  // initial guess from the stage-input primitives at this metric
  double W, vsq;
  c2p_guess(P, m, gam, I, W, vsq);
  const double vmax = 1.0 - 1e-16;

  bool conv = false;
  double err = 1.0;
  for (int it = 0; it < o.max_iter; ++it) {
    const double g2i = 1.0 - vsq;
    const double rs = krsqrt(g2i);  // gamma
    const double sg = g2i * rs;     // 1 / gamma
    const double p = gf * (W * g2i - D * sg);
    const double BW = Bsq + W;
    const double iW = 1.0 / W;
    const double iW2 = iW * iW, iW3 = iW2 * iW;
    const double f1 = Qtsq - vsq * BW * BW + QdB2 * (Bsq + 2.0 * W) * iW2;
    const double f2 = Qdn + W - p + 0.5 * Bsq * (1.0 + vsq) - 0.5 * QdB2 * iW2;
    const double dpdW = gf * g2i;
    const double dpdv = gf * (-W + 0.5 * D * rs);
    const double j11 = -2.0 * vsq * BW - 2.0 * QdB2 * BW * iW3;
    const double j12 = -BW * BW;
    const double j21 = 1.0 - dpdW + QdB2 * iW3;
    const double j22 = 0.5 * Bsq - dpdv;
    const double idet = 1.0 / (j11 * j22 - j12 * j21);
    const double dW = -(j22 * f1 - j12 * f2) * idet;
    const double dv = -(-j21 * f1 + j11 * f2) * idet;
    double Wn = W + dW;
    double vn = vsq + dv;
    // keep the iterate admissible
    if (!(Wn > 0.0)) Wn = 0.5 * W;
    if (vn < 0.0) vn = 0.0;
    if (vn > vmax) vn = vmax;
    err = fabs(Wn - W) * iW + fabs(vn - vsq);  // step relative to the previous iterate
    W = Wn;
    vsq = vn;
    if (!isfinite(W) || !isfinite(vsq)) return 1;
    if (err < o.tol) {
      conv = true;
      break;
    }
  }
  if (!conv && !(err < 1e-9)) return 1;
  return c2p_output(I, W, vsq, igam, P);
}

// v^2(W) from f1 in closed form, with its W derivative.
KH_HD void vsq_of_W(const C2PInv& I, double W, double& vsq, double& dvsq) {
  const double BW = I.Bsq + W;
  const double N = I.Qtsq * W * W + I.QdB2 * (I.Bsq + 2.0 * W);
  const double Dn = W * W * BW * BW;
  const double dN = 2.0 * (I.Qtsq * W + I.QdB2);
  const double dDn = 2.0 * W * BW * (I.Bsq + 2.0 * W);
  vsq = N / Dn;
  dvsq = (dN * Dn - N * dDn) / (Dn * Dn);
}

// Noble's one-unknown scheme ("1D_W"): Newton on f2(W, v^2(W)); a step that
// leaves W > 0 or v^2 < 1 is halved back towards the iterate.
KH_HD int noble1dw(const double* U, const Met<double>& m, double ig, double gam, double igam, double gf,
                   const C2POpts& o, double* P) {
  C2PInv I;
  c2p_invariants(U, m, ig, I);
  double W, vsq;
  c2p_guess(P, m, gam, I, W, vsq);
  const double vmax = 1.0 - 1e-16;
  double dv;
  vsq_of_W(I, W, vsq, dv);
  // start where v^2(W) < 1 (v^2 decreases towards 0 as W grows)
  for (int g = 0; g < 200 && !(vsq < vmax); ++g) {
    W *= 2.0;
    vsq_of_W(I, W, vsq, dv);
  }
  if (!(vsq < vmax)) return 2;
  bool conv = false;
  double err = 1.0;
  for (int it = 0; it < o.max_iter; ++it) {
    vsq_of_W(I, W, vsq, dv);
    const double g2i = 1.0 - vsq;
    const double rs = krsqrt(g2i);
    const double sg = g2i * rs;
    const double p = gf * (W * g2i - I.D * sg);
    const double iW = 1.0 / W;
    const double iW2 = iW * iW;
    const double f = I.Qdn + W - p + 0.5 * I.Bsq * (1.0 + vsq) - 0.5 * I.QdB2 * iW2;
    const double dpdW = gf * g2i;
    const double dpdv = gf * (-W + 0.5 * I.D * rs);
    const double df = 1.0 - dpdW - dpdv * dv + 0.5 * I.Bsq * dv + I.QdB2 * iW2 * iW;
    double dW = -f / df;
    if (!isfinite(dW)) return 1;
    double Wn = W + dW;
    double vn = 0.0, dn;
    for (int h = 0; h < 60; ++h) {  // keep the iterate admissible
      if (Wn > 0.0) {
        vsq_of_W(I, Wn, vn, dn);
        if (vn < vmax) break;
      }
      dW *= 0.5;
      Wn = W + dW;
    }
    err = fabs(Wn - W) * iW;
    W = Wn;
    if (!(W > 0.0) || !isfinite(W)) return 1;
    if (err < o.tol) {
      conv = true;
      break;
    }
  }
  if (!conv && !(err < 1e-9)) return 1;
  vsq_of_W(I, W, vsq, dv);
  return c2p_output(I, W, vsq, igam, P);
}

// Kastaun, Kalinani & Ciolfi (2021): one unknown mu = 1/(h gamma), in the
// variables scaled by D: q = tau/D (tau = -Q.n - D), r^2 = Q~^2/D^2,
// b^2 = B^2/D, (r.b) = Q.B/D^(3/2). For a trial mu, with x = 1/(1 + mu b^2):
//   rbar^2 = x^2 r^2 + mu x (1 + x) (r.b)^2            (v^2 = mu^2 rbar^2)
//   qbar   = q - b^2/2 - mu^2 x^2 (b^2 r^2 - (r.b)^2)/2
//   v^2 <= r^2 / (h0^2 + r^2) (h0 = 1, the least enthalpy of an ideal gas),
//   gamma, rho = D/gamma, eps = gamma (qbar - mu rbar^2) + v^2 gamma^2/(1 + gamma)
//   (clamped to eps >= 0), a = p/(rho (1 + eps)),
//   nu = max((1 + a)(1 + eps)/gamma, (1 + a)(1 + qbar - mu rbar^2)),
// and the root of f(mu) = mu - 1/(nu + mu rbar^2) in (0, mu+] is the
// solution; mu+ = 1/h0, or for r^2 >= h0^2 the root of
// mu sqrt(h0^2 + rbar^2(mu)) - 1. The root gives W = D/mu and v^2.
struct KastaunVars {
  double q, r2, b2, rb2, brr;  // brr = b^2 r^2 - (r.b)^2 >= 0
};

KH_HD double kastaun_f(const KastaunVars& k, double mu, double gm1, double* vsq_out) {
  const double x = 1.0 / (1.0 + mu * k.b2);
  const double rbar2 = x * x * k.r2 + mu * x * (1.0 + x) * k.rb2;
  const double qbar = k.q - 0.5 * k.b2 - 0.5 * mu * mu * x * x * k.brr;
  const double v0sq = k.r2 / (1.0 + k.r2);
  double vsq = mu * mu * rbar2;
  if (vsq > v0sq) vsq = v0sq;
  const double W = krsqrt(1.0 - vsq);
  double eps = W * (qbar - mu * rbar2) + vsq * W * W / (1.0 + W);
  if (eps < 0.0) eps = 0.0;
  const double a = gm1 * eps / (1.0 + eps);  // p / (rho (1 + eps)) of an ideal gas
  const double nuA = (1.0 + a) * (1.0 + eps) / W;
  const double nuB = (1.0 + a) * (1.0 + qbar - mu * rbar2);
  const double nu = nuA > nuB ? nuA : nuB;
  if (vsq_out) *vsq_out = vsq;
  return mu - 1.0 / (nu + mu * rbar2);
}

KH_HD int kastaun(const double* U, const Met<double>& m, double ig, double gam, double igam, const C2POpts& o,
                  double* P) {
  C2PInv I;
  c2p_invariants(U, m, ig, I);
  if (!(I.D > 0.0)) return 4;
  const double iD = 1.0 / I.D;
  KastaunVars k;
  k.q = -I.Qdn * iD - 1.0;
  k.r2 = I.Qtsq * iD * iD;
  k.b2 = I.Bsq * iD;
  k.rb2 = I.QdB2 * iD * iD * iD;
  k.brr = k.b2 * k.r2 - k.rb2;
  if (k.brr < 0.0) k.brr = 0.0;
  const double gm1 = gam - 1.0;
  // upper end of the bracket
  double mup = 1.0;
  if (k.r2 >= 1.0) {
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 80 && hi - lo > 1e-15 * hi; ++it) {
      const double mu = 0.5 * (lo + hi);
      const double x = 1.0 / (1.0 + mu * k.b2);
      const double rbar2 = x * x * k.r2 + mu * x * (1.0 + x) * k.rb2;
      if (mu * sqrt(1.0 + rbar2) - 1.0 < 0.0) lo = mu; else hi = mu;
    }
    mup = hi;
  }
  // Illinois (modified regula falsi) on f over [0, mu+]
  double a = 0.0, b = mup;
  double fa = kastaun_f(k, a, gm1, nullptr), fb = kastaun_f(k, b, gm1, nullptr);
  if (!(fa <= 0.0 && fb >= 0.0)) return 1;  // no bracket (an unphysical state)
  int side = 0;
  double mu = b;
  bool conv = fb == 0.0;
  const int nmax = 4 * o.max_iter;
  for (int it = 0; it < nmax && !conv; ++it) {
    mu = (a * fb - b * fa) / (fb - fa);
    if (!(mu > a && mu < b)) mu = 0.5 * (a + b);
    const double fm = kastaun_f(k, mu, gm1, nullptr);
    if (fm == 0.0) {
      conv = true;
      break;
    }
    if (fm > 0.0) {
      b = mu;
      fb = fm;
      if (side == 1) fa *= 0.5;
      side = 1;
    } else {
      a = mu;
      fa = fm;
      if (side == -1) fb *= 0.5;
      side = -1;
    }
    if (b - a < o.tol * b) {
      mu = 0.5 * (a + b);
      conv = true;
    }
  }
  if (!conv) return 1;
  double vsq;
  kastaun_f(k, mu, gm1, &vsq);
  return c2p_output(I, I.D / mu, vsq, igam, P);
}

// The solver INV (a compile-time choice: each kernel instance carries one
// solver, so the default keeps the update kernels' register budget).
template <int INV>
KH_HD int invert(const double* U, const Met<double>& m, double ig, double gam, double igam, double gf,
                 const C2POpts& o, double* P) {
  if constexpr (INV == C2P_1DW) return noble1dw(U, m, ig, gam, igam, gf, o, P);
  else if constexpr (INV == C2P_KASTAUN) return kastaun(U, m, ig, gam, igam, o, P);
  else return noble2d(U, m, ig, gam, igam, gf, o, P);
}

// ---------------------------------------------------------------------------
// Floors (after a successful inversion or a fixup):
//   rho >= max(rho_min r^-3/2, 1e-20, b^2/bsq_rho_max)
//   u   >= max(u_min r^-5/2, 1e-20, b^2/bsq_u_max)
//   u   <= u_rho_max rho
//   gamma <= gamma_max (u~ scaled down)
// Mass and energy are injected by raising rho and u at fixed u~ (normal-
// observer frame); the caller recomputes U where the mask is non-zero.
// ---------------------------------------------------------------------------
struct FloorParams {
  double rho_min, u_min, bsq_rho_max, bsq_u_max, u_rho_max, gamma_max;
  double ibsq_rho_max, ibsq_u_max;  // 1 / bsq_rho_max, 1 / bsq_u_max (set with them)
};

// rho_geo, u_geo: the geometric floors max(rho_min r^-3/2, 1e-20) and
// max(u_min r^-5/2, 1e-20) of the zone (cached per (i, j)); bsq: b^2 of P.
KH_HD int apply_floors(const FloorParams& f, const Met<double>& m, double rho_geo, double u_geo, double bsq,
                       double* P) {
  double rf = rho_geo, uf = u_geo;
  const double rb = bsq * f.ibsq_rho_max, ub = bsq * f.ibsq_u_max;
  rf = rf > rb ? rf : rb;
  uf = uf > ub ? uf : ub;
  int mask = 0;
  if (P[V_RHO] < rf) { P[V_RHO] = rf; mask |= 1; }
  if (P[V_U] < uf) { P[V_U] = uf; mask |= 1; }
  if (P[V_U] > f.u_rho_max * P[V_RHO]) { P[V_U] = f.u_rho_max * P[V_RHO]; mask |= 2; }
  // gamma^2 = 1 + q: compare squares, take a root only for the rare zone over the ceiling
  const double g2max = f.gamma_max * f.gamma_max;
  auto qexact = [&]() {
    const double v1 = P[V_U1], v2 = P[V_U2], v3 = P[V_U3];
    return m.gcov[1][1] * v1 * v1 + m.gcov[2][2] * v2 * v2 + m.gcov[3][3] * v3 * v3 +
           2.0 * (m.gcov[1][2] * v1 * v2 + m.gcov[1][3] * v1 * v3 + m.gcov[2][3] * v2 * v3);
  };
  const double q = qexact();
  if (1.0 + q > g2max) {
    const double sc = sqrt((g2max - 1.0) / q);
    P[V_U1] *= sc;
    P[V_U2] *= sc;
    P[V_U3] *= sc;
    mask |= 4;
  }
  return mask;
}

// ---------------------------------------------------------------------------
// Newton's iterations on the (W, v^2) equations of noble2d in precision R
// (the FP32 phase of the mixed update's inversion, on the problem scaled to
// order unity): stops when a step changes |dW/W| + |dv^2| by less than stop.
// ---------------------------------------------------------------------------
template <class R>
KH_HD bool newton_wv(R D, R Qdn, R Qtsq, R Bsq, R QdB2, R gf, int max_iter, R stop, R& W, R& vsq, R& err) {
  const R vmax = R(1) - R(sizeof(R) == 4 ? 1e-7 : 1e-16);
  for (int it = 0; it < max_iter; ++it) {
    const R g2i = R(1) - vsq;
    const R rs = krsqrt(g2i);  // gamma
    const R sg = g2i * rs;     // 1 / gamma
    const R p = gf * (W * g2i - D * sg);
    const R BW = Bsq + W;
    const R iW = kdiv(R(1), W);
    const R iW2 = iW * iW;
    const R f1 = Qtsq - vsq * BW * BW + QdB2 * (Bsq + R(2) * W) * iW2;
    const R f2 = Qdn + W - p + R(0.5) * Bsq * (R(1) + vsq) - R(0.5) * QdB2 * iW2;
    const R dpdW = gf * g2i;
    const R dpdv = gf * (-W + R(0.5) * D * rs);
    const R j11 = -R(2) * vsq * BW - R(2) * QdB2 * BW * iW2 * iW;
    const R j12 = -BW * BW;
    const R j21 = R(1) - dpdW + QdB2 * iW2 * iW;
    const R j22 = R(0.5) * Bsq - dpdv;
    const R idet = kdiv(R(1), j11 * j22 - j12 * j21);
    R Wn = W - (j22 * f1 - j12 * f2) * idet;
    R vn = vsq - (-j21 * f1 + j11 * f2) * idet;
    if (!(Wn > R(0))) Wn = R(0.5) * W;
    if (vn < R(0)) vn = R(0);
    if (vn > vmax) vn = vmax;
    err = kabs(Wn - W) * iW + kabs(vn - vsq);  // step relative to the previous iterate
    W = Wn;
    vsq = vn;
    if (!kfinite(W) || !kfinite(vsq)) return false;
    if (err < stop) return true;
  }
  return false;
}

}  // namespace kh
