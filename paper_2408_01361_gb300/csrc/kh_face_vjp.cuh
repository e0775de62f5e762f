// Gradient of one face side's contribution to the LLF objective of the
// adjoint step, by hand-written reverse-mode differentiation:
//   g(P, gam) = sum_v lam_v (F_v(P) / 2 + kappa U_v(P)) + lct * c(P),
// kappa = sgn ct / 2 (ct held fixed), c = cmax (active > 0), -cmin
// (active < 0) or 0 (active = 0), with F, U, the signal speeds and the fluid
// state exactly as fluid_state / flux_cons / signal_speeds compute them.
// g_out[0..7] = dg/dP, g_out[8] = dg/dgam. The forward sweep keeps its
// intermediates; the reverse sweep visits them in the opposite order.
// Branches: the clamps of c_ms^2 and of the discriminant pass no derivative,
// sqrt at 0 passes none, cmax/cmin follow the forward's comparison (as the
// dual-number version does).
#pragma once

#include "kh_dual.cuh"
#include "kh_physics.cuh"

namespace kh {

KH_HD void side_grad_rev(const double* P, const Met<double>& m, double gam, const double* lam, double kappa, int d,
                         int active, double lct, double* g_out) {
  // ---------------- forward ----------------
  const double rho = P[V_RHO], ui = P[V_U];
  const double v[4] = {0.0, P[V_U1], P[V_U2], P[V_U3]};
  const double Bv[4] = {0.0, P[V_B1], P[V_B2], P[V_B3]};
  double q = 0.0;
  for (int i = 1; i < 4; ++i)
    for (int j = 1; j < 4; ++j) q += m.gcov[i][j] * v[i] * v[j];
  const double opq = 1.0 + q;
  const double rg = krsqrt(opq);
  const double Gm = opq * rg;  // Lorentz factor
  const double al = m.alpha;
  const double ga = Gm * al;
  double u[4];
  u[0] = Gm / al;
  for (int i = 1; i < 4; ++i) u[i] = v[i] - ga * m.gcon[0][i];
  double uc[4];
  for (int mu = 0; mu < 4; ++mu) uc[mu] = m.gcov[mu][0] * u[0] + m.gcov[mu][1] * u[1] + m.gcov[mu][2] * u[2] + m.gcov[mu][3] * u[3];
  const double bt = Bv[1] * uc[1] + Bv[2] * uc[2] + Bv[3] * uc[3];
  const double iut = al * rg;
  double b[4];
  b[0] = bt;
  for (int i = 1; i < 4; ++i) b[i] = (Bv[i] + bt * u[i]) * iut;
  double bc[4];
  for (int mu = 0; mu < 4; ++mu) bc[mu] = m.gcov[mu][0] * b[0] + m.gcov[mu][1] * b[1] + m.gcov[mu][2] * b[2] + m.gcov[mu][3] * b[3];
  const double bsq = b[0] * bc[0] + b[1] * bc[1] + b[2] * bc[2] + b[3] * bc[3];
  const double pg = (gam - 1.0) * ui;
  const double eta = rho + ui + pg + bsq;
  const double g = m.gdet;
  const double ud = u[d], bd = b[d];

  // ---------------- reverse: fluxes and conserved vector ----------------
  double a_rho = 0.0, a_ui = 0.0, a_eta = 0.0, a_ptot = 0.0, a_bsq = 0.0, a_pg = 0.0, a_gam = 0.0;
  double a_u[4] = {0, 0, 0, 0}, a_uc[4] = {0, 0, 0, 0}, a_b[4] = {0, 0, 0, 0}, a_bc[4] = {0, 0, 0, 0};
  double a_B[4] = {0, 0, 0, 0};
  {
    // F_rho = g rho u^d ; U_rho = g rho u^0
    const double gF = 0.5 * lam[V_RHO] * g, gU = kappa * lam[V_RHO] * g;
    a_rho += gF * ud + gU * u[0];
    a_u[d] += gF * rho;
    a_u[0] += gU * rho;
  }
  {
    // F_u = g (eta u^d u_0 - b^d b_0 + rho u^d) ; U_u = g (eta u^0 u_0 - b^0 b_0 + ptot + rho u^0)
    const double gF = 0.5 * lam[V_U] * g, gU = kappa * lam[V_U] * g;
    a_eta += gF * ud * uc[0] + gU * u[0] * uc[0];
    a_u[d] += gF * (eta * uc[0] + rho);
    a_u[0] += gU * (eta * uc[0] + rho);
    a_uc[0] += gF * eta * ud + gU * eta * u[0];
    a_b[d] -= gF * bc[0];
    a_b[0] -= gU * bc[0];
    a_bc[0] -= gF * bd + gU * b[0];
    a_rho += gF * ud + gU * u[0];
    a_ptot += gU;
  }
  for (int i = 1; i < 4; ++i) {
    // F_i = g (eta u^d u_i - b^d b_i + delta_id ptot) ; U_i = g (eta u^0 u_i - b^0 b_i)
    const double gF = 0.5 * lam[V_U1 + i - 1] * g, gU = kappa * lam[V_U1 + i - 1] * g;
    a_eta += gF * ud * uc[i] + gU * u[0] * uc[i];
    a_u[d] += gF * eta * uc[i];
    a_u[0] += gU * eta * uc[i];
    a_uc[i] += gF * eta * ud + gU * eta * u[0];
    a_b[d] -= gF * bc[i];
    a_b[0] -= gU * bc[i];
    a_bc[i] -= gF * bd + gU * b[0];
    if (i == d) a_ptot += gF;
  }
  for (int i = 1; i < 4; ++i) {
    // F_Bi = g (b^i u^d - b^d u^i) ; U_Bi = g B^i
    const double gF = 0.5 * lam[V_B1 + i - 1] * g, gU = kappa * lam[V_B1 + i - 1] * g;
    a_b[i] += gF * ud;
    a_u[d] += gF * b[i];
    a_b[d] -= gF * u[i];
    a_u[i] -= gF * bd;
    a_B[i] += gU;
  }
  // ---------------- reverse: the active signal speed ----------------
  if (active != 0 && lct != 0.0) {
    const double w = rho + ui + pg;
    const double N = gam * pg + bsq, Dn = w + bsq;
    double cms2 = kdiv(N, Dn);
    const bool clamped = cms2 < 0.0 || cms2 > 1.0;
    cms2 = cms2 < 0.0 ? 0.0 : (cms2 > 1.0 ? 1.0 : cms2);
    const double Au = u[d], Bu = u[0];
    const double A = Bu * Bu - (m.gcon[0][0] + Bu * Bu) * cms2;
    const double Bq = 2.0 * (Au * Bu - (m.gcon[0][d] + Au * Bu) * cms2);
    const double C = Au * Au - (m.gcon[d][d] + Au * Au) * cms2;
    const double disc_raw = Bq * Bq - 4.0 * A * C;
    const double disc = disc_raw < 0.0 ? 0.0 : disc_raw;
    const double sd = sqrt(disc);
    const double i2a = kdiv(1.0, 2.0 * A);
    const double vp = (Bq + sd) * i2a, vm = (Bq - sd) * i2a;
    // which root: cmax = the larger, cmin = the smaller (as the forward compares)
    const bool p_is_max = vp > vm;
    const bool want_max = active > 0;
    const double s = (want_max == p_is_max) ? 1.0 : -1.0;  // r = (Bq + s sd) / (2A)
    const double r = (Bq + s * sd) * i2a;
    const double gr = lct * (want_max ? 1.0 : -1.0);  // c = cmax or -cmin
    double a_Bq = gr * i2a, a_sd = gr * s * i2a, a_A = -gr * r / A;
    const double a_disc = (disc_raw >= 0.0 && sd > 0.0) ? a_sd * 0.5 / sd : 0.0;
    a_Bq += a_disc * 2.0 * Bq;
    a_A += -4.0 * C * a_disc;
    const double a_C = -4.0 * A * a_disc;
    const double a_cms2 = -a_A * (m.gcon[0][0] + Bu * Bu) - a_Bq * 2.0 * (m.gcon[0][d] + Au * Bu) -
                          a_C * (m.gcon[d][d] + Au * Au);
    a_u[0] += a_A * 2.0 * Bu * (1.0 - cms2) + a_Bq * 2.0 * Au * (1.0 - cms2);
    a_u[d] += a_Bq * 2.0 * Bu * (1.0 - cms2) + a_C * 2.0 * Au * (1.0 - cms2);
    if (!clamped) {
      const double a_N = a_cms2 / Dn, a_Dn = -a_cms2 * cms2 / Dn;
      a_gam += a_N * pg;
      a_pg += a_N * gam + a_Dn;
      a_bsq += a_N + a_Dn;
      a_rho += a_Dn;
      a_ui += a_Dn;
    }
  }
  // ---------------- reverse: thermodynamics ----------------
  // eta = rho + u + pg + bsq ; ptot = pg + bsq / 2 ; pg = (gam - 1) u
  a_rho += a_eta;
  a_ui += a_eta;
  a_pg += a_eta + a_ptot;
  a_bsq += a_eta + 0.5 * a_ptot;
  a_ui += a_pg * (gam - 1.0);
  a_gam += a_pg * ui;
  // ---------------- reverse: the magnetic 4-vector ----------------
  // bsq = b^mu b_mu ; b_mu = g_{mu nu} b^nu
  for (int mu = 0; mu < 4; ++mu) {
    a_bc[mu] += a_bsq * b[mu];
    a_b[mu] += a_bsq * bc[mu];
  }
  for (int nu = 0; nu < 4; ++nu)
    a_b[nu] += m.gcov[0][nu] * a_bc[0] + m.gcov[1][nu] * a_bc[1] + m.gcov[2][nu] * a_bc[2] + m.gcov[3][nu] * a_bc[3];
  // b^i = (B^i + bt u^i) iut ; b^0 = bt ; iut = alpha rg ; bt = B^i u_i
  double a_bt = a_b[0], a_iut = 0.0;
  for (int i = 1; i < 4; ++i) {
    a_bt += a_b[i] * u[i] * iut;
    a_B[i] += a_b[i] * iut;
    a_u[i] += a_b[i] * bt * iut;
    a_iut += a_b[i] * (Bv[i] + bt * u[i]);
  }
  for (int i = 1; i < 4; ++i) {
    a_B[i] += a_bt * uc[i];
    a_uc[i] += a_bt * Bv[i];
  }
  double a_rg = a_iut * al;
  // ---------------- reverse: the velocity 4-vector ----------------
  for (int nu = 0; nu < 4; ++nu)
    a_u[nu] += m.gcov[0][nu] * a_uc[0] + m.gcov[1][nu] * a_uc[1] + m.gcov[2][nu] * a_uc[2] + m.gcov[3][nu] * a_uc[3];
  // u^i = v^i - ga g^{0i} ; u^0 = Gm / alpha ; ga = Gm alpha
  double a_v[4] = {0, 0, 0, 0}, a_ga = 0.0;
  for (int i = 1; i < 4; ++i) {
    a_v[i] += a_u[i];
    a_ga -= a_u[i] * m.gcon[0][i];
  }
  const double a_Gm = a_u[0] / al + a_ga * al;
  // Gm = opq rg ; rg = opq^{-1/2}
  double a_opq = a_Gm * rg;
  a_rg += a_Gm * opq;
  a_opq += a_rg * (-0.5 * rg / opq);
  // opq = 1 + v^T g v
  for (int i = 1; i < 4; ++i) {
    double gv = 0.0;
    for (int j = 1; j < 4; ++j) gv += m.gcov[i][j] * v[j];
    a_v[i] += 2.0 * a_opq * gv;
  }
  g_out[V_RHO] = a_rho;
  g_out[V_U] = a_ui;
  g_out[V_U1] = a_v[1];
  g_out[V_U2] = a_v[2];
  g_out[V_U3] = a_v[3];
  g_out[V_B1] = a_B[1];
  g_out[V_B2] = a_B[2];
  g_out[V_B3] = a_B[3];
  g_out[8] = a_gam;
}

// The same gradient by forward-mode dual numbers (9 tangents) over the
// templated forward physics: the reference the reverse sweep is checked
// against (kappa = sgn ct / 2 as above).
KH_HD void side_grad_dual(const double* Pside, const Met<double>& m, double gam, const double* lam, double kappa,
                          int D, int active, double lct, double* g) {
  Dn<9> Pd[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Pd[v] = Dn<9>::var(Pside[v], v);
  const Dn<9> gd = Dn<9>::var(gam, 8);
  FState<Dn<9>> s;
  fluid_state(Pd, m, s);
  Dn<9> F[NV], U[NV];
  flux_cons(Pd, s, m, gd, D, F, U);
  Dn<9> acc(0.0);
#pragma unroll
  for (int v = 0; v < NV; ++v) acc += lam[v] * (0.5 * F[v] + kappa * U[v]);
  if (active) {
    Dn<9> cmax, cmin;
    signal_speeds(Pd, s, m, gd, D, cmax, cmin);
    acc += lct * (active > 0 ? cmax : -cmin);
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) g[q] = acc.d[q];
}

}  // namespace kh
