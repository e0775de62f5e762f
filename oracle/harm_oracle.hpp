// Plain FP64 CPU oracle of the HARM ideal-GRMHD finite-volume step.
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may include, link or
// call this code; only tests/, the smoke check and the CPU-baseline leg of the
// benchmark use it. It shares no code with the CUDA library.
//
// Everything here is written from the definitions, one formula at a time, with
// no blocking or fusion. Citations are to arXiv 2408.01361 (KHARMA) sections
// and to the published methods it names:
//   * ideal-MHD stress-energy tensor: "Extended GRMHD" section, the T^{mu nu}_ideal equation;
//   * HARM scheme (Gammie, McKinney & Toth 2003): "Algorithm" section;
//   * primitive 3-velocity relative to the normal observer (McKinney & Gammie 2004);
//   * 1D_w primitive recovery equations (Noble et al. 2006);
//   * Flux-CT (Toth 2000); MC limiter (van Leer 1977); WENO5 (Liu et al. 1994);
//   * LLF flux (Beckwith & Stone 2011 usage);
//   * funky MKS coordinates (Wong et al. 2022): "Requirements" section.
//
// Parity status of every function: see the oracle header comments below; each
// function is pinned by a CPU test in tests/test_oracle_*.py.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "dual.hpp"
#include "opcount.hpp"

namespace oracle {

// Primitive/conserved variable slots.
enum { RHO = 0, UU = 1, U1 = 2, U2 = 3, U3 = 4, B1 = 5, B2 = 6, B3 = 7, NVAR = 8 };
enum { MINKOWSKI = 0, KS = 1, MKS = 2, FMKS = 3 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_POLAR = 2, BC_DIRICHLET = 3 };
enum { RECON_MC = 0, RECON_WENO5 = 1, RECON_DONOR = 2 };
enum { LOC_CENT = 0, LOC_FACE1 = 1, LOC_FACE2 = 2, LOC_FACE3 = 3, LOC_CORN = 4 };

// Problem parameters (plain C layout, filled from Python through ctypes).
struct Params {
  int kind;            // MINKOWSKI | KS | MKS | FMKS
  int n1, n2, n3;      // interior zones; n3 == 1 means a 2-D (x1,x2) problem
  int ng;              // ghost zones in each active direction
  int recon;           // RECON_MC | RECON_WENO5 | RECON_DONOR (first order)
  int bc[6];           // x1 inner, x1 outer, x2 inner, x2 outer, x3 inner, x3 outer
  double a;            // black-hole spin (M = 1)
  double gam;          // adiabatic index of the ideal-gas EOS p = (gam-1) u
  double x1min, x1max, x2min, x2max, x3min, x3max;  // native coordinate box
  double hslope;       // MKS/FMKS theta concentration
  double poly_xt, poly_alpha, mks_smooth;           // FMKS parameters
  double cfl;
  double rho_min, u_min;          // geometric floor coefficients (r^-3/2, r^-5/2)
  double bsq_rho_max, bsq_u_max;  // magnetisation floors
  double u_rho_max;               // temperature ceiling u/rho
  double gamma_max;               // Lorentz-factor ceiling
  double x1ref;                   // FMKS blending reference: the x1 start of the whole domain
  int fofc;                       // first-order flux correction (see stage())
  int bfield;                     // BFIELD_FLUXCT | BFIELD_FACE (face-centred constrained transport)
  int emf;                        // face CT edge EMFs: EMF_AVERAGE | EMF_GS05 (contact-upwinded)
  int integrator;                 // INT_VL2 (predictor-corrector) | INT_RK1 | INT_RK2 | INT_SSPRK54
};

enum { INT_VL2 = 0, INT_RK1 = 1, INT_RK2 = 2, INT_SSPRK54 = 3 };

enum { BFIELD_FLUXCT = 0, BFIELD_FACE = 1 };
enum { EMF_AVERAGE = 0, EMF_GS05 = 1 };

// Geometry of one point.
struct Geo {
  double gcov[4][4];
  double gcon[4][4];
  double gdet;   // sqrt(-det g)
  double alpha;  // lapse, (-g^{00})^{-1/2}
};

// ---------------------------------------------------------------------------
// Coordinates and metric ("Requirements" section: MKS and funky MKS; the code
// structure section: GRCoordinates caches metric and connection).
// ---------------------------------------------------------------------------

// Map native (x1, x2) to Kerr-Schild (r, theta).
//   KS:   r = x1, theta = x2.
//   MKS:  r = exp(x1), theta = pi x2 + (1 - h)/2 sin(2 pi x2).
//   FMKS: r = exp(x1); theta_G = MKS theta; y = 2 x2 - 1;
//         theta_J = pi/2 + N y (1 + (y/x_t)^alpha / (alpha + 1)),  N such that
//         theta_J(x2=0) = 0 and theta_J(x2=1) = pi;
//         theta = theta_G + exp(s (x1ref - x1)) (theta_J - theta_G), x1ref the
//         x1 start of the whole domain,
//         continued past the poles by reflection (below).
template <class R>
void native_to_ks(const Params& c, const R& x1, const R& x2, R& r, R& th) {
  using std::exp; using std::sin; using std::pow;
  const double pi = M_PI;
  if (c.kind == KS) {
    r = x1;
    th = x2;
    return;
  }
  r = exp(x1);
  R thG = pi * x2 + (0.5 * (1.0 - c.hslope)) * sin((2.0 * pi) * x2);
  if (c.kind == MKS) {
    th = thG;
    return;
  }
  // Beyond the poles (ghost rows) the map is continued by reflection:
  // theta(x1, -x2) = -theta(x1, x2) and theta(x1, 2 - x2) = 2 pi - theta(x1, x2).
  // MKS satisfies this by itself; the FMKS polynomial does not.
  if (val(x2) < 0.0) {
    R rr, tt;
    native_to_ks<R>(c, x1, -x2, rr, tt);
    th = -tt;
    return;
  }
  if (val(x2) > 1.0) {
    R rr, tt;
    native_to_ks<R>(c, x1, 2.0 - x2, rr, tt);
    th = 2.0 * pi - tt;
    return;
  }
  R y = 2.0 * x2 - 1.0;
  double norm = 0.5 * pi / (1.0 + std::pow(c.poly_xt, -c.poly_alpha) / (c.poly_alpha + 1.0));
  R thJ = 0.5 * pi + norm * y * (1.0 + pow(y / c.poly_xt, c.poly_alpha) / (c.poly_alpha + 1.0));
  th = thG + exp(c.mks_smooth * (c.x1ref - x1)) * (thJ - thG);
}

// Kerr metric in spherical Kerr-Schild coordinates (t, r, theta, phi), M = 1.
// sin(theta) is kept away from exact zero (|sin| >= 1e-20) so that the metric
// at a face lying on the polar axis stays invertible; fluxes through such faces
// are zeroed by the polar boundary rule anyway.
template <class R>
void ks_gcov(double a, const R& r, const R& th, R g[4][4]) {
  using std::cos; using std::sin;
  R cth = cos(th);
  R sth = sin(th);
  if (std::fabs(val(sth)) < 1e-20) sth = R(1e-20);
  R s2 = sth * sth;
  R rho2 = r * r + (a * a) * (cth * cth);
  R z = 2.0 * r / rho2;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) g[m][n] = R(0.0);
  g[0][0] = z - 1.0;
  g[0][1] = z;
  g[1][0] = z;
  g[0][3] = -(a * z) * s2;
  g[3][0] = g[0][3];
  g[1][1] = 1.0 + z;
  g[1][3] = -(a * s2) * (1.0 + z);
  g[3][1] = g[1][3];
  g[2][2] = rho2;
  g[3][3] = s2 * (rho2 + (a * a) * s2 * (1.0 + z));
}

// Covariant metric in native coordinates: g'_{mn} = J^a_m J^b_n g_{ab}, with the
// Jacobian J^a_m = d x_KS^a / d x_native^m obtained by exact forward-mode
// differentiation of native_to_ks. Minkowski is Cartesian: diag(-1, 1, 1, 1).
template <class R>
void native_gcov(const Params& c, const R& x1, const R& x2, R g[4][4]) {
  if (c.kind == MINKOWSKI) {
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) g[m][n] = R(m == n ? (m == 0 ? -1.0 : 1.0) : 0.0);
    return;
  }
  Dual<R> ra, tha, rb, thb;
  native_to_ks<Dual<R>>(c, mk<R>(x1, R(1.0)), mk<R>(x2, R(0.0)), ra, tha);
  native_to_ks<Dual<R>>(c, mk<R>(x1, R(0.0)), mk<R>(x2, R(1.0)), rb, thb);
  R J[4][4];
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) J[m][n] = R(0.0);
  J[0][0] = R(1.0);
  J[3][3] = R(1.0);
  J[1][1] = ra.d;   // dr/dx1
  J[1][2] = rb.d;   // dr/dx2
  J[2][1] = tha.d;  // dtheta/dx1
  J[2][2] = thb.d;  // dtheta/dx2
  R gks[4][4];
  ks_gcov<R>(c.a, ra.v, tha.v, gks);
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) {
      R s(0.0);
      for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) s += J[p][m] * J[q][n] * gks[p][q];
      g[m][n] = s;
    }
}

// Inverse and determinant of a 4x4 matrix by Gauss-Jordan elimination with
// partial pivoting. Returns false for a singular matrix.
inline bool invert4(const double m[4][4], double inv[4][4], double* det) {
  double a[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 8; ++j) a[i][j] = (j < 4) ? m[i][j] : (j - 4 == i ? 1.0 : 0.0);
  double d = 1.0;
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
    if (a[piv][col] == 0.0) return false;
    if (piv != col) {
      for (int j = 0; j < 8; ++j) std::swap(a[piv][j], a[col][j]);
      d = -d;
    }
    double p = a[col][col];
    d *= p;
    for (int j = 0; j < 8; ++j) a[col][j] /= p;
    for (int r = 0; r < 4; ++r) {
      if (r == col) continue;
      double f = a[r][col];
      if (f == 0.0) continue;
      for (int j = 0; j < 8; ++j) a[r][j] -= f * a[col][j];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) inv[i][j] = a[i][j + 4];
  *det = d;
  return true;
}

// Complete a Geo from its covariant metric.
inline void geo_from_gcov(Geo& G) {
  double det = 0.0;
  invert4(G.gcov, G.gcon, &det);
  G.gdet = std::sqrt(std::fabs(det));
  G.alpha = 1.0 / std::sqrt(-G.gcon[0][0]);
}

// Native coordinates of a location in the (ghosted) grid. Cell i (0-based,
// ghosts included) has its centre at x1min + (i - ng + 1/2) dx1; the lower face
// of cell i is at x1min + (i - ng) dx1.
struct GridInfo {
  int n1, n2, n3, ng, ng3;
  int N1, N2, N3;
  int ndim;
  double dx1, dx2, dx3;
};

inline GridInfo grid_info(const Params& c) {
  GridInfo g;
  g.n1 = c.n1; g.n2 = c.n2; g.n3 = c.n3; g.ng = c.ng;
  g.ng3 = (c.n3 > 1) ? c.ng : 0;
  g.N1 = c.n1 + 2 * c.ng;
  g.N2 = c.n2 + 2 * c.ng;
  g.N3 = c.n3 + 2 * g.ng3;
  g.ndim = (c.n3 > 1) ? 3 : 2;
  g.dx1 = (c.x1max - c.x1min) / c.n1;
  g.dx2 = (c.x2max - c.x2min) / c.n2;
  g.dx3 = (c.x3max - c.x3min) / c.n3;
  return g;
}

inline void loc_coords(const Params& c, const GridInfo& g, int loc, int i, int j, double& x1, double& x2) {
  double o1 = (loc == LOC_FACE1 || loc == LOC_CORN) ? 0.0 : 0.5;
  double o2 = (loc == LOC_FACE2 || loc == LOC_CORN) ? 0.0 : 0.5;
  x1 = c.x1min + (i - g.ng + o1) * g.dx1;
  x2 = c.x2min + (j - g.ng + o2) * g.dx2;
}

inline Geo geo_at(const Params& c, double x1, double x2) {
  Geo G;
  native_gcov<double>(c, x1, x2, G.gcov);
  geo_from_gcov(G);
  return G;
}

// Connection coefficients Gamma^l_{mn} = 1/2 g^{lk} (d_m g_{kn} + d_n g_{km} - d_k g_{mn}),
// with d_0 = d_3 = 0 (stationary, axisymmetric) and d_1, d_2 taken exactly by
// forward-mode differentiation of the native metric.
inline void connection_at(const Params& c, double x1, double x2, double conn[4][4][4]) {
  double dg[4][4][4] = {};  // dg[k][m][n] = d_k g_{mn}
  if (c.kind != MINKOWSKI) {
    Dual<double> gd[4][4];
    native_gcov<Dual<double>>(c, mk<double>(x1, 1.0), mk<double>(x2, 0.0), gd);
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) dg[1][m][n] = gd[m][n].d;
    native_gcov<Dual<double>>(c, mk<double>(x1, 0.0), mk<double>(x2, 1.0), gd);
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) dg[2][m][n] = gd[m][n].d;
  }
  Geo G = geo_at(c, x1, x2);
  for (int l = 0; l < 4; ++l)
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) {
        double s = 0.0;
        for (int k = 0; k < 4; ++k) s += G.gcon[l][k] * (dg[m][k][n] + dg[n][k][m] - dg[k][m][n]);
        conn[l][m][n] = 0.5 * s;
      }
}

// ---------------------------------------------------------------------------
// Fluid state from primitives (McKinney & Gammie 2004 velocity; HARM b^mu).
// ---------------------------------------------------------------------------
template <class R> struct FluidState {
  R ucon[4], ucov[4], bcon[4], bcov[4], bsq;
};

// u^mu from the primitive velocity u~^i, defined relative to the normal
// observer n^mu = -alpha g^{mu 0}: u^mu = u~^mu + gamma n^mu with u~^0 = 0 and
// gamma = sqrt(1 + g_ij u~^i u~^j). The cell-centred field B^i = *F^{i t}
// gives b^t = B^i u_i and b^i = (B^i + b^t u^i) / u^t.
template <class R>
void fluid_state(const R P[NVAR], const Geo& G, FluidState<R>& S) {
  using std::sqrt;
  R qsq(0.0);
  for (int i = 1; i < 4; ++i)
    for (int j = 1; j < 4; ++j) qsq += G.gcov[i][j] * P[U1 + i - 1] * P[U1 + j - 1];
  R gamma = sqrt(1.0 + qsq);
  double n[4];
  for (int m = 0; m < 4; ++m) n[m] = -G.alpha * G.gcon[m][0];
  S.ucon[0] = gamma * n[0];
  for (int i = 1; i < 4; ++i) S.ucon[i] = P[U1 + i - 1] + gamma * n[i];
  for (int m = 0; m < 4; ++m) {
    R s(0.0);
    for (int k = 0; k < 4; ++k) s += G.gcov[m][k] * S.ucon[k];
    S.ucov[m] = s;
  }
  R bt(0.0);
  for (int i = 1; i < 4; ++i) bt += P[B1 + i - 1] * S.ucov[i];
  S.bcon[0] = bt;
  for (int i = 1; i < 4; ++i) S.bcon[i] = (P[B1 + i - 1] + bt * S.ucon[i]) / S.ucon[0];
  for (int m = 0; m < 4; ++m) {
    R s(0.0);
    for (int k = 0; k < 4; ++k) s += G.gcov[m][k] * S.bcon[k];
    S.bcov[m] = s;
  }
  R b2(0.0);
  for (int m = 0; m < 4; ++m) b2 += S.bcon[m] * S.bcov[m];
  S.bsq = b2;
}

// Mixed stress-energy tensor of ideal MHD ("Extended GRMHD" section):
// T^mu_nu = (rho + u + p + b^2) u^mu u_nu + (p + b^2/2) delta^mu_nu - b^mu b_nu.
template <class R, class Gm>
R t_mixed(const R P[NVAR], const FluidState<R>& S, const Gm& gam, int mu, int nu) {
  R p = (gam - 1.0) * P[UU];
  R w = P[RHO] + P[UU] + p;
  R out = (w + S.bsq) * S.ucon[mu] * S.ucov[nu] - S.bcon[mu] * S.bcov[nu];
  if (mu == nu) out += p + 0.5 * S.bsq;
  return out;
}

// Conserved variables (dir == 0) or the flux through an x^dir face (dir = 1..3):
//   sqrt(-g) (rho u^d, T^d_t + rho u^d, T^d_1, T^d_2, T^d_3, b^i u^d - b^d u^i).
// For dir == 0 the induction entry equals sqrt(-g) B^i by definition.
template <class R, class Gm>
void prim_to_flux(const R P[NVAR], const FluidState<R>& S, const Geo& G, const Gm& gam, int dir, R F[NVAR]) {
  R mflux = P[RHO] * S.ucon[dir];
  F[RHO] = G.gdet * mflux;
  F[UU] = G.gdet * (t_mixed(P, S, gam, dir, 0) + mflux);
  for (int i = 1; i < 4; ++i) F[U1 + i - 1] = G.gdet * t_mixed(P, S, gam, dir, i);
  for (int i = 1; i < 4; ++i) {
    if (dir == 0)
      F[B1 + i - 1] = G.gdet * P[B1 + i - 1];
    else
      F[B1 + i - 1] = G.gdet * (S.bcon[i] * S.ucon[dir] - S.bcon[dir] * S.ucon[i]);
  }
}

// Fast-magnetosonic signal speeds dx^dir/dt (Gammie et al. 2003): with the
// isotropic bound c_ms^2 = c_s^2 + v_A^2 - c_s^2 v_A^2, c_s^2 = gam p / w,
// v_A^2 = b^2 / (b^2 + w), a wave vector k_mu = delta_mu^dir - v delta_mu^t obeys
// (k.u)^2 = c_ms^2 (k.k + (k.u)^2), a quadratic in v. Its discriminant is
// clamped at zero; c_ms^2 is clamped to [0, 1].
template <class R, class Gm>
void signal_speeds(const R P[NVAR], const FluidState<R>& S, const Geo& G, const Gm& gam, int dir, R& cmax,
                   R& cmin) {
  using std::sqrt;
  R p = (gam - 1.0) * P[UU];
  R w = P[RHO] + P[UU] + p;
  R cs2 = gam * p / w;
  R va2 = S.bsq / (S.bsq + w);
  R cms2 = cs2 + va2 - cs2 * va2;
  if (cms2 < 0.0) cms2 = R(0.0);
  if (cms2 > 1.0) cms2 = R(1.0);
  // covariant wave vector k_mu = delta_mu^dir - v delta_mu^t contracted with u^mu
  R ku0 = S.ucon[dir];  // (k.u) at v = 0
  R ku1 = S.ucon[0];    // coefficient of -v in k.u
  double kk0 = G.gcon[dir][dir], kk1 = G.gcon[0][dir], kk2 = G.gcon[0][0];
  // (ku0 - v ku1)^2 - cms2 [ (kk0 - 2 v kk1 + v^2 kk2) + (ku0 - v ku1)^2 ] = 0
  R qa = ku1 * ku1 - cms2 * (kk2 + ku1 * ku1);
  R qb = -2.0 * (ku0 * ku1 - cms2 * (kk1 + ku0 * ku1));
  R qc = ku0 * ku0 - cms2 * (kk0 + ku0 * ku0);
  R disc = qb * qb - 4.0 * qa * qc;
  if (disc < 0.0) disc = R(0.0);
  R sq = sqrt(disc);
  R v1 = (-qb + sq) / (2.0 * qa);
  R v2 = (-qb - sq) / (2.0 * qa);
  if (v1 > v2) { cmax = v1; cmin = v2; } else { cmax = v2; cmin = v1; }
}

// Local Lax-Friedrichs flux through an x^dir face from left/right states:
// F = (F_L + F_R)/2 - c_top (U_R - U_L)/2, c_top = max(0, c+_L, c+_R, -c-_L, -c-_R).
template <class R, class Gm>
void llf_flux(const R PL[NVAR], const R PR[NVAR], const Geo& G, const Gm& gam, int dir, R F[NVAR], R& ctop) {
  FluidState<R> SL, SR;
  fluid_state(PL, G, SL);
  fluid_state(PR, G, SR);
  R FL[NVAR], FR[NVAR], UL[NVAR], UR[NVAR];
  prim_to_flux(PL, SL, G, gam, dir, FL);
  prim_to_flux(PR, SR, G, gam, dir, FR);
  prim_to_flux(PL, SL, G, gam, 0, UL);
  prim_to_flux(PR, SR, G, gam, 0, UR);
  R cmaxL, cminL, cmaxR, cminR;
  signal_speeds(PL, SL, G, gam, dir, cmaxL, cminL);
  signal_speeds(PR, SR, G, gam, dir, cmaxR, cminR);
  R c(0.0);
  if (cmaxL > c) c = cmaxL;
  if (cmaxR > c) c = cmaxR;
  if (-cminL > c) c = -cminL;
  if (-cminR > c) c = -cminR;
  ctop = c;
  for (int v = 0; v < NVAR; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * c * (UR[v] - UL[v]);
}

// Connection source terms for the energy and momentum equations:
// S_nu = sqrt(-g) T^k_l Gamma^l_{nu k}; zero for rho and B.
template <class R, class Gm>
void source_terms(const R P[NVAR], const Geo& G, const double conn[4][4][4], const Gm& gam, R S[NVAR]) {
  FluidState<R> st;
  fluid_state(P, G, st);
  R T[4][4];
  for (int k = 0; k < 4; ++k)
    for (int l = 0; l < 4; ++l) T[k][l] = t_mixed(P, st, gam, k, l);
  for (int v = 0; v < NVAR; ++v) S[v] = R(0.0);
  for (int nu = 0; nu < 4; ++nu) {
    R s(0.0);
    for (int k = 0; k < 4; ++k)
      for (int l = 0; l < 4; ++l) s += T[k][l] * conn[l][nu][k];
    S[UU + nu] = G.gdet * s;
  }
}

// ---------------------------------------------------------------------------
// Reconstruction ("Algorithm" section: linear/MC and WENO5).
// ---------------------------------------------------------------------------

// Monotonized-central slope: 0 if the one-sided differences disagree in sign
// (or one is zero), else the candidate of least magnitude among 2 d-, 2 d+ and
// (d- + d+)/2 (ties go to the earlier candidate).
template <class R>
R mc_slope(const R& qm, const R& q0, const R& qp) {
  using std::fabs;
  R dm = q0 - qm, dp = qp - q0;
  if (dm * dp <= 0.0) return R(0.0);
  R cand[3] = {2.0 * dm, 2.0 * dp, 0.5 * (dm + dp)};
  R s = cand[0];
  for (int i = 1; i < 3; ++i)
    if (fabs(cand[i]) < fabs(s)) s = cand[i];
  return s;
}

// WENO5 point value at the upper face of the centre cell of x[0..4]
// (Jiang-Shu smoothness indicators, power 2, eps = 1e-26; candidate stencils
// are the quadratic interpolants at x = +1/2, linear weights 1/16, 5/8, 5/16).
template <class R>
R weno5_upper(const R x[5]) {
  using std::pow;
  const double eps = 1e-26;
  R c[3];
  c[0] = (3.0 / 8.0) * x[0] - (5.0 / 4.0) * x[1] + (15.0 / 8.0) * x[2];
  c[1] = (-1.0 / 8.0) * x[1] + (3.0 / 4.0) * x[2] + (3.0 / 8.0) * x[3];
  c[2] = (3.0 / 8.0) * x[2] + (3.0 / 4.0) * x[3] - (1.0 / 8.0) * x[4];
  R b[3];
  b[0] = (13.0 / 12.0) * pow(x[0] - 2.0 * x[1] + x[2], 2.0) + 0.25 * pow(x[0] - 4.0 * x[1] + 3.0 * x[2], 2.0);
  b[1] = (13.0 / 12.0) * pow(x[1] - 2.0 * x[2] + x[3], 2.0) + 0.25 * pow(x[1] - x[3], 2.0);
  b[2] = (13.0 / 12.0) * pow(x[2] - 2.0 * x[3] + x[4], 2.0) + 0.25 * pow(3.0 * x[2] - 4.0 * x[3] + x[4], 2.0);
  const double d[3] = {1.0 / 16.0, 5.0 / 8.0, 5.0 / 16.0};
  R al[3], sum(0.0);
  for (int k = 0; k < 3; ++k) {
    al[k] = d[k] / pow(eps + b[k], 2.0);
    sum += al[k];
  }
  R out(0.0);
  for (int k = 0; k < 3; ++k) out += (al[k] / sum) * c[k];
  return out;
}

// Face values of the centre cell of stencil q[0..4] (q[2] is the cell):
// lo = value at its lower face, hi = value at its upper face.
template <class R>
void recon_cell(int recon, const R q[5], R& lo, R& hi) {
  if (recon == RECON_DONOR) {  // piecewise constant
    lo = q[2];
    hi = q[2];
  } else if (recon == RECON_MC) {
    R s = mc_slope(q[1], q[2], q[3]);
    lo = q[2] - 0.5 * s;
    hi = q[2] + 0.5 * s;
  } else {
    R rev[5] = {q[4], q[3], q[2], q[1], q[0]};
    hi = weno5_upper(q);
    lo = weno5_upper(rev);
  }
}

// ---------------------------------------------------------------------------
// Primitive recovery: Noble et al. (2006) equations in the single unknown W,
// solved by bracketing plus bisection to full double precision.
// ---------------------------------------------------------------------------
enum { C2P_OK = 0, C2P_NOCONV = 1, C2P_VSQ = 2, C2P_WNEG = 3, C2P_RHONEG = 4, C2P_UNEG = 5 };

struct C2PIn {
  double D, Qdotn, Qtsq, QdotB, Bsq;
  double Qt[4], Bcal[4];  // projected momentum Q~^mu, field B^mu = alpha B^i
};

// v^2 as a function of W from the momentum equation
// Q~^2 = v^2 (B^2 + W)^2 - (Q.B)^2 (B^2 + 2W) / W^2.
inline double vsq_of_W(const C2PIn& in, double W) {
  double num = in.Qtsq * W * W + in.QdotB * in.QdotB * (in.Bsq + 2.0 * W);
  double den = W * W * (in.Bsq + W) * (in.Bsq + W);
  return num / den;
}

// Energy residual Q.n + W - p(W, v^2) + B^2 (1 + v^2)/2 - (Q.B)^2 / (2 W^2),
// with the ideal-gas p = (gam-1)/gam (W (1 - v^2) - D sqrt(1 - v^2)).
inline double energy_residual(const C2PIn& in, double gam, double W) {
  double v2 = vsq_of_W(in, W);
  double g2inv = 1.0 - v2;
  double p = (gam - 1.0) / gam * (W * g2inv - in.D * std::sqrt(g2inv));
  return in.Qdotn + W - p + 0.5 * in.Bsq * (1.0 + v2) - in.QdotB * in.QdotB / (2.0 * W * W);
}

// Invert densitized conserved variables U at one point. P holds the guess on
// entry (used only to start the bracket search) and the result on exit (fluid
// part; B^i = U_B / sqrt(-g) always). Returns a C2P_* code.
inline int cons_to_prim_point(const double U[NVAR], const Geo& G, double gam, double P[NVAR]) {
  double u[NVAR];
  for (int v = 0; v < NVAR; ++v) u[v] = U[v] / G.gdet;
  for (int i = 0; i < 3; ++i) P[B1 + i] = u[B1 + i];
  double a = G.alpha;
  C2PIn in;
  in.D = a * u[RHO];
  double Qcov[4] = {a * (u[UU] - u[RHO]), a * u[U1], a * u[U2], a * u[U3]};
  double Qcon[4];
  for (int m = 0; m < 4; ++m) {
    Qcon[m] = 0.0;
    for (int k = 0; k < 4; ++k) Qcon[m] += G.gcon[m][k] * Qcov[k];
  }
  double ncov[4] = {-a, 0.0, 0.0, 0.0};
  double ncon[4];
  for (int m = 0; m < 4; ++m) ncon[m] = G.gcon[m][0] * ncov[0];
  double Qn = 0.0, Qsq = 0.0;
  for (int m = 0; m < 4; ++m) {
    Qn += Qcov[m] * ncon[m];
    Qsq += Qcov[m] * Qcon[m];
  }
  in.Qdotn = Qn;
  // Q~^2 is the square of a spacelike vector (>= 0 by definition); for a fluid
  // at rest in the normal frame rounding can leave it slightly negative.
  in.Qtsq = std::max(Qsq + Qn * Qn, 0.0);
  for (int m = 0; m < 4; ++m) in.Qt[m] = Qcon[m] + ncon[m] * Qn;
  in.Bcal[0] = 0.0;
  for (int i = 1; i < 4; ++i) in.Bcal[i] = a * u[B1 + i - 1];
  double Bcov[4];
  for (int m = 0; m < 4; ++m) {
    Bcov[m] = 0.0;
    for (int k = 0; k < 4; ++k) Bcov[m] += G.gcov[m][k] * in.Bcal[k];
  }
  in.Bsq = 0.0;
  in.QdotB = 0.0;
  for (int m = 0; m < 4; ++m) {
    in.Bsq += in.Bcal[m] * Bcov[m];
    in.QdotB += Qcov[m] * in.Bcal[m];
  }

  // Lower end of the admissible W range: v^2(W) is strictly decreasing, and the
  // root must have v^2 < 1. Find W_lo with v^2(W_lo) = 1 by bisection.
  double Wlo = 0.0;
  if (in.Qtsq > 0.0 || in.QdotB != 0.0) {
    double lo = 0.0, hi = 1.0;
    int guard = 0;
    while (vsq_of_W(in, hi) >= 1.0 && guard < 2000) { hi *= 2.0; ++guard; }
    for (int it = 0; it < 3000; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (vsq_of_W(in, mid) >= 1.0) lo = mid; else hi = mid;
    }
    Wlo = hi;  // smallest representable W found with v^2 < 1
  }

  // Starting value from the guess: W = (rho + u + p) gamma^2 at this metric.
  FluidState<double> S;
  fluid_state(P, G, S);
  double gam_guess = G.alpha * S.ucon[0];
  double W0 = (P[RHO] + gam * P[UU]) * gam_guess * gam_guess;
  if (!(W0 > Wlo) || !std::isfinite(W0)) W0 = (Wlo > 0.0) ? 2.0 * Wlo : 1.0;

  // Bracket a sign change of the energy residual: f -> +inf as W -> inf.
  double wa = W0, wb = W0;
  double fa = energy_residual(in, gam, wa);
  if (!std::isfinite(fa)) return C2P_NOCONV;
  if (fa < 0.0) {
    int k = 0;
    double fb = fa;
    while (fb < 0.0 && k < 2000) {
      wa = wb;
      wb *= 2.0;
      fb = energy_residual(in, gam, wb);
      ++k;
    }
    if (fb < 0.0) return C2P_NOCONV;
  } else {
    int k = 0;
    double fl = fa;
    while (fl >= 0.0 && k < 2000) {
      wb = wa;
      wa = Wlo + 0.5 * (wa - Wlo);
      if (wa <= Wlo) break;
      fl = energy_residual(in, gam, wa);
      ++k;
    }
    if (!(fl < 0.0)) return C2P_NOCONV;
  }
  // Bisection until the bracket cannot shrink further.
  for (int it = 0; it < 5000; ++it) {
    double mid = 0.5 * (wa + wb);
    if (mid <= wa || mid >= wb) break;
    if (energy_residual(in, gam, mid) < 0.0) wa = mid; else wb = mid;
  }
  double W = (std::fabs(energy_residual(in, gam, wa)) < std::fabs(energy_residual(in, gam, wb))) ? wa : wb;

  if (!(W > 0.0)) return C2P_WNEG;
  double v2 = vsq_of_W(in, W);
  if (!(v2 < 1.0) || v2 < 0.0) return C2P_VSQ;
  double gamma = 1.0 / std::sqrt(1.0 - v2);
  double rho = in.D / gamma;
  double w = W / (gamma * gamma);
  double uint = (w - rho) / gam;  // p = (gam-1)/gam (w - rho), u = p/(gam-1)
  if (!(rho > 0.0)) return C2P_RHONEG;
  if (!(uint >= 0.0)) return C2P_UNEG;
  P[RHO] = rho;
  P[UU] = uint;
  double fac = gamma / (W + in.Bsq);
  for (int i = 1; i < 4; ++i) P[U1 + i - 1] = fac * (in.Qt[i] + in.QdotB * in.Bcal[i] / W);
  return C2P_OK;
}

}  // namespace oracle
