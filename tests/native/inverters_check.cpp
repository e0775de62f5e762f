// Host check of the three FP64 primitive-recovery solvers of the update
// (Noble et al.'s two-unknown Newton iteration, their one-unknown 1D_W
// scheme, and Kastaun, Kalinani & Ciolfi's bracketed scheme) on seeded
// magnetised states in Minkowski and in the funky-MKS Kerr metric (points
// from the oracle). Set A: sigma up to 50, |u~| from 3e-5 to 3, guesses 1e-3
// off. Set B (stress): sigma up to 1e4, |u~| up to 50, the guess an
// unrelated state. Prints per solver: the largest relative error against
// the state on set A, its failures on set A and on set B, the largest
// relative error of its successes on set B; then the sizes of the two sets.
#include <cmath>
#include <cstdio>
#include <random>

#include "kh_physics.cuh"

extern "C" {
struct orp {
  int kind, n1, n2, n3, ng, recon, bc[6];
  double a, gam, x1min, x1max, x2min, x2max, x3min, x3max, hslope, poly_xt, poly_alpha, mks_smooth, cfl, rho_min,
      u_min, bsq_rho_max, bsq_u_max, u_rho_max, gamma_max, x1ref;
  int fofc, bfield, emf, integrator;
};
void or_metric_points(const orp*, int, const double*, const double*, double*, double*, double*, double*);
}

using namespace kh;

static void metric(std::mt19937_64& rng, const orp& p, int t, Met<double>& m) {
  std::uniform_real_distribution<double> U01(0.0, 1.0);
  if (t % 4 == 0) {
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) m.gcov[a][b] = m.gcon[a][b] = (a == b) ? (a == 0 ? -1.0 : 1.0) : 0.0;
    m.gdet = 1.0;
    m.alpha = 1.0;
    return;
  }
  const double x1 = 0.3 + 6.0 * U01(rng), x2 = 0.02 + 0.96 * U01(rng);
  double go[16], gc[16], gd, cn[64];
  or_metric_points(&p, 1, &x1, &x2, go, gc, &gd, cn);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      m.gcov[a][b] = go[a * 4 + b];
      m.gcon[a][b] = gc[a * 4 + b];
    }
  m.gdet = gd;
  m.alpha = 1.0 / std::sqrt(-m.gcon[0][0]);
}

static int solve(int method, const double* U, const Met<double>& m, double gam, double* P) {
  C2POpts o{30, 1e-14, method};
  const double ig = 1.0 / m.gdet;
  if (method == C2P_1DW) return invert<C2P_1DW>(U, m, ig, gam, 1.0 / gam, (gam - 1.0) / gam, o, P);
  if (method == C2P_KASTAUN) return invert<C2P_KASTAUN>(U, m, ig, gam, 1.0 / gam, (gam - 1.0) / gam, o, P);
  return invert<C2P_NOBLE2D>(U, m, ig, gam, 1.0 / gam, (gam - 1.0) / gam, o, P);
}

int main() {
  std::mt19937_64 rng(11);
  std::uniform_real_distribution<double> U01(0.0, 1.0);
  orp p{};
  p.kind = 3;
  p.a = 0.9375;
  p.x1min = 0.1;
  p.x1ref = 0.1;
  p.hslope = 0.3;
  p.poly_xt = 0.82;
  p.poly_alpha = 14.0;
  p.mks_smooth = 0.5;
  const double gam = 13.0 / 9.0;
  double worst[3] = {0, 0, 0}, worstB[3] = {0, 0, 0};
  long failA[3] = {0, 0, 0}, failB[3] = {0, 0, 0}, nA = 0, nB = 0;
  for (int set = 0; set < 2; ++set)
    for (int t = 0; t < 60000; ++t) {
      Met<double> m;
      metric(rng, p, t, m);
      double P[8];
      P[0] = std::exp(std::log(1e-8) * U01(rng));
      P[1] = P[0] * std::exp(std::log(1e-4) * U01(rng)) * 10.0;
      const double vtop = set == 0 ? 3.0 : 50.0, stop = set == 0 ? 30.0 : 1e4;
      const double vmag = std::exp(std::log(1e-5) * U01(rng)) * vtop;
      for (int q = 0; q < 3; ++q) {
        P[2 + q] = vmag * (2 * U01(rng) - 1) / std::sqrt(std::fabs(m.gcov[1 + q][1 + q]));
        P[5 + q] = (2 * U01(rng) - 1) * std::sqrt(P[0] * stop * U01(rng)) / std::sqrt(std::fabs(m.gcov[1 + q][1 + q]));
      }
      FState<double> s;
      fluid_state(P, m, s);
      if (set == 0 && s.bsq > 50.0 * P[0]) continue;
      double U[8];
      cons_only(P, s, m, gam, U);
      double G[8];
      if (set == 0) {
        for (int v = 0; v < 8; ++v) G[v] = P[v] * (1.0 + 1e-3 * (2 * U01(rng) - 1));
        ++nA;
      } else {
        G[0] = std::exp(std::log(1e-8) * U01(rng));
        G[1] = G[0] * std::exp(std::log(1e-4) * U01(rng)) * 10.0;
        for (int q = 0; q < 3; ++q) G[2 + q] = (2 * U01(rng) - 1) / std::sqrt(std::fabs(m.gcov[1 + q][1 + q]));
        for (int q = 0; q < 3; ++q) G[5 + q] = P[5 + q];
        ++nB;
      }
      const double sc_th = std::fmax(P[0], P[1]);
      double sc_u = 0.0;
      for (int q = 0; q < 3; ++q) sc_u = std::fmax(sc_u, std::fabs(P[2 + q]) * std::sqrt(std::fabs(m.gcov[1 + q][1 + q])));
      sc_u = std::fmax(sc_u, 1e-300);
      for (int meth = 0; meth < 3; ++meth) {
        double Q[8];
        for (int v = 0; v < 8; ++v) Q[v] = G[v];
        const int f = solve(meth, U, m, gam, Q);
        if (f) {
          (set == 0 ? failA : failB)[meth]++;
          continue;
        }
        for (int v = 0; v < 5; ++v) {
          const double sc = v < 2 ? sc_th : sc_u / std::sqrt(std::fabs(m.gcov[v - 1][v - 1]));
          double& w = set == 0 ? worst[meth] : worstB[meth];
          w = std::fmax(w, std::fabs(Q[v] - P[v]) / sc);
        }
      }
    }
  for (int meth = 0; meth < 3; ++meth)
    std::printf("%.3e %ld %ld %.3e ", worst[meth], failA[meth], failB[meth], worstB[meth]);
  std::printf("%ld %ld\n", nA, nB);
  return 0;
}
