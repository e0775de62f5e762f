// Host check of the adjoint's reverse-mode face gradient (side_grad_rev)
// against the dual-number evaluation of the same quantity (side_grad_dual)
// on seeded magnetised states in the funky-MKS Kerr metric (from the oracle)
// and in Minkowski, every direction, both signs and both speed branches.
// Prints the largest relative difference.
#include <cmath>
#include <cstdio>
#include <random>

#include "kh_face_vjp.cuh"

extern "C" {
struct orp {
  int kind, n1, n2, n3, ng, recon, bc[6];
  double a, gam, x1min, x1max, x2min, x2max, x3min, x3max, hslope, poly_xt, poly_alpha, mks_smooth, cfl, rho_min,
      u_min, bsq_rho_max, bsq_u_max, u_rho_max, gamma_max, x1ref;
};
void or_metric_points(const orp*, int, const double*, const double*, double*, double*, double*, double*);
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
  double worst = 0.0;
  for (int t = 0; t < 4000; ++t) {
    kh::Met<double> m;
    if (t % 4 == 0) {
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) m.gcov[a][b] = m.gcon[a][b] = (a == b) ? (a == 0 ? -1.0 : 1.0) : 0.0;
      m.gdet = 1.0;
      m.alpha = 1.0;
    } else {
      const double x1 = 0.3 + 3.0 * U01(rng), x2 = 0.05 + 0.9 * U01(rng);
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
    double P[8];
    P[0] = std::exp(std::log(1e-3) * U01(rng));
    P[1] = std::exp(std::log(1e-3) * U01(rng));
    for (int q = 0; q < 3; ++q) {
      P[2 + q] = (2 * U01(rng) - 1) / std::sqrt(std::fabs(m.gcov[1 + q][1 + q]));
      P[5 + q] = (2 * U01(rng) - 1) * std::sqrt(P[0]) / std::sqrt(std::fabs(m.gcov[1 + q][1 + q]));
    }
    double lam[8];
    for (int v = 0; v < 8; ++v) lam[v] = 2 * U01(rng) - 1;
    const double gam = 4.0 / 3.0 + 0.3 * U01(rng);
    const int d = 1 + t % 3;
    const int active = (t / 3) % 3 - 1;
    const double kappa = (U01(rng) - 0.5), lct = 2 * U01(rng) - 1;
    double gr[9], gd2[9];
    kh::side_grad_rev(P, m, gam, lam, kappa, d, active, lct, gr);
    kh::side_grad_dual(P, m, gam, lam, kappa, d, active, lct, gd2);
    double sc = 0.0;
    for (int q = 0; q < 9; ++q) sc = std::fmax(sc, std::fabs(gd2[q]));
    for (int q = 0; q < 9; ++q) worst = std::fmax(worst, std::fabs(gr[q] - gd2[q]) / (sc + 1e-300));
  }
  std::printf("%.3e\n", worst);
  return 0;
}
