// Host check of the mixed update's double-float inversion (noble2d_df)
// against the FP64 inversion (noble2d) on seeded magnetised states in
// Minkowski and in the funky-MKS Kerr metric (points from the oracle): both
// recover the primitives whose conserved variables they were given. Prints
// the largest relative error of the double-float result against the state
// (fluid primitives, normalised per zone by max(|P|) over rho, u and by the
// Lorentz-factor scale for u~), the same for the FP64 inversion, the largest
// difference between the two, the number of zones handed back to FP64, the
// number of other failures, the number of states, and the largest relative
// error of the floors' FP32 b^2, Lorentz factor and u_mu (floor_f32) against
// the FP64 fluid state.
#include <cmath>
#include <cstdio>
#include <random>

#include "kh_mixed.cuh"

extern "C" {
struct orp {
  int kind, n1, n2, n3, ng, recon, bc[6];
  double a, gam, x1min, x1max, x2min, x2max, x3min, x3max, hslope, poly_xt, poly_alpha, mks_smooth, cfl, rho_min,
      u_min, bsq_rho_max, bsq_u_max, u_rho_max, gamma_max, x1ref;
};
void or_metric_points(const orp*, int, const double*, const double*, double*, double*, double*, double*);
}

using namespace kh;

int main() {
  std::mt19937_64 rng(5);
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
  FloorParams fl{};
  fl.gamma_max = 50.0;
  fl.u_rho_max = 100.0;
  fl.ibsq_rho_max = 0.01;
  fl.ibsq_u_max = 1.0 / 5000.0;
  const MixedConsts mx = mixed_consts(gam, fl);
  C2POpts o{30, 1e-14};
  double worst_df = 0.0, worst_64 = 0.0, worst_d = 0.0, worst_fl = 0.0;
  long need = 0, fails = 0, n = 0;
  for (int t = 0; t < 200000; ++t) {
    Met<double> m;
    if (t % 4 == 0) {
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) m.gcov[a][b] = m.gcon[a][b] = (a == b) ? (a == 0 ? -1.0 : 1.0) : 0.0;
      m.gdet = 1.0;
      m.alpha = 1.0;
    } else {
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
    double P[8];
    P[0] = std::exp(std::log(1e-8) * U01(rng));
    P[1] = P[0] * std::exp(std::log(1e-4) * U01(rng)) * 10.0;
    const double vmag = std::exp(std::log(1e-5) * U01(rng)) * 3.0;  // |u~| from 3e-5 to 3
    for (int q = 0; q < 3; ++q) {
      P[2 + q] = vmag * (2 * U01(rng) - 1) / std::sqrt(std::fabs(m.gcov[1 + q][1 + q]));
      P[5 + q] = (2 * U01(rng) - 1) * std::sqrt(P[0] * 30.0 * U01(rng)) / std::sqrt(std::fabs(m.gcov[1 + q][1 + q]));
    }
    FState<double> s;
    fluid_state(P, m, s);
    if (s.bsq > 50.0 * P[0]) continue;  // magnetisation within the floors' range
    double U[8];
    cons_only(P, s, m, gam, U);
    ++n;
    // guess: the state perturbed by 1e-3 (a stage input)
    double G[8];
    for (int v = 0; v < 8; ++v) G[v] = P[v] * (1.0 + 1e-3 * (2 * U01(rng) - 1));
    double P64[8];
    for (int v = 0; v < 8; ++v) P64[v] = G[v];
    const double ig = 1.0 / m.gdet;
    const int f64 = noble2d(U, m, ig, gam, 1.0 / gam, (gam - 1.0) / gam, o, P64);
    MetDF md;
    for (int a = 0; a < 4; ++a) md.gcon0[a] = df_of_f64(m.gcon[0][a]);
    const int gs[6][2] = {{1, 1}, {1, 2}, {1, 3}, {2, 2}, {2, 3}, {3, 3}};
    for (int q = 0; q < 6; ++q) {
      const int a = gs[q][0], b = gs[q][1];
      md.gsp[q] = df_of_f64(m.gcon[a][b] - m.gcon[0][a] * m.gcon[0][b] / m.gcon[0][0]);
      md.gcov[q] = df_of_f64(m.gcov[a][b]);
    }
    md.alpha = df_of_f64(m.alpha);
    md.ig = df_of_f64(ig);
    df64 Ud[8], Pd[8];
    for (int v = 0; v < 8; ++v) Ud[v] = df_of_f64(U[v]);
    float W0, vsq0;
    {
      FState<double> sg;
      fluid_state(G, m, sg);
      const double gam2 = (m.alpha * sg.ucon[0]) * (m.alpha * sg.ucon[0]);
      W0 = (float)((G[0] + gam * G[1]) * gam2);
      vsq0 = (float)((gam2 - 1.0) / gam2);
    }
    const int fdf = noble2d_df(Ud, md, mx, W0, vsq0, Pd);
    if (fdf == C2P_NEED_FP64) { ++need; continue; }
    if (fdf != 0 || f64 != 0) { ++fails; continue; }
    const double sc_th = std::fmax(P[0], P[1]);
    double sc_u = 0.0;
    for (int q = 0; q < 3; ++q) sc_u = std::fmax(sc_u, std::fabs(P[2 + q]) * std::sqrt(std::fabs(m.gcov[1 + q][1 + q])));
    sc_u = std::fmax(sc_u, 1e-300);
    {  // the floors' FP32 b^2, Lorentz factor and u_mu against the FP64 fluid state
      df64 Pf[8];
      for (int v = 0; v < 8; ++v) Pf[v] = df_of_f64(P[v]);
      const FloorF32 ff = floor_f32(md, Pf);
      const double g2 = (m.alpha * s.ucon[0]) * (m.alpha * s.ucon[0]);
      worst_fl = std::fmax(worst_fl, std::fabs(ff.bsq - s.bsq) / s.bsq);
      worst_fl = std::fmax(worst_fl, std::fabs(ff.g2 - g2) / g2);
      const float a = md.alpha.hi, gl = std::sqrt(ff.g2);
      const float u_t = a * (a * (md.gcon0[1].hi * ff.ucov[0] + md.gcon0[2].hi * ff.ucov[1] +
                                  md.gcon0[3].hi * ff.ucov[2]) - gl);
      const double usc = std::sqrt(g2) * std::fmax(1.0, m.alpha);
      worst_fl = std::fmax(worst_fl, std::fabs(u_t - s.ucov[0]) / usc);
      for (int q = 0; q < 3; ++q)  // u_i on the scale sqrt(g_ii) gamma
        worst_fl = std::fmax(worst_fl, std::fabs(ff.ucov[q] - s.ucov[1 + q]) /
                                           (std::sqrt(std::fabs(m.gcov[1 + q][1 + q]) * g2)));
    }
    for (int v = 0; v < 5; ++v) {
      const double sc = v < 2 ? sc_th : sc_u / std::sqrt(std::fabs(m.gcov[v - 1][v - 1]));
      const double dv = (double)Pd[v].hi + (double)Pd[v].lo;
      worst_df = std::fmax(worst_df, std::fabs(dv - P[v]) / sc);
      worst_64 = std::fmax(worst_64, std::fabs(P64[v] - P[v]) / sc);
      worst_d = std::fmax(worst_d, std::fabs(dv - P64[v]) / sc);
    }
  }
  std::printf("%.3e %.3e %.3e %ld %ld %ld %.3e\n", worst_df, worst_64, worst_d, need, fails, n, worst_fl);
  return 0;
}
