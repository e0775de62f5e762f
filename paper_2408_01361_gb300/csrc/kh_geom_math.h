// Geometry arithmetic of the CUDA path (host+device, FP64): the native ->
// Kerr-Schild coordinate map with its first and second derivatives written
// out analytically, the Kerr-Schild metric with its analytic r- and
// theta-derivatives, the chain rule to the native metric and its
// derivatives, a cofactor 4x4 inverse, and the connection
// Gamma^l_{mn} = 1/2 g^{lk} (d_m g_kn + d_n g_km - d_k g_mn).
//
// arXiv 2408.01361: "Code Structure" (GRCoordinates caches the metric and
// connection of a stationary spacetime), "Requirements" (funky MKS widens the
// polar zones; coordinates of Wong et al. 2022).
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define KH_HD __host__ __device__ __forceinline__
#else
#define KH_HD inline
#endif

namespace kh {

enum { COORD_MINKOWSKI = 0, COORD_KS = 1, COORD_MKS = 2, COORD_FMKS = 3 };

struct CoordParams {
  int kind;
  double a;
  double x1min;  // start of the x1 domain (FMKS blending reference)
  double hslope, poly_xt, poly_alpha, mks_smooth;
};

// (r, theta) and their derivatives with respect to the native (x1, x2).
// For every supported map dr/dx2 = 0 and r depends on x1 only.
struct MapD {
  double r, r1, r11;
  double th, th1, th2, th11, th12, th22;
};

KH_HD MapD map_inside(const CoordParams& c, double x1, double x2) {
  const double pi = 3.14159265358979323846;
  MapD m;
  if (c.kind == COORD_KS) {
    m.r = x1; m.r1 = 1.0; m.r11 = 0.0;
    m.th = x2; m.th1 = 0.0; m.th2 = 1.0; m.th11 = 0.0; m.th12 = 0.0; m.th22 = 0.0;
    return m;
  }
  m.r = exp(x1); m.r1 = m.r; m.r11 = m.r;
  const double cc = 0.5 * (1.0 - c.hslope);
  const double s2p = sin(2.0 * pi * x2), c2p = cos(2.0 * pi * x2);
  const double tg = pi * x2 + cc * s2p;
  const double tg2 = pi + 2.0 * pi * cc * c2p;
  const double tg22 = -4.0 * pi * pi * cc * s2p;
  if (c.kind == COORD_MKS) {
    m.th = tg; m.th1 = 0.0; m.th2 = tg2; m.th11 = 0.0; m.th12 = 0.0; m.th22 = tg22;
    return m;
  }
  // FMKS: theta_J polynomial, blended towards theta_G with E = exp(s (x1min - x1)).
  const double al = c.poly_alpha, xt = c.poly_xt;
  const double N = 0.5 * pi / (1.0 + pow(xt, -al) / (al + 1.0));
  const double y = 2.0 * x2 - 1.0;
  const double yx = pow(y / xt, al);
  const double tj = 0.5 * pi + N * y * (1.0 + yx / (al + 1.0));
  const double tj2 = 2.0 * N * (1.0 + yx);
  const double tj22 = 4.0 * N * al * pow(y, al - 1.0) / pow(xt, al);
  const double s = c.mks_smooth;
  const double E = exp(s * (c.x1min - x1));
  m.th = tg + E * (tj - tg);
  m.th1 = -s * E * (tj - tg);
  m.th11 = s * s * E * (tj - tg);
  m.th2 = tg2 + E * (tj2 - tg2);
  m.th12 = -s * E * (tj2 - tg2);
  m.th22 = tg22 + E * (tj22 - tg22);
  return m;
}

// The map continued past the poles by reflection: theta(x1, -x2) = -theta(x1, x2),
// theta(x1, 2 - x2) = 2 pi - theta(x1, x2) (MKS already has this symmetry).
KH_HD MapD coord_map(const CoordParams& c, double x1, double x2) {
  if (c.kind == COORD_FMKS && (x2 < 0.0 || x2 > 1.0)) {
    const double pi = 3.14159265358979323846;
    const bool lo = x2 < 0.0;
    MapD m = map_inside(c, x1, lo ? -x2 : 2.0 - x2);
    m.th = lo ? -m.th : 2.0 * pi - m.th;
    m.th1 = -m.th1;
    m.th11 = -m.th11;
    m.th22 = -m.th22;
    // th2 and th12 are even under the reflection
    return m;
  }
  return map_inside(c, x1, x2);
}

// Kerr-Schild metric g_ab(r, theta) and (optionally) its partial derivatives.
// |sin theta| is held >= 1e-20 (value only) so that faces on the axis keep an
// invertible metric.
struct KSMetric {
  double g[4][4];
  double dr[4][4];
  double dth[4][4];
};

KH_HD void ks_metric(double a, double r, double th, bool derivs, KSMetric& o) {
  double st = sin(th), ct = cos(th);
  if (fabs(st) < 1e-20) st = 1e-20;
  const double s2 = st * st, c2 = ct * ct, a2 = a * a;
  const double sig = r * r + a2 * c2;
  const double z = 2.0 * r / sig;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) { o.g[m][n] = 0.0; o.dr[m][n] = 0.0; o.dth[m][n] = 0.0; }
  const double G33 = sig + a2 * s2 * (1.0 + z);
  o.g[0][0] = z - 1.0;
  o.g[0][1] = o.g[1][0] = z;
  o.g[0][3] = o.g[3][0] = -a * z * s2;
  o.g[1][1] = 1.0 + z;
  o.g[1][3] = o.g[3][1] = -a * s2 * (1.0 + z);
  o.g[2][2] = sig;
  o.g[3][3] = s2 * G33;
  if (!derivs) return;
  // d/dr
  const double sig_r = 2.0 * r;
  const double z_r = 2.0 / sig - 2.0 * r * sig_r / (sig * sig);
  o.dr[0][0] = z_r;
  o.dr[0][1] = o.dr[1][0] = z_r;
  o.dr[0][3] = o.dr[3][0] = -a * s2 * z_r;
  o.dr[1][1] = z_r;
  o.dr[1][3] = o.dr[3][1] = -a * s2 * z_r;
  o.dr[2][2] = sig_r;
  o.dr[3][3] = s2 * (sig_r + a2 * s2 * z_r);
  // d/dtheta
  const double s2_t = 2.0 * st * ct;
  const double sig_t = -2.0 * a2 * ct * st;
  const double z_t = -2.0 * r * sig_t / (sig * sig);
  o.dth[0][0] = z_t;
  o.dth[0][1] = o.dth[1][0] = z_t;
  o.dth[0][3] = o.dth[3][0] = -a * (z_t * s2 + z * s2_t);
  o.dth[1][1] = z_t;
  o.dth[1][3] = o.dth[3][1] = -a * (s2_t * (1.0 + z) + s2 * z_t);
  o.dth[2][2] = sig_t;
  o.dth[3][3] = s2_t * G33 + s2 * (sig_t + a2 * (s2_t * (1.0 + z) + s2 * z_t));
}

// Inverse of a symmetric 4x4 matrix through its cofactors; returns det.
KH_HD double inverse4_cofactor(const double m[4][4], double inv[4][4]) {
  // 2x2 minors of rows (0,1) and (2,3)
  const double s0 = m[0][0] * m[1][1] - m[1][0] * m[0][1];
  const double s1 = m[0][0] * m[1][2] - m[1][0] * m[0][2];
  const double s2 = m[0][0] * m[1][3] - m[1][0] * m[0][3];
  const double s3 = m[0][1] * m[1][2] - m[1][1] * m[0][2];
  const double s4 = m[0][1] * m[1][3] - m[1][1] * m[0][3];
  const double s5 = m[0][2] * m[1][3] - m[1][2] * m[0][3];
  const double c5 = m[2][2] * m[3][3] - m[3][2] * m[2][3];
  const double c4 = m[2][1] * m[3][3] - m[3][1] * m[2][3];
  const double c3 = m[2][1] * m[3][2] - m[3][1] * m[2][2];
  const double c2 = m[2][0] * m[3][3] - m[3][0] * m[2][3];
  const double c1 = m[2][0] * m[3][2] - m[3][0] * m[2][2];
  const double c0 = m[2][0] * m[3][1] - m[3][0] * m[2][1];
  const double det = s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
  const double id = 1.0 / det;
  inv[0][0] = (m[1][1] * c5 - m[1][2] * c4 + m[1][3] * c3) * id;
  inv[0][1] = (-m[0][1] * c5 + m[0][2] * c4 - m[0][3] * c3) * id;
  inv[0][2] = (m[3][1] * s5 - m[3][2] * s4 + m[3][3] * s3) * id;
  inv[0][3] = (-m[2][1] * s5 + m[2][2] * s4 - m[2][3] * s3) * id;
  inv[1][0] = (-m[1][0] * c5 + m[1][2] * c2 - m[1][3] * c1) * id;
  inv[1][1] = (m[0][0] * c5 - m[0][2] * c2 + m[0][3] * c1) * id;
  inv[1][2] = (-m[3][0] * s5 + m[3][2] * s2 - m[3][3] * s1) * id;
  inv[1][3] = (m[2][0] * s5 - m[2][2] * s2 + m[2][3] * s1) * id;
  inv[2][0] = (m[1][0] * c4 - m[1][1] * c2 + m[1][3] * c0) * id;
  inv[2][1] = (-m[0][0] * c4 + m[0][1] * c2 - m[0][3] * c0) * id;
  inv[2][2] = (m[3][0] * s4 - m[3][1] * s2 + m[3][3] * s0) * id;
  inv[2][3] = (-m[2][0] * s4 + m[2][1] * s2 - m[2][3] * s0) * id;
  inv[3][0] = (-m[1][0] * c3 + m[1][1] * c1 - m[1][2] * c0) * id;
  inv[3][1] = (m[0][0] * c3 - m[0][1] * c1 + m[0][2] * c0) * id;
  inv[3][2] = (-m[3][0] * s3 + m[3][1] * s1 - m[3][2] * s0) * id;
  inv[3][3] = (m[2][0] * s3 - m[2][1] * s1 + m[2][2] * s0) * id;
  return det;
}

// Native metric at (x1, x2) and, if dg != nullptr, dg[k][m][n] = d_k g_mn
// (k = 0..3; d_0 = d_3 = 0).
KH_HD void native_metric(const CoordParams& c, double x1, double x2, double g[4][4], double (*dg)[4][4]) {
  if (c.kind == COORD_MINKOWSKI) {
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) {
        g[m][n] = (m == n) ? (m == 0 ? -1.0 : 1.0) : 0.0;
        if (dg)
          for (int k = 0; k < 4; ++k) dg[k][m][n] = 0.0;
      }
    return;
  }
  const MapD M = coord_map(c, x1, x2);
  KSMetric K;
  ks_metric(c.a, M.r, M.th, dg != nullptr, K);
  // Jacobian J[a][m] = d x_KS^a / d x^m and its derivatives dJ[k][a][m]
  double J[4][4] = {{1, 0, 0, 0}, {0, M.r1, 0.0, 0}, {0, M.th1, M.th2, 0}, {0, 0, 0, 1}};
  for (int m = 0; m < 4; ++m)
    for (int n = m; n < 4; ++n) {
      double s = 0.0;
      for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) s += J[p][m] * J[q][n] * K.g[p][q];
      g[m][n] = s;
      g[n][m] = s;
    }
  if (!dg) return;
  double dJ[3][4][4];
  for (int k = 0; k < 3; ++k)
    for (int p = 0; p < 4; ++p)
      for (int q = 0; q < 4; ++q) dJ[k][p][q] = 0.0;
  dJ[1][1][1] = M.r11;
  dJ[1][2][1] = M.th11;
  dJ[1][2][2] = M.th12;
  dJ[2][2][1] = M.th12;
  dJ[2][2][2] = M.th22;
  const double rk[3] = {0.0, M.r1, 0.0};
  const double tk[3] = {0.0, M.th1, M.th2};
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) {
      dg[0][m][n] = 0.0;
      dg[3][m][n] = 0.0;
    }
  for (int k = 1; k <= 2; ++k)
    for (int m = 0; m < 4; ++m)
      for (int n = m; n < 4; ++n) {
        double s = 0.0;
        for (int p = 0; p < 4; ++p)
          for (int q = 0; q < 4; ++q) {
            const double dgpq = K.dr[p][q] * rk[k] + K.dth[p][q] * tk[k];
            s += (dJ[k][p][m] * J[q][n] + J[p][m] * dJ[k][q][n]) * K.g[p][q] + J[p][m] * J[q][n] * dgpq;
          }
        dg[k][m][n] = s;
        dg[k][n][m] = s;
      }
}

// Connection Gamma^l_{mn} from the inverse metric and metric derivatives.
KH_HD void connection_from(const double gcon[4][4], const double dg[4][4][4], double G[4][4][4]) {
  for (int l = 0; l < 4; ++l)
    for (int m = 0; m < 4; ++m)
      for (int n = m; n < 4; ++n) {
        double s = 0.0;
        for (int k = 0; k < 4; ++k) s += gcon[l][k] * (dg[m][k][n] + dg[n][k][m] - dg[k][m][n]);
        G[l][m][n] = 0.5 * s;
        G[l][n][m] = 0.5 * s;
      }
}

}  // namespace kh
