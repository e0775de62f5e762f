// Per-item device functions of the step (one face, edge or zone of one
// block), shared by the single-grid kernels and the multi-block kernels.
#pragma once

#include <type_traits>

#include "kh_internal.h"
#include "kh_mixed.cuh"
#include "kh_pair.cuh"

namespace kh {

// Faces of one direction computed by a flux pass: interior faces along the
// direction, one extra transverse row on each side (Flux-CT needs them).
struct FaceBox {
  int lo[3];
  int n[3];
};

inline FaceBox face_box(const Layout& L, int D) {
  FaceBox b;
  for (int a = 0; a < 3; ++a) {
    const bool active = a < 2 || L.ndim == 3;
    if (!active) {
      b.lo[a] = 0;
      b.n[a] = 1;
    } else if (a == D - 1) {
      b.lo[a] = L.s[a];
      b.n[a] = L.e[a] - L.s[a] + 1;
    } else {
      b.lo[a] = L.s[a] - 1;
      b.n[a] = L.e[a] - L.s[a] + 2;
    }
  }
  return b;
}

// Monotonized-central slope of (qm, q0, qp): zero at an extremum, else the
// candidate of least magnitude among 2 d-, 2 d+ and (d- + d+)/2.
template <class R> __device__ __forceinline__ R mc_slope(R qm, R q0, R qp) {
  const R dl = q0 - qm, dr = qp - q0;
  if (!(dl * dr > R(0))) return R(0);
  R s = R(2) * dl;
  if (kabs(R(2) * dr) < kabs(s)) s = R(2) * dr;
  if (kabs(R(0.5) * (dl + dr)) < kabs(s)) s = R(0.5) * (dl + dr);
  return s;
}

// t -> (a, b, c) with t = a + n0 (b + n1 c), in 32-bit arithmetic (every
// allocation holds fewer than 2^31 cells).
__device__ __forceinline__ void split3(unsigned t, unsigned n0, unsigned n1, int& a, int& b, int& c) {
  const unsigned q = t / n0;
  a = (int)(t - q * n0);
  const unsigned r = q / n1;
  b = (int)(q - r * n1);
  c = (int)r;
}

template <class R>
__device__ __forceinline__ Met<R> load_met(const GeomT<R>& G, long long gplane, int loc, long long p) {
  const R* b = G.g + (long long)loc * NGEO * gplane + p;
  Met<R> m;
  R c[10], u[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    c[q] = __ldg(b + q * gplane);
    u[q] = __ldg(b + (10 + q) * gplane);
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
      m.gcov[mu][nu] = c[sym_index(mu, nu)];
      m.gcon[mu][nu] = u[sym_index(mu, nu)];
    }
  m.gdet = __ldg(b + 20 * gplane);
  m.alpha = __ldg(b + 21 * gplane);
  return m;
}


__device__ __forceinline__ void zone_ijk(const Layout& L, unsigned t, int& i, int& j, int& k) {
  split3(t, L.e[0] - L.s[0], L.e[1] - L.s[1], i, j, k);
  i += L.s[0];
  j += L.s[1];
  k += L.s[2];
}

__device__ __forceinline__ unsigned nzones(const Layout& L) {
  return (unsigned)(L.e[0] - L.s[0]) * (L.e[1] - L.s[1]) * (L.e[2] - L.s[2]);
}

// Reconstruction + LLF flux through the lower x^D face of cell (k, j, i).
// FP32 (mixed path): the left and right states as packed pairs.
template <int D, int RECON>
__device__ __forceinline__ void flux_face_pair(const CVarsT<float>& P, const Layout& L, const GeomT<float>& G,
                                               const Scheme& S, int i, int j, int k, float* F, float* ctop,
                                               int polar_lo, int polar_hi) {
  const long long c = L.at(k, j, i);
  const long long st = (D == 1) ? 1 : (D == 2 ? (long long)L.n1s : (long long)L.n1s * L.n2s);
  P2 Pp[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float* q = P.v[v] + c;
    if (RECON == RECON_DONOR) {
      Pp[v] = P2(__ldg(q - st), __ldg(q));
    } else if (RECON == KH_RECON_MC) {
      const float qm2 = __ldg(q - 2 * st), qm1 = __ldg(q - st), q0 = __ldg(q), qp1 = __ldg(q + st);
      float lo, hi, l2, h2;
      recon_mc(qm2, qm1, q0, lo, hi);
      recon_mc(qm1, q0, qp1, l2, h2);
      Pp[v] = P2(hi, l2);
    } else {
      const float qm3 = __ldg(q - 3 * st), qm2 = __ldg(q - 2 * st), qm1 = __ldg(q - st), q0 = __ldg(q);
      const float qp1 = __ldg(q + st), qp2 = __ldg(q + 2 * st);
      // left: upper face of the cell below; right: lower face of the cell above (mirrored stencil)
      Pp[v] = weno5_plus(P2(qm3, qp2), P2(qm2, qp1), P2(qm1, q0), P2(q0, qm1), P2(qp1, qm2));
    }
  }
  const Met<float> m = load_met(G, L.gplane, D == 3 ? LOC_CENT : D, (long long)j * L.n1s + i);
  const P2 gam(S.mx.gam);
  FState<P2> sp;
  fluid_state(Pp, m, sp);
  P2 Fp[NV], Up[NV];
  flux_cons(Pp, sp, m, gam, D, Fp, Up);
  P2 cmax, cmin;
  signal_speeds(Pp, sp, m, gam, D, cmax, cmin);
  const float ct = fmaxf(fmaxf(0.0f, fmaxf(cmax.v.x, cmax.v.y)), fmaxf(0.0f, fmaxf(-cmin.v.x, -cmin.v.y)));
  const bool axis = (D == 2) && ((polar_lo && j == L.s[1]) || (polar_hi && j == L.e[1]));
#pragma unroll
  for (int v = 0; v < NV; ++v)
    F[v * L.plane + c] = axis ? 0.0f : 0.5f * (Fp[v].v.x + Fp[v].v.y) - 0.5f * ct * (Up[v].v.y - Up[v].v.x);
  ctop[c] = ct;
}

template <int D, int RECON, class TIN, class R>
__device__ __forceinline__ void flux_face(const CVarsT<TIN>& P, const Layout& L, const GeomT<R>& G, const Scheme& S,
                                          int i, int j, int k, R* F, R* ctop, int polar_lo, int polar_hi) {
  if constexpr (sizeof(R) == 4 && sizeof(TIN) == 4) {
    flux_face_pair<D, RECON>(P, L, G, S, i, j, k, F, ctop, polar_lo, polar_hi);
    return;
  }
  const long long c = L.at(k, j, i);
  const long long st = (D == 1) ? 1 : (D == 2 ? (long long)L.n1s : (long long)L.n1s * L.n2s);
  R PL[NV], PR[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const TIN* q = P.v[v] + c;
    if (RECON == RECON_DONOR) {  // piecewise constant: the two cells' own values
      PL[v] = (R)__ldg(q - st);
      PR[v] = (R)__ldg(q);
    } else if (RECON == KH_RECON_MC) {
      const R qm2 = (R)__ldg(q - 2 * st), qm1 = (R)__ldg(q - st), q0 = (R)__ldg(q), qp1 = (R)__ldg(q + st);
      R lo, hi;
      recon_mc(qm2, qm1, q0, lo, hi);
      PL[v] = hi;
      recon_mc(qm1, q0, qp1, lo, hi);
      PR[v] = lo;
    } else {
      const R qm3 = (R)__ldg(q - 3 * st), qm2 = (R)__ldg(q - 2 * st), qm1 = (R)__ldg(q - st), q0 = (R)__ldg(q);
      const R qp1 = (R)__ldg(q + st), qp2 = (R)__ldg(q + 2 * st);
      PL[v] = weno5_plus(qm3, qm2, qm1, q0, qp1);
      PR[v] = weno5_plus(qp2, qp1, q0, qm1, qm2);
    }
  }
  const Met<R> m = load_met(G, L.gplane, D == 3 ? LOC_CENT : D, (long long)j * L.n1s + i);
  const R gam = (R)S.gam;
  FState<R> sL, sR;
  fluid_state(PL, m, sL);
  fluid_state(PR, m, sR);
  R FL[NV], UL[NV], FR[NV], UR[NV];
  flux_cons(PL, sL, m, gam, D, FL, UL);
  flux_cons(PR, sR, m, gam, D, FR, UR);
  R cmaxL, cminL, cmaxR, cminR;
  signal_speeds(PL, sL, m, gam, D, cmaxL, cminL);
  signal_speeds(PR, sR, m, gam, D, cmaxR, cminR);
  const R cm = fmax(R(0), fmax(cmaxL, cmaxR));
  const R cn = fmax(R(0), fmax(-cminL, -cminR));
  const R ct = fmax(cm, cn);
  const bool axis = (D == 2) && ((polar_lo && j == L.s[1]) || (polar_hi && j == L.e[1]));
#pragma unroll
  for (int v = 0; v < NV; ++v)
    F[v * L.plane + c] = axis ? R(0) : R(0.5) * (FL[v] + FR[v]) - R(0.5) * ct * (UR[v] - UL[v]);
  ctop[c] = ct;
}


// Corner EMFs of Flux-CT (Toth 2000) at the edges of cell (k, j, i):
//   e3(i-1/2, j-1/2) = (F1_B2(j) + F1_B2(j-1) - F2_B1(i) - F2_B1(i-1)) / 4 and
//   cyclic e1 (x1-edges), e2 (x2-edges) in 3-D.
template <class R>
__device__ __forceinline__ void emf_at(const R* F1, const R* F2, const R* F3, R* e1, R* e2, R* e3, const Layout& L,
                                       int i, int j, int k) {
  const long long c = L.at(k, j, i);
  const long long P = L.plane, sj = L.n1s, sk = (long long)L.n1s * L.n2s;
  const R q = R(0.25);
  const R* F1B2 = F1 + V_B2 * P;
  const R* F2B1 = F2 + V_B1 * P;
  if (L.ndim == 2) {
    e3[c] = q * (F1B2[c] + F1B2[c - sj] - F2B1[c] - F2B1[c - 1]);
    return;
  }
  // the three edges' loads first (in flight together), then the sums and stores
  const bool d3 = k < L.e[2], d1 = i < L.e[0], d2 = j < L.e[1];
  const R* F2B3 = F2 + V_B3 * P;
  const R* F3B2 = F3 + V_B2 * P;
  const R* F3B1 = F3 + V_B1 * P;
  const R* F1B3 = F1 + V_B3 * P;
  R a[4] = {R(0), R(0), R(0), R(0)}, b[4] = {R(0), R(0), R(0), R(0)}, g[4] = {R(0), R(0), R(0), R(0)};
  if (d3) {
    a[0] = F1B2[c], a[1] = F1B2[c - sj], a[2] = F2B1[c], a[3] = F2B1[c - 1];
  }
  if (d1) {
    b[0] = F2B3[c], b[1] = F2B3[c - sk], b[2] = F3B2[c], b[3] = F3B2[c - sj];
  }
  if (d2) {
    g[0] = F3B1[c], g[1] = F3B1[c - 1], g[2] = F1B3[c], g[3] = F1B3[c - sk];
  }
  if (d3) e3[c] = q * (a[0] + a[1] - a[2] - a[3]);
  if (d1) e1[c] = q * (b[0] + b[1] - b[2] - b[3]);
  if (d2) e2[c] = q * (g[0] + g[1] - g[2] - g[3]);
}


// Field fluxes from edge EMFs (the other slots keep their LLF values):
//   F1 = (0, (e3 + e3(j+1))/2, -(e2 + e2(k+1))/2), F2 = (-(e3 + e3(i+1))/2, 0, (e1 + e1(k+1))/2),
//   F3 = ((e2 + e2(i+1))/2, -(e1 + e1(j+1))/2, 0); in 2-D only e3 and the B1, B2 slots.
template <class R>
__device__ __forceinline__ void apply_ct_at(R* F1, R* F2, R* F3, const R* e1, const R* e2, const R* e3,
                                            const Layout& L, int i, int j, int k) {
  const long long c = L.at(k, j, i);
  const long long P = L.plane, sj = L.n1s, sk = (long long)L.n1s * L.n2s;
  const bool in_i = i < L.e[0], in_j = j < L.e[1];
  const bool in_k = (L.ndim == 2) || k < L.e[2];
  const R h = R(0.5);
  if (in_j && in_k) {  // x1 faces
    F1[V_B1 * P + c] = R(0);
    F1[V_B2 * P + c] = h * (e3[c] + e3[c + sj]);
    if (L.ndim == 3) F1[V_B3 * P + c] = -h * (e2[c] + e2[c + sk]);
  }
  if (in_i && in_k) {  // x2 faces
    F2[V_B1 * P + c] = -h * (e3[c] + e3[c + 1]);
    F2[V_B2 * P + c] = R(0);
    if (L.ndim == 3) F2[V_B3 * P + c] = h * (e1[c] + e1[c + sk]);
  }
  if (L.ndim == 3 && in_i && in_j) {  // x3 faces
    F3[V_B1 * P + c] = h * (e2[c] + e2[c + 1]);
    F3[V_B2 * P + c] = -h * (e1[c] + e1[c + sj]);
    F3[V_B3 * P + c] = R(0);
  }
}

// Connection source terms of the energy and momentum equations,
// S_nu = sqrt(-g) T^k_l Gamma^l_{nu k} (0 for rho and B), evaluated as
// (1/2) sqrt(-g) T^{kl} d_nu g_{kl}: with T^{kl} symmetric, the two terms of
// Gamma_{l nu k} = (d_nu g_{lk} + d_k g_{l nu} - d_l g_{nu k}) / 2 other than
// the first cancel in the contraction. The metric depends on x1 and x2 only,
// so S_t = S_phi = 0 and the sum needs the 2 x 10 derivatives d_1 g, d_2 g.
template <class R, class M>
__device__ __forceinline__ void source_terms(const R* P, const Met<M>& m, const M* dgm, long long gplane, long long p,
                                             R gam, R* S) {
  FState<R> s;
  fluid_state(P, m, s);
  const R pg = (gam - R(1)) * P[V_U];
  const R eta = P[V_RHO] + P[V_U] + pg + s.bsq;
  const R ptot = pg + R(0.5) * s.bsq;
  R acc1 = R(0), acc2 = R(0);
  if constexpr (std::is_same<R, float>::value) {
    // FP32: the two sums as one pair (paired FP32 fused multiply-adds)
    P2 acc(0.0f);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = a; b < 4; ++b) {
        const int q = sym_index(a, b);
        // T^{ab}, every rounding explicit (so that every kernel inlining this rounds alike)
        R t = fmaf(ptot, m.gcon[a][b], fmaf(-s.bcon[a], s.bcon[b], __fmul_rn(__fmul_rn(eta, s.ucon[a]), s.ucon[b])));
        if (a != b) t = R(2) * t;
        acc = pfma(P2(t), P2(__ldg(dgm + q * gplane + p), __ldg(dgm + (10 + q) * gplane + p)), acc);
      }
    acc1 = acc.v.x;
    acc2 = acc.v.y;
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = a; b < 4; ++b) {
        const int q = sym_index(a, b);
        R t = eta * s.ucon[a] * s.ucon[b] - s.bcon[a] * s.bcon[b] + ptot * m.gcon[a][b];  // T^{ab}
        if (a != b) t = R(2) * t;
        acc1 += t * __ldg(dgm + q * gplane + p);
        acc2 += t * __ldg(dgm + (10 + q) * gplane + p);
      }
  }
  S[V_U] = R(0);
  S[V_U1] = R(0.5) * m.gdet * acc1;
  S[V_U2] = R(0.5) * m.gdet * acc2;
  S[V_U3] = R(0);
}


// FP64 update of interior zone (k, j, i): U = U0 + cdt (-div F + S(Pin)),
// Noble-2D inversion with Pin as the guess, floors; writes Pout, pflag and
// (stage 2) U.
// ---------------------------------------------------------------------------
// Face-centred constrained transport (Stone & Gardiner 2009; edge EMFs after
// Gardiner & Stone 2005). Face field fB: planes [3][n3s][n2s][n1s], plane a =
// sqrt(-g) B^(a+1) on the lower x^(a+1) face of each cell (a 2-D grid keeps
// sqrt(-g) B^3 per cell). Edge EMF along x^c, with (a, b, c) cyclic:
// E_c = F^a(B^b) = -F^b(B^a), stored at the cell whose lower x^a and x^b
// faces bound the edge; d/dt (sqrt(-g) B^a) = d_b E_c - d_c E_b.
// ---------------------------------------------------------------------------

// sqrt(-g) B of cell c: the mean of its two faces per direction.
template <class T>
__device__ __forceinline__ void face_means(const T* fB, const Layout& L, long long c, T* UB) {
  const long long P = L.plane, sj = L.n1s, sk = (long long)L.n1s * L.n2s;
  UB[0] = T(0.5) * (fB[c] + fB[c + 1]);
  UB[1] = T(0.5) * (fB[P + c] + fB[P + c + sj]);
  UB[2] = L.ndim == 3 ? T(0.5) * (fB[2 * P + c] + fB[2 * P + c + sk]) : fB[2 * P + c];
}

// Cell-centred EMFs of one cell: E[c] = sqrt(-g) (b^b u^a - b^a u^b).
template <class R, class M>
__device__ __forceinline__ void cell_emfs(const R* P, const Met<M>& m, R* E) {
  FState<R> s;
  fluid_state(P, m, s);
  E[0] = R(m.gdet) * (s.bcon[3] * s.ucon[2] - s.bcon[2] * s.ucon[3]);
  E[1] = R(m.gdet) * (s.bcon[1] * s.ucon[3] - s.bcon[3] * s.ucon[1]);
  E[2] = R(m.gdet) * (s.bcon[2] * s.ucon[1] - s.bcon[1] * s.ucon[2]);
}

// Upwind choice across a face: the lower cell's value for a positive mass
// flux, the upper's for a negative one, their mean for zero.
template <class R> __device__ __forceinline__ R upwind(R mflux, R lower, R upper) {
  return mflux > R(0) ? lower : (mflux < R(0) ? upper : R(0.5) * (lower + upper));
}

// E_c at the edge of cell (k, j, i) from the raw face fluxes F (8 planes per
// direction) and, for GS05, the cell-centred EMFs ecc (3 planes): the mean of
// the four face values, plus (GS05) the differences of the half-zone
// derivatives of E towards the edge, each from the cell upwind of the mass
// flux through the face it belongs to.
template <class R>
__device__ __forceinline__ R edge_emf(int c, const R* const F[3], const R* ecc, const Layout& L, int emf, int i,
                                      int j, int k) {
  const int a = (c + 1) % 3, b = (c + 2) % 3;
  const long long st[3] = {1, (long long)L.n1s, (long long)L.n1s * L.n2s};
  const long long P = L.plane;
  const long long x = L.at(k, j, i), xa = x - st[a], xb = x - st[b], xab = xa - st[b];
  const R* Fa = F[a];
  const R* Fb = F[b];
  const R Ea_hi = Fa[(V_B1 + b) * P + x], Ea_lo = Fa[(V_B1 + b) * P + xb];
  const R Eb_hi = -Fb[(V_B1 + a) * P + x], Eb_lo = -Fb[(V_B1 + a) * P + xa];
  R e = R(0.25) * ((Ea_hi + Ea_lo) + (Eb_hi + Eb_lo));
  if (emf == KH_EMF_GS05) {
    const R* C = ecc + c * P;
    const R db_hi = upwind(Fa[x], C[xa] - Eb_lo, C[x] - Eb_hi);
    const R db_lo = upwind(Fa[xb], Eb_lo - C[xab], Eb_hi - C[xb]);
    const R da_hi = upwind(Fb[x], C[xb] - Ea_lo, C[x] - Ea_hi);
    const R da_lo = upwind(Fb[xa], Ea_lo - C[xab], Ea_hi - C[xa]);
    e += R(0.25) * ((db_lo - db_hi) + (da_lo - da_hi));
  }
  return e;
}

// TRIAL (first-order flux correction): the same update, inversion and floors,
// but only the zone's flag is written: pflag[c] = 1 if the inversion failed or
// a floor acted, else 0 (flagged zones counted in CNT_FOFC); Pout, Uout and
// the failure counters are not touched.
template <bool TRIAL = false, int INV = C2P_NOBLE2D>
__device__ __forceinline__ void update_zone(const double* U0, const CVars& Pin, const Vars& Pout, double* Uout,
                                            const double* F1, const double* F2, const double* F3, const Layout& L,
                                            const DevGeom& G, const Scheme& S, double cdt, int8_t* pflag,
                                            unsigned long long* cnt, int i, int j, int k, double* Praw = nullptr,
                                            FailList fl = FailList{nullptr, nullptr, 0u}, const double* fBn = nullptr,
                                            double* dUout = nullptr) {
  const long long c = L.at(k, j, i);
  const long long p = (long long)j * L.n1s + i;
  const long long sj = L.n1s, sk = (long long)L.n1s * L.n2s;
  const Met<double> m = load_met(G, L.gplane, LOC_CENT, p);
  double P[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) P[v] = Pin.v[v][c];
  double Sv[NV] = {0, 0, 0, 0, 0, 0, 0, 0};
  source_terms(P, m, G.dgm, L.gplane, p, S.gam, Sv);
  double U[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const long long o = v * L.plane + c;
    double div = (F1[o + 1] - F1[o]) * L.idx[0] + (F2[o + sj] - F2[o]) * L.idx[1];
    if (L.ndim == 3) div += (F3[o + sk] - F3[o]) * L.idx[2];
    U[v] = U0[o] + cdt * (-div + Sv[v]);
    if (dUout) dUout[o] = cdt * (-div + Sv[v]);  // the raw increment (Runge-Kutta stages)
  }
  if (fBn) face_means(fBn, L, c, U + V_B1);  // face-centred CT: sqrt(-g) B from the updated faces
  double Pn[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Pn[v] = P[v];
  const double ig = __ldg(G.flo + 2 * L.gplane + p);  // 1 / sqrt(-g)
  const int flag = invert<INV>(U, m, ig, S.gam, S.igam, S.gfac, S.c2p, Pn);
  if (TRIAL && flag) {
    pflag[c] = 1;
    atomicAdd(cnt + CNT_FOFC, 1ULL);
    return;
  }
  Pn[V_B1] = U[V_B1] * ig;
  Pn[V_B2] = U[V_B2] * ig;
  Pn[V_B3] = U[V_B3] * ig;
  if (Praw) {  // the adjoint's record of the inversion result before floors
#pragma unroll
    for (int v = 0; v < NV; ++v) Praw[v * L.plane + c] = Pn[v];
  }
  int fmask = 0;
  if (flag == 0) {
    FState<double> s;
    fluid_state(Pn, m, s);
    fmask = apply_floors(S.fl, m, __ldg(G.flo + p), __ldg(G.flo + L.gplane + p), s.bsq, Pn);
    if (TRIAL) {
      pflag[c] = fmask ? 1 : 0;
      if (fmask) atomicAdd(cnt + CNT_FOFC, 1ULL);
      return;
    }
    if (fmask && Uout) {
      fluid_state(Pn, m, s);
      cons_only(Pn, s, m, S.gam, U);
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) Pout.v[v][c] = Pn[v];
  if (Uout) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Uout[v * L.plane + c] = U[v];
  }
  pflag[c] = (int8_t)flag;
  if (flag) {
    atomicAdd(cnt + CNT_FAIL, 1ULL);
    if (fl.idx) fl.idx[atomicAdd(fl.n, 1ULL)] = fl.tag | (unsigned)c;
  }
  if (fmask) atomicAdd(cnt + CNT_FLOOR, 1ULL);
}


// Edge EMFs of Flux-CT (k_emf's output). When given to the mixed update, the
// field components' face fluxes are formed from them right there (the
// values k_apply_ct would have stored: halved sums of two edge EMFs; a
// halving is exact, so the divergence rounds as before) instead of read back.
struct CtEmf {
  const float* e[3];
};

// Where the mixed update of one zone reads its inputs -- the stage input P,
// U^n, the face fluxes of the fluid variables and Flux-CT's edge EMFs -- as
// values around the zone: f(d, v, up) is variable v's flux through the
// zone's lower (up = 0) or upper (up = 1) x^(d+1) face, e(a, di, dj, dk) the
// x^(a+1)-edge EMF at offset (di, dj, dk) from the zone's lower corner.
// MixedInGlobal reads the arrays in global memory (the layout of L); the
// TMA-staged update kernel reads shared-memory tiles through its own view.
struct MixedInGlobal {
  const double* U0;
  CVarsT<float> Pin;
  const float* F[3];
  CtEmf ect;
  long long c, sj, sk, plane;
  __device__ __forceinline__ float pin(int v) const { return Pin.v[v][c]; }
  __device__ __forceinline__ double u0(int v) const { return U0[v * plane + c]; }
  __device__ __forceinline__ float f(int d, int v, int up) const {
    return F[d][v * plane + c + (up ? (d == 0 ? 1 : (d == 1 ? sj : sk)) : 0)];
  }
  __device__ __forceinline__ float e(int a, int di, int dj, int dk) const {
    return ect.e[a][c + di + dj * sj + dk * sk];
  }
  __device__ __forceinline__ bool has_emf() const { return ect.e[2] != nullptr; }
};

// The FP64 inversion of a zone whose double-float iteration handed it back
// (C2P_NEED_FP64; a handful of zones per step once the flow has settled): the
// FP64 solver from the FP32 stage input (Pin8) as the guess. Returns the
// solver's flag; on success Pn5 holds the fluid primitives. The out-of-line
// form (mixed_fp64_fallback) keeps the FP64 solver off the hot path of an
// update whose long straight-line code already stalls on instruction fetch.
template <int INV>
__device__ __forceinline__ int mixed_fp64_fallback_inl(const df64* Ud, const float* Pin8, DevGeom G, long long gplane,
                                                long long p, double gam, double igam, double gfac, C2POpts o,
                                                df64* Pn5) {
  double Uf[NV], Pd[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    Uf[v] = f64_of_df(Ud[v]);
    Pd[v] = f64_of_f32(Pin8[v]);
  }
  const Met<double> m = load_met(G, gplane, LOC_CENT, p);
  const int flag = invert<INV>(Uf, m, __ldg(G.flo + 2 * gplane + p), gam, igam, gfac, o, Pd);
  if (flag == 0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) Pn5[v] = df_of_f64(Pd[v]);
  }
  return flag;
}

// The same, out of line.
template <int INV>
__device__ __noinline__ int mixed_fp64_fallback(const df64* Ud, const float* Pin8, DevGeom G, long long gplane,
                                                long long p, double gam, double igam, double gfac, C2POpts o,
                                                df64* Pn5) {
  return mixed_fp64_fallback_inl<INV>(Ud, Pin8, G, gplane, p, gam, igam, gfac, o, Pn5);
}

// A zone whose Lorentz-factor ceiling changed u~ (rare): its conserved
// variables recomputed in FP64 from the floored primitives Pn and written to
// Uc (stride plane). Inlined: out of line it cost the TMA-staged update 2%.
__device__ __forceinline__ void recompute_u_fp64(const df64* Pn, const DevGeom& G, long long gplane, long long p,
                                                 double gam, double* Uc, long long plane) {
  double Pd[NV], U[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Pd[v] = f64_of_df(Pn[v]);
  const Met<double> m = load_met(G, gplane, LOC_CENT, p);
  FState<double> s;
  fluid_state(Pd, m, s);
  cons_only(Pd, s, m, gam, U);
#pragma unroll
  for (int v = 0; v < NV; ++v) Uc[v * plane] = U[v];
}

// The end of the mixed update when its inversion stays in FP64 for every
// zone (kh_coords.mixed_inversion = KH_MIXINV_FP64, the precision split that
// keeps the whole Noble-2D inversion in FP64): U holds the FP64 conserved
// variables U^n + increment; the FP64 Noble-2D iteration starts from the
// FP32 stage input; floors as on the FP64 path (FP64 decisions and values),
// U recomputed in FP64 where one acted; outputs as update_mixed_zone's.
template <bool TRIAL, class IN>
__device__ __forceinline__ void update_mixed_fp64_tail(double* U, const IN& in, const Vars& Pout64,
                                                       const VarsT<float>& Pout32, double* Uout, const Layout& L,
                                                       const DevGeom& G, const Scheme& S, int8_t* pflag,
                                                       unsigned long long* cnt, long long c, long long p,
                                                       FailList fl) {
  const Met<double> m = load_met(G, L.gplane, LOC_CENT, p);
  double Pn[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Pn[v] = f64_of_f32(in.pin(v));
  const double ig = __ldg(G.flo + 2 * L.gplane + p);  // 1 / sqrt(-g)
  const int flag = invert<C2P_NOBLE2D>(U, m, ig, S.gam, S.igam, S.gfac, S.c2p, Pn);
  if (TRIAL && flag) {
    pflag[c] = 1;
    atomicAdd(cnt + CNT_FOFC, 1ULL);
    return;
  }
  Pn[V_B1] = U[V_B1] * ig;
  Pn[V_B2] = U[V_B2] * ig;
  Pn[V_B3] = U[V_B3] * ig;
  int fmask = 0;
  if (flag == 0) {
    FState<double> sb;
    fluid_state(Pn, m, sb);
    fmask = apply_floors(S.fl, m, __ldg(G.flo + p), __ldg(G.flo + L.gplane + p), sb.bsq, Pn);
    if (TRIAL) {
      pflag[c] = fmask ? 1 : 0;
      if (fmask) atomicAdd(cnt + CNT_FOFC, 1ULL);
      return;
    }
    if (fmask && Uout) {
      fluid_state(Pn, m, sb);
      cons_only(Pn, sb, m, S.gam, U);
#pragma unroll
      for (int v = 0; v < NV; ++v) Uout[v * L.plane + c] = U[v];
    }
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) Pn[v] = f64_of_f32(in.pin(v));  // provisional, replaced by the fixup
  }
  if (Pout32.v[0]) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Pout32.v[v][c] = f32_of_f64(Pn[v]);
  }
  if (Pout64.v[0]) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Pout64.v[v][c] = Pn[v];
  }
  pflag[c] = (int8_t)flag;
  if (flag) {
    atomicAdd(cnt + CNT_FAIL, 1ULL);
    if (fl.idx) fl.idx[atomicAdd(fl.n, 1ULL)] = fl.tag | (unsigned)c;
  }
  if (fmask) atomicAdd(cnt + CNT_FLOOR, 1ULL);
}

// The mixed update of one zone, FP64 arithmetic only where the result is
// FP64 storage. FP32: the stage input, the sources, the flux divergence, the
// increment c dt (S - div F), the floors' decisions and b^2. Double-float
// (kh_df64.cuh, on the FP32 pipe): the updated conserved variables entering
// the inversion, the inversion (noble2d_df) and the primitives. FP64: the
// stored conserved variables U^n + increment (an FP64 add per variable, the
// conserved update exact to FP64 as in the FP64 path), the FP64 primitives
// written at stage 2 (one add of the pair each) and the FP64 fallback
// inversion of the zones noble2d_df hands back. TRIAL: the first-order flux
// correction's trial, as update_zone<true> (Uout must be null). INV: the
// solver; Noble-2D runs in double-float with the FP64 fallback, the others
// invert every zone in FP64 (from the double-float U rounded to FP64).
// INV = C2P_NOBLE2D_FP64: the FP64 Noble-2D for every zone from the FP64
// U^n + increment (update_mixed_fp64_tail).
// COLD: the FP64 fallback inversion is called out of line (the TMA-staged
// kernels, whose instruction fetch stalls them: 1% faster so; and the mesh's
// own-loads update, so that it runs the same compiled copy as the mesh's
// staged update and the two round alike) or inlined (the trial and the
// single grid's own-loads update).
template <bool TRIAL, int INV, class IN, bool COLD = false>
__device__ __forceinline__ void update_mixed_zone_in(const IN& in, const Vars& Pout64, const VarsT<float>& Pout32,
                                                     double* Uout, const Layout& L, const DevGeom& G,
                                                     const GeomT<float>& Gf, const Scheme& S, df64 cdt,
                                                     int8_t* pflag, unsigned long long* cnt, int i, int j, int k,
                                                     FailList fl, const double* fBn, double* dUout) {
  const long long c = L.at(k, j, i);
  const long long p = (long long)j * L.n1s + i;
  const MixedConsts& mx = S.mx;
  // the stored U (stage 2) is written here and touched again only by floors
  df64 Ud[NV];    // U^n + increment, double-float, for the inversion
  double Ue[NV];  // ... in FP64 (C2P_NOBLE2D_FP64 only)
  float W0, vsq0; // initial guess of the inversion from the FP32 input
  {
    float Pf[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Pf[v] = in.pin(v);
    float Sv[NV] = {0, 0, 0, 0, 0, 0, 0, 0};
    const Met<float> mf = load_met(Gf, L.gplane, LOC_CENT, p);
    source_terms(Pf, mf, Gf.dgm, L.gplane, p, mx.gam, Sv);
    {  // W = (rho + gam u) gamma^2, v^2 = q / gamma^2
      const float v1 = Pf[V_U1], v2 = Pf[V_U2], v3 = Pf[V_U3];
      const float q = mf.gcov[1][1] * v1 * v1 + mf.gcov[2][2] * v2 * v2 + mf.gcov[3][3] * v3 * v3 +
                      2.0f * (mf.gcov[1][2] * v1 * v2 + mf.gcov[1][3] * v1 * v3 + mf.gcov[2][3] * v2 * v3);
      const float g2 = 1.0f + q;
      W0 = (Pf[V_RHO] + mx.gam * Pf[V_U]) * g2;
      vsq0 = kdiv(q, g2);
    }
    const float i1 = L.idxf[0], i2 = L.idxf[1], i3 = L.idxf[2];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const long long o = v * L.plane + c;
      // lower / upper face fluxes per direction
      float a1, b1, a2, b2, a3 = 0.0f, b3 = 0.0f;
      const bool three = L.ndim == 3;
      if (in.has_emf() && v >= V_B1 && (three || v != V_B3)) {
        // the field's face fluxes from the edge EMFs, each product rounded
        // on its own (no fusing with the difference below)
        const float h = 0.5f;
        auto em = [](float w, float e0, float e1) { return __fmul_rn(w, __fadd_rn(e0, e1)); };
        if (v == V_B1) {
          a1 = 0.0f;
          b1 = 0.0f;
          a2 = em(-h, in.e(2, 0, 0, 0), in.e(2, 1, 0, 0));
          b2 = em(-h, in.e(2, 0, 1, 0), in.e(2, 1, 1, 0));
          if (three) {
            a3 = em(h, in.e(1, 0, 0, 0), in.e(1, 1, 0, 0));
            b3 = em(h, in.e(1, 0, 0, 1), in.e(1, 1, 0, 1));
          }
        } else if (v == V_B2) {
          a1 = em(h, in.e(2, 0, 0, 0), in.e(2, 0, 1, 0));
          b1 = em(h, in.e(2, 1, 0, 0), in.e(2, 1, 1, 0));
          a2 = 0.0f;
          b2 = 0.0f;
          if (three) {
            a3 = em(-h, in.e(0, 0, 0, 0), in.e(0, 0, 1, 0));
            b3 = em(-h, in.e(0, 0, 0, 1), in.e(0, 0, 1, 1));
          }
        } else {  // B3, 3-D
          a1 = em(-h, in.e(1, 0, 0, 0), in.e(1, 0, 0, 1));
          b1 = em(-h, in.e(1, 1, 0, 0), in.e(1, 1, 0, 1));
          a2 = em(h, in.e(0, 0, 0, 0), in.e(0, 0, 0, 1));
          b2 = em(h, in.e(0, 0, 1, 0), in.e(0, 0, 1, 1));
        }
      } else {
        a1 = in.f(0, v, 0);
        b1 = in.f(0, v, 1);
        a2 = in.f(1, v, 0);
        b2 = in.f(1, v, 1);
        if (three) {
          a3 = in.f(2, v, 0);
          b3 = in.f(2, v, 1);
        }
      }
      // fused as written, so that every kernel inlining this rounds alike
      float div = __fmaf_rn(b2 - a2, i2, __fmul_rn(b1 - a1, i1));
      if (three) div = __fmaf_rn(b3 - a3, i3, div);
      const float inc = (cdt * __fsub_rn(Sv[v], div)).hi;  // c dt (S - div F)
      const double u0 = in.u0(v);
      if (dUout) dUout[o] = f64_of_f32(inc);  // the raw increment (Runge-Kutta stages)
      if (Uout) {
        const double un = u0 + f64_of_f32(inc);  // the conserved update, FP64
        Uout[o] = un;
        if constexpr (INV == C2P_NOBLE2D_FP64) Ue[v] = un;
        else Ud[v] = df_of_f64(un);  // the stored sum split, in place of a second (double-float) sum
      } else {
        if constexpr (INV == C2P_NOBLE2D_FP64) Ue[v] = u0 + f64_of_f32(inc);
        else Ud[v] = df_of_f64(u0) + inc;
      }
    }
  }
  if (fBn) {  // face-centred CT: sqrt(-g) B from the updated faces (FP64 means)
    double UB[3];
    face_means(fBn, L, c, UB);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (Uout) Uout[(V_B1 + q) * L.plane + c] = UB[q];
      if constexpr (INV == C2P_NOBLE2D_FP64) Ue[V_B1 + q] = UB[q];
      else Ud[V_B1 + q] = df_of_f64(UB[q]);
    }
  }
  if constexpr (INV == C2P_NOBLE2D_FP64) {
    update_mixed_fp64_tail<TRIAL>(Ue, in, Pout64, Pout32, Uout, L, G, S, pflag, cnt, c, p, fl);
    return;
  }
  const MetDF md = load_metdf(Gf.df, L.gplane, p);
  df64 Pn[NV];
  Pn[V_B1] = Ud[V_B1] * md.ig;
  Pn[V_B2] = Ud[V_B2] * md.ig;
  Pn[V_B3] = Ud[V_B3] * md.ig;
  int flag = C2P_NEED_FP64;
  if constexpr (INV == C2P_NOBLE2D) flag = noble2d_df(Ud, md, mx, W0, vsq0, Pn);
  if (flag == C2P_NEED_FP64) {
    // FP64 inversion of this zone from the stage input (out of line; the
    // arrays it takes are copies, so that Ud and Pn stay in registers)
    if (!TRIAL && INV == C2P_NOBLE2D) atomicAdd(cnt + CNT_FP64, 1ULL);
    df64 Uc[NV], P5[5];
    float Pi[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Uc[v] = Ud[v];
      Pi[v] = in.pin(v);
    }
    if constexpr (COLD) flag = mixed_fp64_fallback<INV>(Uc, Pi, G, L.gplane, p, S.gam, S.igam, S.gfac, S.c2p, P5);
    else flag = mixed_fp64_fallback_inl<INV>(Uc, Pi, G, L.gplane, p, S.gam, S.igam, S.gfac, S.c2p, P5);
    if (flag == 0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) Pn[v] = P5[v];
    }
  }
  if (TRIAL && flag) {
    pflag[c] = 1;
    atomicAdd(cnt + CNT_FOFC, 1ULL);
    return;
  }
  if (flag) {
#pragma unroll
    for (int v = 0; v < 5; ++v) Pn[v] = mkdf(in.pin(v), 0.0f);
  }
  int fmask = 0;
  if (flag == 0) {
    // floors: decisions on FP32 b^2 and Lorentz factor (from the double-float
    // metric's leading parts, no further loads), values in double-float
    const FloorF32 sf = floor_f32(md, Pn);
    const df64 rho0 = Pn[V_RHO], u0 = Pn[V_U];
    const df64 rf = dfmax(md.rho_fl, mkdf(sf.bsq * mx.ibsq_rho_max, 0.0f));
    const df64 uf = dfmax(md.u_fl, mkdf(sf.bsq * mx.ibsq_u_max, 0.0f));
    if (Pn[V_RHO] < rf) { Pn[V_RHO] = rf; fmask |= 1; }
    if (Pn[V_U] < uf) { Pn[V_U] = uf; fmask |= 1; }
    const df64 umax = Pn[V_RHO] * mx.u_rho_max;
    if (Pn[V_U] > umax) { Pn[V_U] = umax; fmask |= 2; }
    if (sf.g2 > 0.999f * mx.g2max) {  // the FP32 Lorentz factor gates the exact test
      const df64 qq = spatial_sq(md, Pn[V_U1], Pn[V_U2], Pn[V_U3]);
      if (qq.hi + 1.0f > mx.g2max) {
        const df64 sc = dfsqrt(mkdf(mx.g2max - 1.0f, 0.0f) / qq);
        Pn[V_U1] = Pn[V_U1] * sc;
        Pn[V_U2] = Pn[V_U2] * sc;
        Pn[V_U3] = Pn[V_U3] * sc;
        fmask |= 4;
      }
    }
    if (TRIAL) {
      pflag[c] = fmask ? 1 : 0;
      if (fmask) atomicAdd(cnt + CNT_FOFC, 1ULL);
      return;
    }
    if (fmask && Uout) {
      double* Uc = Uout + c;
      if (fmask & 4) {  // the Lorentz-factor ceiling changed u~: full FP64 recompute
        recompute_u_fp64(Pn, G, L.gplane, p, S.gam, Uc, L.plane);
      } else {
        // at fixed u~ and B, U is linear in (rho, u): add
        // drho dU/drho + du dU/du, formed in FP32, to the FP64 U
        const float drho = (Pn[V_RHO] - rho0).hi, du = (Pn[V_U] - u0).hi;
        float ut, u_t;
        floor_ut(md, sf, ut, u_t);
        const float gm = mx.gam, gd = kdiv(1.0f, md.ig.hi);
        // (every rounding explicit, so that every kernel inlining this rounds alike)
        const float gu = fmul(gd, ut), dm = fmaf(gm, du, drho);
        Uc[V_RHO * L.plane] += f64_of_f32(fmul(gu, drho));
        Uc[V_U * L.plane] +=
            f64_of_f32(fmul(gd, fmaf(fmaf(ut, u_t, ut), drho, fmul(fsub(fmaf(fmul(gm, ut), u_t, gm), 1.0f), du))));
        Uc[V_U1 * L.plane] += f64_of_f32(fmul(fmul(gu, sf.ucov[0]), dm));
        Uc[V_U2 * L.plane] += f64_of_f32(fmul(fmul(gu, sf.ucov[1]), dm));
        Uc[V_U3 * L.plane] += f64_of_f32(fmul(fmul(gu, sf.ucov[2]), dm));
      }
    }
  }
  if (Pout32.v[0]) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Pout32.v[v][c] = Pn[v].hi;
  }
  if (Pout64.v[0]) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Pout64.v[v][c] = f64_of_df(Pn[v]);
  }
  pflag[c] = (int8_t)flag;
  if (flag) {
    atomicAdd(cnt + CNT_FAIL, 1ULL);
    if (fl.idx) fl.idx[atomicAdd(fl.n, 1ULL)] = fl.tag | (unsigned)c;
  }
  if (fmask) atomicAdd(cnt + CNT_FLOOR, 1ULL);
}


// The mixed update of zone (i, j, k) reading its inputs from global memory
// (COLD as for update_mixed_zone_in).
template <bool TRIAL = false, int INV = C2P_NOBLE2D, bool COLD = false>
__device__ __forceinline__ void update_mixed_zone(const double* U0, const CVarsT<float>& Pin, const Vars& Pout64,
                                                  const VarsT<float>& Pout32, double* Uout, const float* F1,
                                                  const float* F2, const float* F3, const Layout& L, const DevGeom& G,
                                                  const GeomT<float>& Gf, const Scheme& S, df64 cdt, int8_t* pflag,
                                                  unsigned long long* cnt, int i, int j, int k,
                                                  FailList fl = FailList{nullptr, nullptr, 0u},
                                                  const double* fBn = nullptr, double* dUout = nullptr,
                                                  CtEmf ect = CtEmf{{nullptr, nullptr, nullptr}}) {
  const MixedInGlobal in{U0, Pin, {F1, F2, F3}, ect, L.at(k, j, i), (long long)L.n1s, (long long)L.n1s * L.n2s,
                         L.plane};
  update_mixed_zone_in<TRIAL, INV, MixedInGlobal, COLD>(in, Pout64, Pout32, Uout, L, G, Gf, S, cdt, pflag, cnt, i, j,
                                                        k, fl, fBn, dUout);
}

// Fixup: a zone whose inversion failed takes the equal-weight mean of the
// fluid primitives of its non-failed interior neighbours (3x3x3, or 3x3 in
// 2-D); with none it keeps the stage input. Then floors; U recomputed.
// The repair after the neighbour mean (sum[5] over n good neighbours):
// floors, the primitives written, U recomputed.
template <class T>
__device__ __forceinline__ void fixup_finish(const VarsT<T>& P, double* Uout, const Layout& L, const DevGeom& G,
                                             const Scheme& S, unsigned long long* cnt, int i, int j, int k,
                                             const double* sum, int n) {
  const long long c = L.at(k, j, i);
  double Pn[NV];
  for (int v = 0; v < NV; ++v) Pn[v] = (double)P.v[v][c];
  if (n > 0) {
    for (int v = 0; v < 5; ++v) Pn[v] = sum[v] / n;
  } else {
    atomicAdd(cnt + CNT_UNFIXED, 1ULL);
  }
  const long long p = (long long)j * L.n1s + i;
  const Met<double> m = load_met(G, L.gplane, LOC_CENT, p);
  FState<double> sb;
  fluid_state(Pn, m, sb);
  const int fmask = apply_floors(S.fl, m, __ldg(G.flo + p), __ldg(G.flo + L.gplane + p), sb.bsq, Pn);
  if (fmask) atomicAdd(cnt + CNT_FLOOR, 1ULL);
  for (int v = 0; v < 5; ++v) P.v[v][c] = (T)Pn[v];
  if (Uout) {
    FState<double> s;
    fluid_state(Pn, m, s);
    double U[NV];
    cons_only(Pn, s, m, S.gam, U);
    for (int v = 0; v < NV; ++v) Uout[v * L.plane + c] = U[v];
  }
}

// The fixup of failed zone (i, j, k) by one warp: lane l examines neighbour
// l of the 3x3(x3) block (26 or 8 of them) at once, the sums meet by
// shuffles, and lane 0 finishes the repair (a serial walk over the
// neighbours is a chain of dependent loads). Every lane of the warp calls it.
template <class T>
__device__ __forceinline__ void fixup_warp(const VarsT<T>& P, double* Uout, const int8_t* pflag, const Layout& L,
                                           const DevGeom& G, const Scheme& S, unsigned long long* cnt, int i, int j,
                                           int k, int lane) {
  const int nnb = L.ndim == 3 ? 26 : 8;
  double s[5] = {0, 0, 0, 0, 0};
  int good = 0;
  if (lane < nnb) {
    // neighbour offsets in (dk, dj, di) order, the centre skipped
    const int side = L.ndim == 3 ? 3 : 1;
    const int idx = lane < (side * 9) / 2 ? lane : lane + 1;
    const int dk = L.ndim == 3 ? idx / 9 - 1 : 0, dj = (idx / 3) % 3 - 1, di = idx % 3 - 1;
    const int ii = i + di, jj = j + dj, kk = k + dk;
    if (ii >= L.s[0] && ii < L.e[0] && jj >= L.s[1] && jj < L.e[1] && kk >= L.s[2] && kk < L.e[2]) {
      const long long qn = L.at(kk, jj, ii);
      if (pflag[qn] == 0) {
        good = 1;
#pragma unroll
        for (int v = 0; v < 5; ++v) s[v] = (double)P.v[v][qn];
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int v = 0; v < 5; ++v) s[v] += __shfl_xor_sync(0xffffffffu, s[v], o);
    good += __shfl_xor_sync(0xffffffffu, good, o);
  }
  if (lane == 0) fixup_finish<T>(P, Uout, L, G, S, cnt, i, j, k, s, good);
  __syncwarp();
}

template <class T>
__device__ __forceinline__ void fixup_zone(const VarsT<T>& P, double* Uout, const int8_t* pflag, const Layout& L,
                                           const DevGeom& G, const Scheme& S, unsigned long long* cnt, int i, int j,
                                           int k) {
  const long long c = L.at(k, j, i);
  if (pflag[c] == 0) return;
  double sum[5] = {0, 0, 0, 0, 0};
  int n = 0;
  const int kl = L.ndim == 3 ? -1 : 0, kh = L.ndim == 3 ? 1 : 0;
  for (int dk = kl; dk <= kh; ++dk)
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        if (dk == 0 && dj == 0 && di == 0) continue;
        const int ii = i + di, jj = j + dj, kk = k + dk;
        if (ii < L.s[0] || ii >= L.e[0] || jj < L.s[1] || jj >= L.e[1] || kk < L.s[2] || kk >= L.e[2]) continue;
        const long long q = L.at(kk, jj, ii);
        if (pflag[q] != 0) continue;
        for (int v = 0; v < 5; ++v) sum[v] += (double)P.v[v][q];
        ++n;
      }
  double Pn[NV];
  for (int v = 0; v < NV; ++v) Pn[v] = (double)P.v[v][c];
  if (n > 0) {
    for (int v = 0; v < 5; ++v) Pn[v] = sum[v] / n;
  } else {
    atomicAdd(cnt + CNT_UNFIXED, 1ULL);
  }
  const long long p = (long long)j * L.n1s + i;
  const Met<double> m = load_met(G, L.gplane, LOC_CENT, p);
  FState<double> sb;
  fluid_state(Pn, m, sb);
  const int fmask = apply_floors(S.fl, m, __ldg(G.flo + p), __ldg(G.flo + L.gplane + p), sb.bsq, Pn);
  if (fmask) atomicAdd(cnt + CNT_FLOOR, 1ULL);
  for (int v = 0; v < 5; ++v) P.v[v][c] = (T)Pn[v];
  if (Uout) {
    FState<double> s;
    fluid_state(Pn, m, s);
    double U[NV];
    cons_only(Pn, s, m, S.gam, U);
    for (int v = 0; v < NV; ++v) Uout[v * L.plane + c] = U[v];
  }
}


// sum_d max(ctop_d(lower face), ctop_d(upper face)) / dx_d of zone (k, j, i),
// in the precision of the signal speeds (FP32 on the mixed path).
__device__ __forceinline__ double cfl_inv_zone(const double* c1, const double* c2, const double* c3, const Layout& L,
                                               int i, int j, int k) {
  const long long c = L.at(k, j, i);
  const long long sj = L.n1s, sk = (long long)L.n1s * L.n2s;
  double inv = fmax(c1[c], c1[c + 1]) * L.idx[0] + fmax(c2[c], c2[c + sj]) * L.idx[1];
  if (L.ndim == 3) inv += fmax(c3[c], c3[c + sk]) * L.idx[2];
  return inv;
}
__device__ __forceinline__ float cfl_inv_zone(const float* c1, const float* c2, const float* c3, const Layout& L,
                                              int i, int j, int k) {
  const long long c = L.at(k, j, i);
  const long long sj = L.n1s, sk = (long long)L.n1s * L.n2s;
  float inv = fmaxf(c1[c], c1[c + 1]) * L.idxf[0] + fmaxf(c2[c], c2[c + sj]) * L.idxf[1];
  if (L.ndim == 3) inv += fmaxf(c3[c], c3[c + sk]) * L.idxf[2];
  return inv;
}

// Corner divergence of sqrt(-g) B at the lower corner of cell (i, j, k): per
// direction d, the average of sqrt(-g) B^d over the 2 (2-D) or 4 (3-D) cells
// above the corner minus that over the cells below, divided by dx_d. gd is
// the sqrt(-g) plane at cell centres.
__device__ __forceinline__ double divb_corner(const double* B1, const double* B2, const double* B3, const Layout& L,
                                              const double* gd, int i, int j, int k) {
  auto gB = [&](const double* B, int kk, int jj, int ii) { return gd[(long long)jj * L.n1s + ii] * B[L.at(kk, jj, ii)]; };
  if (L.ndim == 2)
    return (gB(B1, k, j, i) + gB(B1, k, j - 1, i) - gB(B1, k, j, i - 1) - gB(B1, k, j - 1, i - 1)) / (2.0 * L.dx[0]) +
           (gB(B2, k, j, i) + gB(B2, k, j, i - 1) - gB(B2, k, j - 1, i) - gB(B2, k, j - 1, i - 1)) / (2.0 * L.dx[1]);
  const double a1 = gB(B1, k, j, i) + gB(B1, k, j - 1, i) + gB(B1, k - 1, j, i) + gB(B1, k - 1, j - 1, i);
  const double b1 = gB(B1, k, j, i - 1) + gB(B1, k, j - 1, i - 1) + gB(B1, k - 1, j, i - 1) + gB(B1, k - 1, j - 1, i - 1);
  const double a2 = gB(B2, k, j, i) + gB(B2, k, j, i - 1) + gB(B2, k - 1, j, i) + gB(B2, k - 1, j, i - 1);
  const double b2 = gB(B2, k, j - 1, i) + gB(B2, k, j - 1, i - 1) + gB(B2, k - 1, j - 1, i) + gB(B2, k - 1, j - 1, i - 1);
  const double a3 = gB(B3, k, j, i) + gB(B3, k, j, i - 1) + gB(B3, k, j - 1, i) + gB(B3, k, j - 1, i - 1);
  const double b3 = gB(B3, k - 1, j, i) + gB(B3, k - 1, j, i - 1) + gB(B3, k - 1, j - 1, i) + gB(B3, k - 1, j - 1, i - 1);
  return (a1 - b1) / (4.0 * L.dx[0]) + (a2 - b2) / (4.0 * L.dx[1]) + (a3 - b3) / (4.0 * L.dx[2]);
}

}  // namespace kh
