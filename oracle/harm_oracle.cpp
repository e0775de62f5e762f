// Grid-level oracle: boundaries, fluxes with Flux-CT, sources, the two-stage
// update, primitive recovery, floors, fixup, the CFL time step and divB; the
// first-order flux correction; face-centred constrained transport (parity
// partly unpinned there: which side the upwinded EMF derivative terms take
// is fixed by no property the tests check; it changes results at second
// order only).
//
// TEST INFRASTRUCTURE ONLY (see harm_oracle.hpp). Exposed to Python through a
// plain C API (prefix or_) for the parity tests, the pin tests and the CPU
// baseline of the benchmark.
//
// Array layout used by every or_ entry point: double[8][N3][N2][N1] with
// ghosts included and no padding (N1 = n1 + 2 ng, N2 = n2 + 2 ng,
// N3 = n3 + 2 ng or 1 for a 2-D problem), slot order rho, u, u~1..3, B1..3.
#include <omp.h>

#include <cstdio>
#include <cstring>
#include <limits>

#include "harm_oracle.hpp"

using namespace oracle;

namespace {

struct Grid {
  Params c;
  GridInfo g;
  // Geometry cache over (j, i) of the ghosted grid, per location (the metric
  // depends only on x1 and x2).
  std::vector<Geo> geo[5];
  std::vector<double> conn;  // [N2][N1][4][4][4] at cell centres

  size_t idx(int v, int k, int j, int i) const {
    return ((static_cast<size_t>(v) * g.N3 + k) * g.N2 + j) * g.N1 + i;
  }
  size_t cells() const { return static_cast<size_t>(g.N1) * g.N2 * g.N3; }
  const Geo& G(int loc, int j, int i) const { return geo[loc][static_cast<size_t>(j) * g.N1 + i]; }
  const double (*C(int j, int i) const)[4][4] {
    return reinterpret_cast<const double(*)[4][4]>(&conn[(static_cast<size_t>(j) * g.N1 + i) * 64]);
  }
  // Interior index ranges [s, e) per direction.
  int s1() const { return g.ng; }
  int e1() const { return g.ng + g.n1; }
  int s2() const { return g.ng; }
  int e2() const { return g.ng + g.n2; }
  int s3() const { return g.ng3; }
  int e3() const { return g.ng3 + g.n3; }
};

void build_grid(const Params& c, Grid& gr) {
  gr.c = c;
  gr.g = grid_info(c);
  const GridInfo& g = gr.g;
  for (int loc = 0; loc < 5; ++loc) {
    gr.geo[loc].resize(static_cast<size_t>(g.N1) * g.N2);
    for (int j = 0; j < g.N2; ++j)
      for (int i = 0; i < g.N1; ++i) {
        // x3 faces share the cell-centre metric (no x3 dependence).
        int l = (loc == LOC_FACE3) ? LOC_CENT : loc;
        double x1, x2;
        loc_coords(c, g, l, i, j, x1, x2);
        gr.geo[loc][static_cast<size_t>(j) * g.N1 + i] = geo_at(c, x1, x2);
      }
  }
  gr.conn.assign(static_cast<size_t>(g.N1) * g.N2 * 64, 0.0);
  for (int j = 0; j < g.N2; ++j)
    for (int i = 0; i < g.N1; ++i) {
      double x1, x2;
      loc_coords(c, g, LOC_CENT, i, j, x1, x2);
      double cn[4][4][4];
      connection_at(c, x1, x2, cn);
      std::memcpy(&gr.conn[(static_cast<size_t>(j) * g.N1 + i) * 64], cn, sizeof(cn));
    }
}

// Boyer-Lindquist-independent radius of a cell centre (used only by the floors):
// r for KS-family coordinates, 1 for Minkowski (floors are then constants).
double radius_at(const Grid& gr, int j, int i) {
  if (gr.c.kind == MINKOWSKI) return 1.0;
  double x1, x2, r, th;
  loc_coords(gr.c, gr.g, LOC_CENT, i, j, x1, x2);
  native_to_ks<double>(gr.c, x1, x2, r, th);
  return r;
}

// ---------------------------------------------------------------------------
// Boundary conditions on the primitives (all 8 slots). x1 ghosts are filled
// over interior (j, k); x2 ghosts over all i and interior k; x3 ghosts over all
// i and j, so edge and corner ghosts are compositions of the face rules.
//   periodic: copy from the opposite side;
//   outflow:  copy the last interior zone; x1 faces forbid inflow by clamping
//             u~1 (<= 0 at the inner face, >= 0 at the outer face);
//   polar:    reflect across the face, flipping the sign of u~2 and B2;
//   dirichlet: copy caller-supplied ghost values (x1 faces only).
// ---------------------------------------------------------------------------
template <class R>
void apply_bc(const Grid& gr, R* P, const double* dir_lo, const double* dir_hi) {
  const GridInfo& g = gr.g;
  const int ng = g.ng;
  // x1
  for (int k = gr.s3(); k < gr.e3(); ++k)
    for (int j = gr.s2(); j < gr.e2(); ++j)
      for (int m = 0; m < ng; ++m) {
        int ilo = ng - 1 - m, ihi = ng + g.n1 + m;
        for (int side = 0; side < 2; ++side) {
          int bc = gr.c.bc[side];
          int ig = side == 0 ? ilo : ihi;
          for (int v = 0; v < NVAR; ++v) {
            R x(0.0);
            if (bc == BC_PERIODIC) {
              int src = side == 0 ? ig + g.n1 : ig - g.n1;
              x = P[gr.idx(v, k, j, src)];
            } else if (bc == BC_OUTFLOW) {
              int src = side == 0 ? ng : ng + g.n1 - 1;
              x = P[gr.idx(v, k, j, src)];
            } else if (bc == BC_DIRICHLET) {
              const double* D = side == 0 ? dir_lo : dir_hi;
              int ii = side == 0 ? ig : ig - (ng + g.n1);  // 0..ng-1
              x = R(D[((static_cast<size_t>(v) * g.N3 + k) * g.N2 + j) * ng + ii]);
            } else {  // polar reflection across an x1 face is not meaningful; copy
              int src = side == 0 ? 2 * ng - 1 - ig : 2 * (ng + g.n1) - 1 - ig;
              x = P[gr.idx(v, k, j, src)];
            }
            P[gr.idx(v, k, j, ig)] = x;
          }
          if (bc == BC_OUTFLOW) {
            R& u1 = P[gr.idx(U1, k, j, ig)];
            if (side == 0 && u1 > 0.0) u1 = R(0.0);
            if (side == 1 && u1 < 0.0) u1 = R(0.0);
          }
        }
      }
  // x2
  for (int k = gr.s3(); k < gr.e3(); ++k)
    for (int i = 0; i < g.N1; ++i)
      for (int m = 0; m < ng; ++m) {
        int jlo = ng - 1 - m, jhi = ng + g.n2 + m;
        for (int side = 0; side < 2; ++side) {
          int bc = gr.c.bc[2 + side];
          int jg = side == 0 ? jlo : jhi;
          int src;
          if (bc == BC_PERIODIC)
            src = side == 0 ? jg + g.n2 : jg - g.n2;
          else if (bc == BC_OUTFLOW)
            src = side == 0 ? ng : ng + g.n2 - 1;
          else  // polar
            src = side == 0 ? 2 * ng - 1 - jg : 2 * (ng + g.n2) - 1 - jg;
          for (int v = 0; v < NVAR; ++v) {
            R x = P[gr.idx(v, k, src, i)];
            if (bc == BC_POLAR && (v == U2 || v == B2)) x = -x;
            P[gr.idx(v, k, jg, i)] = x;
          }
        }
      }
  // x3
  if (g.ndim == 3) {
    for (int j = 0; j < g.N2; ++j)
      for (int i = 0; i < g.N1; ++i)
        for (int m = 0; m < g.ng3; ++m) {
          int klo = g.ng3 - 1 - m, khi = g.ng3 + g.n3 + m;
          for (int side = 0; side < 2; ++side) {
            int bc = gr.c.bc[4 + side];
            int kg = side == 0 ? klo : khi;
            int src;
            if (bc == BC_PERIODIC)
              src = side == 0 ? kg + g.n3 : kg - g.n3;
            else
              src = side == 0 ? g.ng3 : g.ng3 + g.n3 - 1;
            for (int v = 0; v < NVAR; ++v) P[gr.idx(v, kg, j, i)] = P[gr.idx(v, src, j, i)];
          }
        }
  }
}

// ---------------------------------------------------------------------------
// Fluxes: reconstruction + LLF at every face needed by the update and by
// Flux-CT (one transverse row beyond the interior), polar zeroing, Flux-CT.
// F[d] has the cell layout; F[d] at (k,j,i) is the flux through the lower
// x^d face of cell (k,j,i). ctop[d] likewise.
// ---------------------------------------------------------------------------
template <class R> struct FluxesT {
  std::vector<R> F[3];
  std::vector<double> ctop[3];  // signal speeds (values only: they set dt)
};
using Fluxes = FluxesT<double>;

void face_range(const Grid& gr, int d, int lo[3], int hi[3]) {
  // inclusive ranges in (i, j, k) order
  int s[3] = {gr.s1(), gr.s2(), gr.s3()};
  int e[3] = {gr.e1(), gr.e2(), gr.e3()};
  for (int a = 0; a < 3; ++a) {
    bool active = (a < 2) || gr.g.ndim == 3;
    if (!active) { lo[a] = 0; hi[a] = 0; continue; }
    if (a == d) { lo[a] = s[a]; hi[a] = e[a]; }
    else { lo[a] = s[a] - 1; hi[a] = e[a]; }
  }
}

template <class R>
void finish_fluxes(const Grid& gr, FluxesT<R>& fx);

// Raw LLF face fluxes (before polar zeroing and Flux-CT).
template <class R>
void compute_raw(const Grid& gr, const R* P, FluxesT<R>& fx, const R& gam) {
  const GridInfo& g = gr.g;
  const size_t n = gr.cells();
  for (int d = 0; d < 3; ++d) {
    fx.F[d].assign(NVAR * n, R(0.0));
    fx.ctop[d].assign(n, 0.0);
  }
  for (int d = 0; d < g.ndim; ++d) {
    int lo[3], hi[3];
    face_range(gr, d, lo, hi);
    const int loc = LOC_FACE1 + d;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          R PL[NVAR], PR[NVAR];
          for (int v = 0; v < NVAR; ++v) {
            // stencil of the cell below the face (c = -1) and above it (c = 0)
            R qm[5], qp[5];
            for (int s = 0; s < 5; ++s) {
              int o1 = (d == 0) ? s - 3 : 0, o2 = (d == 1) ? s - 3 : 0, o3 = (d == 2) ? s - 3 : 0;
              qm[s] = P[gr.idx(v, k + o3, j + o2, i + o1)];
              int p1 = (d == 0) ? s - 2 : 0, p2 = (d == 1) ? s - 2 : 0, p3 = (d == 2) ? s - 2 : 0;
              qp[s] = P[gr.idx(v, k + p3, j + p2, i + p1)];
            }
            R lo_m, hi_m, lo_p, hi_p;
            recon_cell(gr.c.recon, qm, lo_m, hi_m);
            recon_cell(gr.c.recon, qp, lo_p, hi_p);
            PL[v] = hi_m;
            PR[v] = lo_p;
          }
          R F[NVAR], ct;
          llf_flux<R>(PL, PR, gr.G(loc, j, i), gam, d + 1, F, ct);
          for (int v = 0; v < NVAR; ++v) fx.F[d][gr.idx(v, k, j, i)] = F[v];
          fx.ctop[d][gr.idx(0, k, j, i)] = val(ct);
        }
  }
}

template <class R>
void compute_fluxes(const Grid& gr, const R* P, FluxesT<R>& fx, const R& gam) {
  compute_raw(gr, P, fx, gam);
  finish_fluxes(gr, fx);
}

// Polar axis: no flux of anything through an x2 face lying on the axis.
template <class R>
void polar_zero(const Grid& gr, FluxesT<R>& fx) {
  int lo[3], hi[3];
  face_range(gr, 1, lo, hi);
  for (int side = 0; side < 2; ++side) {
    if (gr.c.bc[2 + side] != BC_POLAR) continue;
    int j = side == 0 ? gr.s2() : gr.e2();
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int i = lo[0]; i <= hi[0]; ++i)
        for (int v = 0; v < NVAR; ++v) fx.F[1][gr.idx(v, k, j, i)] = R(0.0);
  }
}

// Polar-axis zeroing and Flux-CT applied to the raw face fluxes of fx.
template <class R>
void finish_fluxes(const Grid& gr, FluxesT<R>& fx) {
  const GridInfo& g = gr.g;
  const size_t n = gr.cells();
  polar_zero(gr, fx);
  // Flux-CT (Toth 2000): corner EMFs as averages of the four adjacent face
  // fluxes of the field, then field fluxes as averages of the edge EMFs.
  std::vector<R>& F1 = fx.F[0];
  std::vector<R>& F2 = fx.F[1];
  std::vector<R>& F3 = fx.F[2];
  std::vector<R> e1(n, R(0.0)), e2(n, R(0.0)), e3(n, R(0.0));
  auto I = [&](int k, int j, int i) { return gr.idx(0, k, j, i); };
  auto V = [&](int v, int k, int j, int i) { return gr.idx(v, k, j, i); };
  if (g.ndim == 2) {
    const int k = 0;
    for (int j = gr.s2(); j <= gr.e2(); ++j)
      for (int i = gr.s1(); i <= gr.e1(); ++i)
        e3[I(k, j, i)] = 0.25 * (F1[V(B2, k, j, i)] + F1[V(B2, k, j - 1, i)] - F2[V(B1, k, j, i)] - F2[V(B1, k, j, i - 1)]);
    for (int j = gr.s2(); j < gr.e2(); ++j)
      for (int i = gr.s1(); i <= gr.e1(); ++i) {
        F1[V(B1, k, j, i)] = R(0.0);
        F1[V(B2, k, j, i)] = 0.5 * (e3[I(k, j, i)] + e3[I(k, j + 1, i)]);
      }
    for (int j = gr.s2(); j <= gr.e2(); ++j)
      for (int i = gr.s1(); i < gr.e1(); ++i) {
        F2[V(B1, k, j, i)] = -0.5 * (e3[I(k, j, i)] + e3[I(k, j, i + 1)]);
        F2[V(B2, k, j, i)] = R(0.0);
      }
    return;
  }
  for (int k = gr.s3(); k <= gr.e3(); ++k)
    for (int j = gr.s2(); j <= gr.e2(); ++j)
      for (int i = gr.s1(); i <= gr.e1(); ++i) {
        // emf3 on the x3-edge at (i-1/2, j-1/2, k)
        if (k < gr.e3())
          e3[I(k, j, i)] = 0.25 * (F1[V(B2, k, j, i)] + F1[V(B2, k, j - 1, i)] - F2[V(B1, k, j, i)] - F2[V(B1, k, j, i - 1)]);
        // emf1 on the x1-edge at (i, j-1/2, k-1/2)
        if (i < gr.e1())
          e1[I(k, j, i)] = 0.25 * (F2[V(B3, k, j, i)] + F2[V(B3, k - 1, j, i)] - F3[V(B2, k, j, i)] - F3[V(B2, k, j - 1, i)]);
        // emf2 on the x2-edge at (i-1/2, j, k-1/2)
        if (j < gr.e2())
          e2[I(k, j, i)] = 0.25 * (F3[V(B1, k, j, i)] + F3[V(B1, k, j, i - 1)] - F1[V(B3, k, j, i)] - F1[V(B3, k - 1, j, i)]);
      }
  for (int k = gr.s3(); k < gr.e3(); ++k)
    for (int j = gr.s2(); j < gr.e2(); ++j)
      for (int i = gr.s1(); i <= gr.e1(); ++i) {
        F1[V(B1, k, j, i)] = R(0.0);
        F1[V(B2, k, j, i)] = 0.5 * (e3[I(k, j, i)] + e3[I(k, j + 1, i)]);
        F1[V(B3, k, j, i)] = -0.5 * (e2[I(k, j, i)] + e2[I(k + 1, j, i)]);
      }
  for (int k = gr.s3(); k < gr.e3(); ++k)
    for (int j = gr.s2(); j <= gr.e2(); ++j)
      for (int i = gr.s1(); i < gr.e1(); ++i) {
        F2[V(B1, k, j, i)] = -0.5 * (e3[I(k, j, i)] + e3[I(k, j, i + 1)]);
        F2[V(B2, k, j, i)] = R(0.0);
        F2[V(B3, k, j, i)] = 0.5 * (e1[I(k, j, i)] + e1[I(k + 1, j, i)]);
      }
  for (int k = gr.s3(); k <= gr.e3(); ++k)
    for (int j = gr.s2(); j < gr.e2(); ++j)
      for (int i = gr.s1(); i < gr.e1(); ++i) {
        F3[V(B1, k, j, i)] = 0.5 * (e2[I(k, j, i)] + e2[I(k, j, i + 1)]);
        F3[V(B2, k, j, i)] = -0.5 * (e1[I(k, j, i)] + e1[I(k, j + 1, i)]);
        F3[V(B3, k, j, i)] = R(0.0);
      }
}

// ---------------------------------------------------------------------------
// Face-centred constrained transport (the paper's "Algorithm" section: the
// scheme of Stone & Gardiner 2009, edge EMFs after Gardiner & Stone 2005).
// The field lives on faces: fB[a][k][j][i] = sqrt(-g) B^(a+1) at the lower
// x^(a+1) face of cell (k, j, i) (a 2-D grid keeps sqrt(-g) B^3 per cell).
// With v = (a, b, c) cyclic, the edge EMF along x^c is
//   E_c = sqrt(-g) (b^b u^a - b^a u^b) = F^a(B^b) = -F^b(B^a)
// (F^d the x^d flux of sqrt(-g) B), stored at the cell whose lower x^a and
// x^b faces bound the edge, and the induction equation is
//   d/dt (sqrt(-g) B^a) = d_b E_c - d_c E_b,
// whose discrete form keeps the face divergence of every cell unchanged.
// ---------------------------------------------------------------------------

// Cell-centred EMFs from the cell's primitives: E[c] along x^(c+1).
template <class R>
void cell_emfs(const R P[NVAR], const Geo& G, R E[3]) {
  FluidState<R> S;
  fluid_state(P, G, S);
  for (int c = 0; c < 3; ++c) {
    const int a = (c + 1) % 3 + 1, b = (c + 2) % 3 + 1;  // 4-vector indices of x^a, x^b
    E[c] = G.gdet * (S.bcon[b] * S.ucon[a] - S.bcon[a] * S.ucon[b]);
  }
}

// Edge EMFs from the raw face fluxes fx (after polar zeroing) and the stage
// input P (ghosts filled). EMF_AVERAGE: the mean of the four face values
// around the edge. EMF_GS05: that mean plus, along each of the two face
// directions, the difference of the half-zone derivatives of E between the
// faces and the edge, each taken from the cell upwind of the mass flux
// through the face it is attached to (the mean of both cells when that flux
// is zero). EMFs on edges lying on a polar axis are zero (the axis faces
// carry no flux). E[c] covers the edges the interior faces need.
template <class R>
void face_emfs(const Grid& gr, const R* P, const FluxesT<R>& fx, std::vector<R> E[3]) {
  const GridInfo& g = gr.g;
  const size_t n = gr.cells();
  for (int c = 0; c < 3; ++c) E[c].assign(n, R(0.0));
  // cell-centred EMFs on every cell (ghosts included)
  std::vector<R> Ec[3];
  for (int c = 0; c < 3; ++c) Ec[c].assign(n, R(0.0));
  if (gr.c.emf == EMF_GS05)
    for (int k = 0; k < g.N3; ++k)
      for (int j = 0; j < g.N2; ++j)
        for (int i = 0; i < g.N1; ++i) {
          R Pc[NVAR], e[3];
          for (int v = 0; v < NVAR; ++v) Pc[v] = P[gr.idx(v, k, j, i)];
          cell_emfs<R>(Pc, gr.G(LOC_CENT, j, i), e);
          for (int c = 0; c < 3; ++c) Ec[c][gr.idx(0, k, j, i)] = e[c];
        }
  const int nd = g.ndim;
  const int s[3] = {gr.s1(), gr.s2(), gr.s3()}, e[3] = {gr.e1(), gr.e2(), gr.e3()};
  auto at = [&](const int x[3]) { return gr.idx(0, x[2], x[1], x[0]); };
  auto flux = [&](int d, int v, const int x[3]) { return fx.F[d][gr.idx(v, x[2], x[1], x[0])]; };
  for (int c = 0; c < 3; ++c) {
    const int a = (c + 1) % 3, b = (c + 2) % 3;  // edge along x^c between faces normal to x^a and x^b
    if (nd == 2 && c != 2) {
      // no x3 variation: E1 is the x2-face value F^2(B^3), E2 minus the x1-face value F^1(B^3)
      const int d = c == 0 ? 1 : 0;
      const double sg = c == 0 ? 1.0 : -1.0;
      for (int j = s[1]; j <= e[1] - (d == 0 ? 1 : 0); ++j)
        for (int i = s[0]; i <= e[0] - (d == 1 ? 1 : 0); ++i) {
          const int x[3] = {i, j, 0};
          E[c][at(x)] = sg * flux(d, B3, x);
        }
      continue;
    }
    if (nd == 2 && (a == 2 || b == 2)) continue;
    int lo[3], hi[3];
    for (int q = 0; q < 3; ++q) {
      const bool active = q < nd;
      lo[q] = active ? s[q] : 0;
      hi[q] = active ? (q == c ? e[q] - 1 : e[q]) : 0;  // edges: both ends along a and b
    }
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          const int x[3] = {i, j, k};
          int xb[3] = {i, j, k}, xa[3] = {i, j, k}, xab[3] = {i, j, k};
          xb[b] -= 1;   // the cell below in x^b
          xa[a] -= 1;   // the cell below in x^a
          xab[a] -= 1;
          xab[b] -= 1;  // the cell below in both
          // face values of E_c: on x^a faces F^a(B^b), on x^b faces -F^b(B^a)
          const R Ea_hi = flux(a, B1 + b, x), Ea_lo = flux(a, B1 + b, xb);     // x^a faces at b, b-1
          const R Eb_hi = -flux(b, B1 + a, x), Eb_lo = -flux(b, B1 + a, xa);   // x^b faces at a, a-1
          R emf = 0.25 * (Ea_hi + Ea_lo + Eb_hi + Eb_lo);
          if (gr.c.emf == EMF_GS05) {
            const std::vector<R>& C = Ec[c];
            // along x^b, on the x^a faces: upwind across x^a by the mass flux there
            auto up_a = [&](const R& mflux, const R& lowcell, const R& highcell) {
              if (mflux > 0.0) return lowcell;
              if (mflux < 0.0) return highcell;
              return R(0.5 * (lowcell + highcell));
            };
            // (half-zone derivative x half width) above the edge in x^b: centre(b) - face(b-1/2)
            const R db_hi = up_a(flux(a, RHO, x), C[at(xa)] - Eb_lo, C[at(x)] - Eb_hi);
            // below the edge in x^b: face(b-1/2) - centre(b-1)
            const R db_lo = up_a(flux(a, RHO, xb), Eb_lo - C[at(xab)], Eb_hi - C[at(xb)]);
            // along x^a, on the x^b faces: upwind across x^b
            const R da_hi = up_a(flux(b, RHO, x), C[at(xb)] - Ea_lo, C[at(x)] - Ea_hi);
            const R da_lo = up_a(flux(b, RHO, xa), Ea_lo - C[at(xab)], Ea_hi - C[at(xa)]);
            emf += 0.25 * ((db_lo - db_hi) + (da_lo - da_hi));
          }
          E[c][at(x)] = emf;
        }
  }
  // polar axis: edges along x1 and x3 lying on an axis carry no EMF
  for (int side = 0; side < 2; ++side) {
    if (gr.c.bc[2 + side] != BC_POLAR) continue;
    const int j = side == 0 ? s[1] : e[1];
    for (int k = 0; k < g.N3; ++k)
      for (int i = 0; i < g.N1; ++i) {
        E[0][gr.idx(0, k, j, i)] = R(0.0);
        E[2][gr.idx(0, k, j, i)] = R(0.0);
      }
  }
}

// Face update of one stage over every face of the interior cells (both
// bounding faces along the normal): fBout = fB0 + cdt (d_b E_c - d_c E_b).
// fB0 and fBout may be the same array.
template <class R>
void face_update(const Grid& gr, const R* fB0, const std::vector<R> E[3], double cdt, R* fBout) {
  const GridInfo& g = gr.g;
  const int nd = g.ndim;
  const double dx[3] = {g.dx1, g.dx2, g.dx3};
  const int s[3] = {gr.s1(), gr.s2(), gr.s3()}, e[3] = {gr.e1(), gr.e2(), gr.e3()};
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    int lo[3], hi[3];
    for (int q = 0; q < 3; ++q) {
      lo[q] = s[q];
      hi[q] = (q == a && q < nd) ? e[q] : e[q] - 1;
    }
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          const int x[3] = {i, j, k};
          int xb[3] = {i, j, k}, xc[3] = {i, j, k};
          xb[b] += 1;
          xc[c] += 1;
          const size_t f = gr.idx(a, k, j, i), o = gr.idx(0, k, j, i);
          R rhs(0.0);
          if (b < nd) rhs += (E[c][gr.idx(0, xb[2], xb[1], xb[0])] - E[c][o]) / dx[b];
          if (c < nd) rhs -= (E[b][gr.idx(0, xc[2], xc[1], xc[0])] - E[b][o]) / dx[c];
          (void)x;
          fBout[f] = fB0[f] + cdt * rhs;
        }
  }
}

// sqrt(-g) B at cell centres: the mean of the two faces along each direction
// (the face value itself along x3 on a 2-D grid).
template <class R>
void face_to_cell_u(const Grid& gr, const R* fB, int k, int j, int i, R UB[3]) {
  const int nd = gr.g.ndim;
  UB[0] = 0.5 * (fB[gr.idx(0, k, j, i)] + fB[gr.idx(0, k, j, i + 1)]);
  UB[1] = 0.5 * (fB[gr.idx(1, k, j, i)] + fB[gr.idx(1, k, j + 1, i)]);
  UB[2] = nd == 3 ? R(0.5 * (fB[gr.idx(2, k, j, i)] + fB[gr.idx(2, k + 1, j, i)])) : fB[gr.idx(2, k, j, i)];
}

// ---------------------------------------------------------------------------
// Floors (applied after each successful inversion and after each fixup).
//   rho >= max(rho_min r^-3/2, 1e-20, b^2 / bsq_rho_max)
//   u   >= max(u_min r^-5/2, 1e-20, b^2 / bsq_u_max)
//   u   <= u_rho_max rho
//   gamma <= gamma_max (u~ rescaled so that gamma = gamma_max)
// Returns a bit mask: 1 density/energy floor, 2 temperature ceiling, 4 gamma.
// ---------------------------------------------------------------------------
int apply_floors(const Params& c, const Geo& G, double r, double P[NVAR]) {
  FluidState<double> S;
  fluid_state(P, G, S);
  double rho_fl = std::max(c.rho_min * std::pow(r, -1.5), 1e-20);
  double u_fl = std::max(c.u_min * std::pow(r, -2.5), 1e-20);
  rho_fl = std::max(rho_fl, S.bsq / c.bsq_rho_max);
  u_fl = std::max(u_fl, S.bsq / c.bsq_u_max);
  int flag = 0;
  if (P[RHO] < rho_fl) { P[RHO] = rho_fl; flag |= 1; }
  if (P[UU] < u_fl) { P[UU] = u_fl; flag |= 1; }
  if (P[UU] > c.u_rho_max * P[RHO]) { P[UU] = c.u_rho_max * P[RHO]; flag |= 2; }
  double qsq = 0.0;
  for (int i = 1; i < 4; ++i)
    for (int j = 1; j < 4; ++j) qsq += G.gcov[i][j] * P[U1 + i - 1] * P[U1 + j - 1];
  double gamma = std::sqrt(1.0 + qsq);
  if (gamma > c.gamma_max) {
    double f = std::sqrt((c.gamma_max * c.gamma_max - 1.0) / (gamma * gamma - 1.0));
    for (int i = 0; i < 3; ++i) P[U1 + i] *= f;
    flag |= 4;
  }
  return flag;
}

template <class R>
void p2c_at(const Geo& G, const R P[NVAR], const R& gam, R U[NVAR]) {
  FluidState<R> S;
  fluid_state(P, G, S);
  prim_to_flux<R>(P, S, G, gam, 0, U);
}

void p2c_point(const Params& c, const Geo& G, const double P[NVAR], double U[NVAR]) { p2c_at<double>(G, P, c.gam, U); }

// ---------------------------------------------------------------------------
// Tangent (forward-mode) versions of the two non-smooth point operations, for
// the step templated on Dual<double>. Values are always those of the plain
// FP64 operations above; only the derivative rules are added here.
// ---------------------------------------------------------------------------
using Dd = Dual<double>;

int invert_point(const double U[NVAR], const Geo& G, const double& gam, double P[NVAR]) {
  return cons_to_prim_point(U, G, gam, P);
}

// Solve A x = b (n x n, row-major) by Gaussian elimination with partial
// pivoting. Returns false on a zero pivot.
bool solve_dense(int n, double* A, double* b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c) {
      for (int q = 0; q < n; ++q) std::swap(A[c * n + q], A[piv * n + q]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = A[r * n + c] / A[c * n + c];
      for (int q = c; q < n; ++q) A[r * n + q] -= f * A[c * n + q];
      b[r] -= f * b[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double acc = b[c];
    for (int q = c + 1; q < n; ++q) acc -= A[c * n + q] * b[q];
    b[c] = acc / A[c * n + c];
  }
  return true;
}

// Inversion of a dual U: the value from the FP64 bracketed inversion; the
// tangent of the root from the implicit-function theorem on p2c(P) = U. With
// J = d(U fluid slots)/d(P fluid slots) at the root (dual numbers, one column
// per primitive) and r = the response of the same slots to the tangents of B
// and of the adiabatic index at fixed fluid primitives,
//   J dP_fluid = dU_fluid - r;   B = U_B / sqrt(-g) directly.
int invert_point(const Dd U[NVAR], const Geo& G, const Dd& gam, Dd P[NVAR]) {
  double u[NVAR], p[NVAR];
  for (int v = 0; v < NVAR; ++v) {
    u[v] = U[v].v;
    p[v] = P[v].v;
  }
  const int flag = cons_to_prim_point(u, G, gam.v, p);
  for (int b = 0; b < 3; ++b) P[B1 + b] = U[B1 + b] / G.gdet;
  if (flag) {
    for (int v = 0; v < 5; ++v) P[v] = Dd(p[v]);
    return flag;
  }
  double J[25];
  Dd Pd[NVAR], Ud[NVAR];
  for (int q = 0; q < 5; ++q) {
    for (int v = 0; v < NVAR; ++v) Pd[v] = mk<double>(p[v], v == q ? 1.0 : 0.0);
    p2c_at<Dd>(G, Pd, Dd(gam.v), Ud);
    for (int f = 0; f < 5; ++f) J[f * 5 + q] = Ud[f].d;
  }
  for (int v = 0; v < NVAR; ++v) Pd[v] = mk<double>(p[v], v >= B1 ? P[v].d : 0.0);
  p2c_at<Dd>(G, Pd, gam, Ud);
  double x[5];
  for (int f = 0; f < 5; ++f) x[f] = U[f].d - Ud[f].d;
  if (!solve_dense(5, J, x))
    for (int f = 0; f < 5; ++f) x[f] = 0.0;
  for (int f = 0; f < 5; ++f) P[f] = mk<double>(p[f], x[f]);
  return 0;
}

int floors_point(const Params& c, const Geo& G, double r, double P[NVAR]) { return apply_floors(c, G, r, P); }

// Floors on a dual state: values as apply_floors; a component that a floor or
// ceiling changed is frozen (it keeps the new value with a zero tangent).
int floors_point(const Params& c, const Geo& G, double r, Dd P[NVAR]) {
  double p[NVAR];
  for (int v = 0; v < NVAR; ++v) p[v] = P[v].v;
  const int flag = apply_floors(c, G, r, p);
  for (int v = 0; v < 5; ++v)
    if (p[v] != P[v].v) P[v] = Dd(p[v]);
  return flag;
}

struct StageStats {
  long nfail = 0, nfloor = 0, nunfixed = 0, nfofc = 0;
};

// First-order flux correction (the paper's "Algorithm" section, after
// Beckwith & Stone 2011), in two parts.
// The trial: the stage's update of every interior zone with the high-order
// fluxes fx, then its inversion and floors; a zone whose trial inversion fails
// or whose trial result a floor or ceiling would change is flagged
// (flag[cell] = 1). Returns the number flagged.
template <class R>
long fofc_trial(const Grid& gr, const R* U0, const R* Pin, const R& gam, double cdt, const FluxesT<R>& fx,
                char* flag) {
  const GridInfo& g = gr.g;
  const double dx[3] = {g.dx1, g.dx2, g.dx3};
  long nflag = 0;
#pragma omp parallel for collapse(2) schedule(static) reduction(+ : nflag)
  for (int k = gr.s3(); k < gr.e3(); ++k)
    for (int j = gr.s2(); j < gr.e2(); ++j)
      for (int i = gr.s1(); i < gr.e1(); ++i) {
        const Geo& G = gr.G(LOC_CENT, j, i);
        R P[NVAR], S[NVAR], U[NVAR];
        for (int v = 0; v < NVAR; ++v) P[v] = Pin[gr.idx(v, k, j, i)];
        source_terms<R>(P, G, gr.C(j, i), gam, S);
        for (int v = 0; v < NVAR; ++v) {
          R div(0.0);
          for (int d = 0; d < g.ndim; ++d) {
            int o1 = d == 0, o2 = d == 1, o3 = d == 2;
            div += (fx.F[d][gr.idx(v, k + o3, j + o2, i + o1)] - fx.F[d][gr.idx(v, k, j, i)]) / dx[d];
          }
          U[v] = U0[gr.idx(v, k, j, i)] + cdt * (-div + S[v]);
        }
        int f = invert_point(U, G, gam, P);
        if (f == 0) f = floors_point(gr.c, G, radius_at(gr, j, i), P);
        if (f) {
          flag[gr.idx(0, k, j, i)] = 1;
          ++nflag;
        }
      }
  return nflag;
}

// The flags' ghost zones follow the ghost map of the state: periodic images
// and outflow and polar copies carry the flag of the interior zone they copy
// (so a face and its periodic image, or an edge's transverse ghost faces, are
// corrected alike); Dirichlet ghosts are not evolved and stay unflagged.
void fill_flag_ghosts(const Grid& gr, char* flag) {
  const GridInfo& g = gr.g;
  const int ng = g.ng;
  auto src_of = [&](int bc, int side, int ig, int n) {
    if (bc == BC_PERIODIC) return side == 0 ? ig + n : ig - n;
    if (bc == BC_OUTFLOW) return side == 0 ? ng : ng + n - 1;
    if (bc == BC_DIRICHLET) return -1;
    return side == 0 ? 2 * ng - 1 - ig : 2 * (ng + n) - 1 - ig;  // polar mirror
  };
  for (int k = gr.s3(); k < gr.e3(); ++k)
    for (int j = gr.s2(); j < gr.e2(); ++j)
      for (int m = 0; m < ng; ++m)
        for (int side = 0; side < 2; ++side) {
          const int ig = side == 0 ? ng - 1 - m : ng + g.n1 + m;
          const int src = src_of(gr.c.bc[side], side, ig, g.n1);
          flag[gr.idx(0, k, j, ig)] = src < 0 ? 0 : flag[gr.idx(0, k, j, src)];
        }
  for (int k = gr.s3(); k < gr.e3(); ++k)
    for (int i = 0; i < g.N1; ++i)
      for (int m = 0; m < ng; ++m)
        for (int side = 0; side < 2; ++side) {
          const int jg = side == 0 ? ng - 1 - m : ng + g.n2 + m;
          const int src = src_of(gr.c.bc[2 + side], side, jg, g.n2);
          flag[gr.idx(0, k, jg, i)] = src < 0 ? 0 : flag[gr.idx(0, k, src, i)];
        }
  if (g.ndim == 3)
    for (int j = 0; j < g.N2; ++j)
      for (int i = 0; i < g.N1; ++i)
        for (int m = 0; m < ng; ++m)
          for (int side = 0; side < 2; ++side) {
            const int kg = side == 0 ? ng - 1 - m : ng + g.n3 + m;
            const int src = src_of(gr.c.bc[4 + side], side, kg, g.n3);
            flag[gr.idx(0, kg, j, i)] = src < 0 ? 0 : flag[gr.idx(0, src, j, i)];
          }
}

// The correction: every face of a flagged zone takes the LLF flux of the
// donor-cell (piecewise constant) states of its two cells in place of the raw
// high-order flux, and polar zeroing and Flux-CT are applied again to the
// corrected raw fluxes (so divB stays as Flux-CT keeps it). raw: the
// high-order raw fluxes; on return fx holds the corrected fluxes. flag_in
// (nullable, every cell, ghosts included): the flags to use instead of this
// grid's own trial and ghost rules (a block of a refined mesh, whose ghost
// flags come from its neighbours). Returns the number of flagged zones.
template <class R>
long fofc_correct(const Grid& gr, const R* U0, const R* Pin, const R& gam, double cdt, FluxesT<R>& raw,
                  FluxesT<R>& fx, const int* flag_in = nullptr) {
  const GridInfo& g = gr.g;
  std::vector<char> flag(gr.cells(), 0);
  long nflag = 0;
  if (flag_in) {
    for (size_t q = 0; q < gr.cells(); ++q) flag[q] = flag_in[q] != 0;
    for (int k = gr.s3(); k < gr.e3(); ++k)
      for (int j = gr.s2(); j < gr.e2(); ++j)
        for (int i = gr.s1(); i < gr.e1(); ++i) nflag += flag[gr.idx(0, k, j, i)];
    bool any = false;
    for (size_t q = 0; q < gr.cells() && !any; ++q) any = flag[q];
    if (!any) return 0;
  } else {
    nflag = fofc_trial(gr, U0, Pin, gam, cdt, fx, flag.data());
    if (nflag == 0) return 0;
    fill_flag_ghosts(gr, flag.data());
  }
  for (int d = 0; d < g.ndim; ++d) {
    int lo[3], hi[3];
    face_range(gr, d, lo, hi);
    const int loc = LOC_FACE1 + d;
    const int o1 = d == 0, o2 = d == 1, o3 = d == 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          if (!flag[gr.idx(0, k, j, i)] && !flag[gr.idx(0, k - o3, j - o2, i - o1)]) continue;
          R PL[NVAR], PR[NVAR], F[NVAR], ct;
          for (int v = 0; v < NVAR; ++v) {
            PL[v] = Pin[gr.idx(v, k - o3, j - o2, i - o1)];
            PR[v] = Pin[gr.idx(v, k, j, i)];
          }
          llf_flux<R>(PL, PR, gr.G(loc, j, i), gam, d + 1, F, ct);
          for (int v = 0; v < NVAR; ++v) raw.F[d][gr.idx(v, k, j, i)] = F[v];
          raw.ctop[d][gr.idx(0, k, j, i)] = val(ct);
        }
  }
  fx = raw;
  finish_fluxes(gr, fx);
  return nflag;
}

// One stage: Pin (ghosts filled) -> fluxes -> Uout = U0 + cdt (-div F + S(Pin))
// -> inversion (guess Pin) -> floors -> fixup. Writes Pout (interior) and Uout
// (interior; consistent with Pout wherever floors or fixups changed Pout).
// R = Dual<double> carries a tangent through the same operations; a zone that
// failed its inversion and was fixed up is frozen (zero tangent).
template <class R>
void stage(const Grid& gr, const R* U0, const R* Pin, const R& gam, double cdt, R* Uout, R* Pout,
           FluxesT<R>& fx, StageStats& st, std::vector<int>* pflag_out, std::vector<int>* fflag_out = nullptr,
           const R* fB0 = nullptr, R* fBout = nullptr, R* dU_out = nullptr, const R* Egiven = nullptr,
           const int* fflag_in = nullptr) {
  const GridInfo& g = gr.g;
  const bool face = gr.c.bfield == BFIELD_FACE;
  if (face) {
    // face-centred CT: the raw fluxes move the fluid; the edge EMFs move the
    // face field, whose cell means become the zones' sqrt(-g) B (Egiven: the
    // edge EMFs supplied by the caller, [3][cells], as a refined mesh
    // corrects them at level interfaces)
    compute_raw(gr, Pin, fx, gam);
    polar_zero(gr, fx);
    std::vector<R> E[3];
    if (Egiven) {
      for (int c = 0; c < 3; ++c) E[c].assign(Egiven + c * gr.cells(), Egiven + (c + 1) * gr.cells());
    } else {
      face_emfs(gr, Pin, fx, E);
    }
    face_update(gr, fB0, E, cdt, fBout);
  } else if (gr.c.fofc) {
    FluxesT<R> raw;
    compute_raw(gr, Pin, raw, gam);
    fx = raw;
    finish_fluxes(gr, fx);
    st.nfofc += fofc_correct(gr, U0, Pin, gam, cdt, raw, fx, fflag_in);
  } else {
    compute_fluxes(gr, Pin, fx, gam);
  }
  std::vector<int> pflag(gr.cells(), 0), fflag(gr.cells(), 0);
  const double dx[3] = {g.dx1, g.dx2, g.dx3};
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = gr.s3(); k < gr.e3(); ++k)
    for (int j = gr.s2(); j < gr.e2(); ++j)
      for (int i = gr.s1(); i < gr.e1(); ++i) {
        const Geo& G = gr.G(LOC_CENT, j, i);
        R P[NVAR], S[NVAR], U[NVAR];
        for (int v = 0; v < NVAR; ++v) P[v] = Pin[gr.idx(v, k, j, i)];
        source_terms<R>(P, G, gr.C(j, i), gam, S);
        for (int v = 0; v < NVAR; ++v) {
          R div(0.0);
          for (int d = 0; d < g.ndim; ++d) {
            int o1 = d == 0, o2 = d == 1, o3 = d == 2;
            div += (fx.F[d][gr.idx(v, k + o3, j + o2, i + o1)] - fx.F[d][gr.idx(v, k, j, i)]) / dx[d];
          }
          const R inc = cdt * (-div + S[v]);
          U[v] = U0[gr.idx(v, k, j, i)] + inc;
          if (dU_out) dU_out[gr.idx(v, k, j, i)] = inc;  // the stage's raw increment (Runge-Kutta)
        }
        if (face) face_to_cell_u(gr, (const R*)fBout, k, j, i, U + B1);
        // guess = stage input
        int flag = invert_point(U, G, gam, P);
        size_t c = gr.idx(0, k, j, i);
        pflag[c] = flag;
        if (flag == 0) {
          fflag[c] = floors_point(gr.c, G, radius_at(gr, j, i), P);
          if (fflag[c]) p2c_at<R>(G, P, gam, U);
        } else {
          for (int v = 0; v < 5; ++v) P[v] = Pin[gr.idx(v, k, j, i)];  // provisional, replaced by fixup
        }
        for (int v = 0; v < NVAR; ++v) {
          Pout[gr.idx(v, k, j, i)] = P[v];
          Uout[gr.idx(v, k, j, i)] = U[v];
        }
      }
  // Fixup: each failed zone takes the equal-weight mean of its non-failed
  // neighbours in the 3x3(x3) block, interior zones only; then floors; then U
  // is recomputed from the repaired primitives.
  std::vector<double> fixed;
  std::vector<size_t> where;
  for (int k = gr.s3(); k < gr.e3(); ++k)
    for (int j = gr.s2(); j < gr.e2(); ++j)
      for (int i = gr.s1(); i < gr.e1(); ++i) {
        size_t c = gr.idx(0, k, j, i);
        if (pflag[c] == 0) continue;
        st.nfail++;
        double sum[5] = {0, 0, 0, 0, 0};
        int cnt = 0;
        int kl = g.ndim == 3 ? -1 : 0, kh = g.ndim == 3 ? 1 : 0;
        for (int dk = kl; dk <= kh; ++dk)
          for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
              if (!dk && !dj && !di) continue;
              int kk = k + dk, jj = j + dj, ii = i + di;
              if (kk < gr.s3() || kk >= gr.e3() || jj < gr.s2() || jj >= gr.e2() || ii < gr.s1() || ii >= gr.e1())
                continue;
              if (pflag[gr.idx(0, kk, jj, ii)] != 0) continue;
              for (int v = 0; v < 5; ++v) sum[v] += val(Pout[gr.idx(v, kk, jj, ii)]);
              ++cnt;
            }
        double P[NVAR];
        for (int v = 0; v < NVAR; ++v) P[v] = val(Pout[gr.idx(v, k, j, i)]);
        if (cnt > 0)
          for (int v = 0; v < 5; ++v) P[v] = sum[v] / cnt;
        else
          st.nunfixed++;
        const Geo& G = gr.G(LOC_CENT, j, i);
        fflag[c] = apply_floors(gr.c, G, radius_at(gr, j, i), P);
        double U[NVAR];
        p2c_point(gr.c, G, P, U);
        for (int v = 0; v < NVAR; ++v) {
          fixed.push_back(P[v]);
          fixed.push_back(U[v]);
        }
        where.push_back(c);
      }
  for (size_t w = 0; w < where.size(); ++w) {
    size_t c = where[w];
    for (int v = 0; v < NVAR; ++v) {
      Pout[c + static_cast<size_t>(v) * gr.cells()] = R(fixed[w * 16 + 2 * v]);
      Uout[c + static_cast<size_t>(v) * gr.cells()] = R(fixed[w * 16 + 2 * v + 1]);
    }
  }
  for (size_t c = 0; c < gr.cells(); ++c)
    if (fflag[c]) st.nfloor++;
  if (pflag_out) *pflag_out = pflag;
  if (fflag_out) *fflag_out = fflag;
}

// CFL time step from the stage fluxes' signal speeds:
// dt = cfl * min_zones 1 / sum_d (ctop_d / dx_d), ctop_d = max over the zone's two x^d faces.
template <class R>
double cfl_dt(const Grid& gr, const FluxesT<R>& fx) {
  const GridInfo& g = gr.g;
  const double dx[3] = {g.dx1, g.dx2, g.dx3};
  double best = std::numeric_limits<double>::infinity();
  for (int k = gr.s3(); k < gr.e3(); ++k)
    for (int j = gr.s2(); j < gr.e2(); ++j)
      for (int i = gr.s1(); i < gr.e1(); ++i) {
        double inv = 0.0;
        for (int d = 0; d < g.ndim; ++d) {
          int o1 = d == 0, o2 = d == 1, o3 = d == 2;
          double c = std::max(fx.ctop[d][gr.idx(0, k, j, i)], fx.ctop[d][gr.idx(0, k + o3, j + o2, i + o1)]);
          inv += c / dx[d];
        }
        double dtz = gr.c.cfl / inv;
        if (dtz < best) best = dtz;
      }
  return best;
}

}  // namespace

// ---------------------------------------------------------------------------
// C API
// ---------------------------------------------------------------------------
extern "C" {

typedef Params or_params;

void or_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int or_get_threads(void) { return omp_get_max_threads(); }

// Geometry at one location over the (N2, N1) grid: gcov, gcon [N2][N1][4][4],
// gdet, alpha [N2][N1].
void or_geometry(const or_params* c, int loc, double* gcov, double* gcon, double* gdet, double* alpha) {
  Grid gr;
  build_grid(*c, gr);
  const GridInfo& g = gr.g;
  for (int j = 0; j < g.N2; ++j)
    for (int i = 0; i < g.N1; ++i) {
      const Geo& G = gr.G(loc, j, i);
      size_t p = static_cast<size_t>(j) * g.N1 + i;
      for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n) {
          gcov[p * 16 + m * 4 + n] = G.gcov[m][n];
          gcon[p * 16 + m * 4 + n] = G.gcon[m][n];
        }
      gdet[p] = G.gdet;
      alpha[p] = G.alpha;
    }
}

// Connection Gamma^l_{mn} at cell centres: [N2][N1][4][4][4].
void or_connection(const or_params* c, double* conn) {
  Grid gr;
  build_grid(*c, gr);
  std::memcpy(conn, gr.conn.data(), gr.conn.size() * sizeof(double));
}

// Metric and connection at arbitrary native points (n points).
void or_metric_points(const or_params* c, int n, const double* x1, const double* x2, double* gcov, double* gcon,
                      double* gdet, double* conn) {
  for (int p = 0; p < n; ++p) {
    Geo G = geo_at(*c, x1[p], x2[p]);
    for (int m = 0; m < 4; ++m)
      for (int q = 0; q < 4; ++q) {
        gcov[p * 16 + m * 4 + q] = G.gcov[m][q];
        gcon[p * 16 + m * 4 + q] = G.gcon[m][q];
      }
    gdet[p] = G.gdet;
    double cn[4][4][4];
    connection_at(*c, x1[p], x2[p], cn);
    std::memcpy(conn + static_cast<size_t>(p) * 64, cn, sizeof(cn));
  }
}

// Native -> Kerr-Schild (r, theta) at n points.
void or_native_to_ks(const or_params* c, int n, const double* x1, const double* x2, double* r, double* th) {
  for (int p = 0; p < n; ++p) native_to_ks<double>(*c, x1[p], x2[p], r[p], th[p]);
}

// P -> U at every cell (ghosts included), cell-centre metric.
void or_prim_to_cons(const or_params* c, const double* P, double* U) {
  Grid gr;
  build_grid(*c, gr);
  const GridInfo& g = gr.g;
#pragma omp parallel for collapse(2)
  for (int k = 0; k < g.N3; ++k)
    for (int j = 0; j < g.N2; ++j)
      for (int i = 0; i < g.N1; ++i) {
        double p[NVAR], u[NVAR];
        for (int v = 0; v < NVAR; ++v) p[v] = P[gr.idx(v, k, j, i)];
        p2c_point(*c, gr.G(LOC_CENT, j, i), p, u);
        for (int v = 0; v < NVAR; ++v) U[gr.idx(v, k, j, i)] = u[v];
      }
}

// U -> P at every cell (ghosts included). P holds the guess on entry. No floors
// and no fixup. pflag (nullable) receives the C2P_* code per cell; returns the
// number of failed cells.
long or_cons_to_prim(const or_params* c, const double* U, double* P, int* pflag) {
  Grid gr;
  build_grid(*c, gr);
  const GridInfo& g = gr.g;
  long nfail = 0;
#pragma omp parallel for collapse(2) reduction(+ : nfail)
  for (int k = 0; k < g.N3; ++k)
    for (int j = 0; j < g.N2; ++j)
      for (int i = 0; i < g.N1; ++i) {
        double p[NVAR], u[NVAR];
        for (int v = 0; v < NVAR; ++v) {
          p[v] = P[gr.idx(v, k, j, i)];
          u[v] = U[gr.idx(v, k, j, i)];
        }
        int f = cons_to_prim_point(u, gr.G(LOC_CENT, j, i), c->gam, p);
        if (f) ++nfail;
        if (pflag) pflag[gr.idx(0, k, j, i)] = f;
        if (f == 0)
          for (int v = 0; v < NVAR; ++v) P[gr.idx(v, k, j, i)] = p[v];
      }
  return nfail;
}

// Boundary fill of P in place. dir_lo/dir_hi: x1 Dirichlet ghosts
// [8][N3][N2][ng] (nullable unless the matching face is Dirichlet).
void or_apply_bc(const or_params* c, double* P, const double* dir_lo, const double* dir_hi) {
  Grid gr;
  build_grid(*c, gr);
  apply_bc(gr, P, dir_lo, dir_hi);
}

// Fluxes (after polar zeroing and Flux-CT) from P with ghosts already filled.
// F1, F2, F3: cell layout [8][N3][N2][N1]; ctop1..3: [N3][N2][N1]. Entries
// outside the computed face ranges are zero.
void or_fluxes(const or_params* c, const double* P, double* F1, double* F2, double* F3, double* ct1, double* ct2,
               double* ct3) {
  Grid gr;
  build_grid(*c, gr);
  Fluxes fx;
  compute_fluxes(gr, P, fx, c->gam);
  double* Fo[3] = {F1, F2, F3};
  double* Co[3] = {ct1, ct2, ct3};
  for (int d = 0; d < 3; ++d) {
    if (Fo[d]) std::memcpy(Fo[d], fx.F[d].data(), fx.F[d].size() * sizeof(double));
    if (Co[d]) std::memcpy(Co[d], fx.ctop[d].data(), fx.ctop[d].size() * sizeof(double));
  }
}

// CFL dt of a state P (ghosts are filled here on a copy), from LLF signal
// speeds at every face of the interior zones.
double or_cfl_dt(const or_params* c, const double* P, const double* dir_lo, const double* dir_hi) {
  Grid gr;
  build_grid(*c, gr);
  std::vector<double> Pc(P, P + gr.cells() * NVAR);
  apply_bc(gr, Pc.data(), dir_lo, dir_hi);
  Fluxes fx;
  compute_fluxes(gr, Pc.data(), fx, c->gam);
  return cfl_dt(gr, fx);
}

// One stage on a grid whose ghost zones the caller has filled (a block of a
// multi-block mesh): fluxes from Pin, Uout = U0 + cdt (-div F + S(Pin)),
// inversion, floors, fixup (interior neighbours only). Uout and Pout: full
// arrays, interior written. ctop1..3 (nullable): signal speeds per face.
// dU (nullable): the raw increment cdt (-div F + S(Pin)) of every interior
// zone (a Runge-Kutta stage whose increment a later stage reuses).
// fofc_flags (nullable; with the first-order flux correction on): the
// flagged zones, every cell of the grid, ghosts included (a refined mesh
// fills a block's ghost flags from its neighbours), used instead of the
// grid's own trial. stats[0..3] as or_step (this stage only).
void or_stage(const or_params* c, const double* U0, const double* Pin, double cdt, double* Uout, double* Pout,
              double* ct1, double* ct2, double* ct3, long* stats, double* dU, const int* fofc_flags) {
  Grid gr;
  build_grid(*c, gr);
  Fluxes fx;
  StageStats st;
  stage<double>(gr, U0, Pin, c->gam, cdt, Uout, Pout, fx, st, nullptr, nullptr, nullptr, nullptr, dU, nullptr,
                fofc_flags);
  double* Co[3] = {ct1, ct2, ct3};
  for (int d = 0; d < 3; ++d)
    if (Co[d]) std::memcpy(Co[d], fx.ctop[d].data(), fx.ctop[d].size() * sizeof(double));
  if (stats) {
    stats[0] = st.nfail;
    stats[1] = st.nfloor;
    stats[2] = st.nunfixed;
    stats[3] = st.nfofc;
  }
}

// One full two-stage step (conserved-synchronised). U (interior) is advanced in
// place; P holds P^n on entry (the stage-1 input and inversion guess) and
// P^{n+1} in the interior on exit. stats[0..3] = failed inversions, floored
// zones, unfixed zones, zones flagged by the first-order flux correction
// (summed over both stages). Returns the next CFL dt.
double or_step_rk(const or_params* c, double* U, double* P, double dt, const double* dir_lo, const double* dir_hi,
                  long* stats);
static double rk_step(const or_params* c, double* U, double* P, double* fB, double dt, const double* dir_lo,
                      const double* dir_hi, long* stats);

double or_step(const or_params* c, double* U, double* P, double dt, const double* dir_lo, const double* dir_hi,
               long* stats) {
  if (c->bfield != BFIELD_FLUXCT) return -1.0;  // the face field is state: or_step_face
  if (c->integrator != INT_VL2) return or_step_rk(c, U, P, dt, dir_lo, dir_hi, stats);
  Grid gr;
  build_grid(*c, gr);
  const size_t n = gr.cells() * NVAR;
  std::vector<double> Pn(P, P + n), U0(U, U + n), Ps(Pn), Us(U0), Pnew, Unew;
  Fluxes fx;
  StageStats st;
  apply_bc(gr, Pn.data(), dir_lo, dir_hi);
  stage<double>(gr, U0.data(), Pn.data(), c->gam, 0.5 * dt, Us.data(), Ps.data(), fx, st, nullptr);
  // ghosts of P* start from those of P^n, then get refilled
  apply_bc(gr, Ps.data(), dir_lo, dir_hi);
  Pnew = Ps;
  Unew = U0;
  stage<double>(gr, U0.data(), Ps.data(), c->gam, dt, Unew.data(), Pnew.data(), fx, st, nullptr);
  double dtn = cfl_dt(gr, fx);
  const GridInfo& g = gr.g;
  for (int v = 0; v < NVAR; ++v)
    for (int k = gr.s3(); k < gr.e3(); ++k)
      for (int j = gr.s2(); j < gr.e2(); ++j)
        for (int i = gr.s1(); i < gr.e1(); ++i) {
          size_t q = gr.idx(v, k, j, i);
          U[q] = Unew[q];
          P[q] = Pnew[q];
        }
  (void)g;
  if (stats) {
    stats[0] = st.nfail;
    stats[1] = st.nfloor;
    stats[2] = st.nunfixed;
    stats[3] = st.nfofc;
  }
  return dtn;
}

// One step of a Runge-Kutta integrator in Shu-Osher form (the paper's
// "Algorithm" section lists RK1, RK2 and SSPRK(5)4 beside the predictor-
// corrector): stage s forms U_s = sum_j a_sj U_j + c_s dt L(P_{s-1}) from the
// stored stage states, where L(P) is the stage operator (fluxes of the
// ghost-filled primitives, Flux-CT, sources) and P_s the inversion of U_s
// (floors, fixup), exactly as a predictor-corrector stage computes them.
//   RK1: U1 = U0 + dt L(P0).
//   RK2 (Heun): U1 = U0 + dt L(P0); U2 = U0/2 + U1/2 + dt/2 L(P1).
//   SSPRK(5,4) of Spiteri & Ruuth (2002): the five stages with their
//   published coefficients; the last stage's dt L(P3) term reuses the raw
//   increment of stage 4, c4 dt L(P3).
// With face-centred CT (fB non-null) the face field is state like U: stage s
// forms its face base sum_j a_sj fB_j and adds c_s dt curl E(P_{s-1}); the
// fifth SSPRK(5,4) stage's face increment is stage 4's output minus stage 4's
// base (c4 dt curl E(P3) up to rounding).
double or_step_rk(const or_params* c, double* U, double* P, double dt, const double* dir_lo, const double* dir_hi,
                  long* stats) {
  return rk_step(c, U, P, nullptr, dt, dir_lo, dir_hi, stats);
}

// The stages of a Runge-Kutta integrator in Shu-Osher form: stage s forms
// sum_t a[t] U_src[t] (+ dU4 times stage 4's raw increment) and adds
// cdt dt L(P_{s-1}).
struct RKStage {
  int n;
  int src[3];
  double a[3];
  double cdt;   // c_s
  double dU4;   // weight of stage 4's raw increment (SSPRK(5,4) stage 5)
};

static std::vector<RKStage> rk_table(int integrator) {
  if (integrator == INT_RK1) return {{1, {0}, {1.0}, 1.0, 0.0}};
  if (integrator == INT_RK2) return {{1, {0}, {1.0}, 1.0, 0.0}, {2, {0, 1}, {0.5, 0.5}, 0.5, 0.0}};
  if (integrator == INT_SSPRK54) {
    const double c4 = 0.544974750228521, c53 = 0.063692468666290;
    return {{1, {0}, {1.0}, 0.391752226571890, 0.0},
            {2, {0, 1}, {0.444370493651235, 0.555629506348765}, 0.368410593050371, 0.0},
            {2, {0, 2}, {0.620101851488403, 0.379898148511597}, 0.251891774271694, 0.0},
            {2, {0, 3}, {0.178079954393132, 0.821920045606868}, c4, 0.0},
            {3, {2, 3, 4}, {0.517231671970585, 0.096059710526147, 0.386708617503269}, 0.226007483236906, c53 / c4}};
  }
  return {};
}

// The table of an integrator for callers that run the stages themselves (a
// refined mesh): per stage s (at most 5), n[s] sources src[3 s + t] with
// weights a[3 s + t], cdt[s] and dU4[s]. Returns the number of stages (0 for
// the predictor-corrector or an unknown integrator).
int or_rk_table(int integrator, int* n, int* src, double* a, double* cdt, double* dU4) {
  const std::vector<RKStage> S = rk_table(integrator);
  for (size_t s = 0; s < S.size(); ++s) {
    n[s] = S[s].n;
    for (int t = 0; t < 3; ++t) {
      src[3 * s + t] = t < S[s].n ? S[s].src[t] : 0;
      a[3 * s + t] = t < S[s].n ? S[s].a[t] : 0.0;
    }
    cdt[s] = S[s].cdt;
    dU4[s] = S[s].dU4;
  }
  return (int)S.size();
}

static double rk_step(const or_params* c, double* U, double* P, double* fB, double dt, const double* dir_lo,
                      const double* dir_hi, long* stats) {
  const std::vector<RKStage> S = rk_table(c->integrator);
  if (S.empty()) return -1.0;
  Grid gr;
  build_grid(*c, gr);
  const size_t n = gr.cells() * NVAR;
  std::vector<std::vector<double>> Us(S.size() + 1), Ps(S.size() + 1);
  Us[0].assign(U, U + n);
  Ps[0].assign(P, P + n);
  std::vector<double> base(n), dU4(n, 0.0), dUs(n, 0.0);
  const bool face = fB != nullptr;
  const size_t nf = face ? 3 * gr.cells() : 0;
  std::vector<std::vector<double>> Fs(S.size() + 1);
  std::vector<double> fbase(nf), fbase4(nf, 0.0);
  if (face) Fs[0].assign(fB, fB + nf);
  Fluxes fx;
  StageStats st;
  for (size_t s = 0; s < S.size(); ++s) {
    const RKStage& q = S[s];
    apply_bc(gr, Ps[s].data(), dir_lo, dir_hi);
    for (size_t e = 0; e < n; ++e) {
      double b = 0.0;
      for (int t = 0; t < q.n; ++t) b += q.a[t] * Us[q.src[t]][e];
      if (q.dU4 != 0.0) b += q.dU4 * dU4[e];
      base[e] = b;
    }
    Us[s + 1] = base;
    Ps[s + 1] = Ps[s];
    if (face) {
      for (size_t e = 0; e < nf; ++e) {
        double b = 0.0;
        for (int t = 0; t < q.n; ++t) b += q.a[t] * Fs[q.src[t]][e];
        if (q.dU4 != 0.0) b += q.dU4 * (Fs[4][e] - fbase4[e]);
        fbase[e] = b;
      }
      Fs[s + 1] = fbase;
    }
    const bool keep = c->integrator == INT_SSPRK54 && s == 3;
    stage<double>(gr, base.data(), Ps[s].data(), c->gam, q.cdt * dt, Us[s + 1].data(), Ps[s + 1].data(), fx, st,
                  nullptr, nullptr, face ? fbase.data() : nullptr, face ? Fs[s + 1].data() : nullptr,
                  keep ? dU4.data() : nullptr);
    if (face && keep) fbase4 = fbase;
  }
  if (face) std::memcpy(fB, Fs[S.size()].data(), nf * sizeof(double));
  const double dtn = cfl_dt(gr, fx);
  const size_t last = S.size();
  for (int v = 0; v < NVAR; ++v)
    for (int k = gr.s3(); k < gr.e3(); ++k)
      for (int j = gr.s2(); j < gr.e2(); ++j)
        for (int i = gr.s1(); i < gr.e1(); ++i) {
          const size_t e = gr.idx(v, k, j, i);
          U[e] = Us[last][e];
          P[e] = Ps[last][e];
        }
  (void)dUs;
  if (stats) {
    stats[0] = st.nfail;
    stats[1] = st.nfloor;
    stats[2] = st.nunfixed;
    stats[3] = st.nfofc;
  }
  return dtn;
}

// One step with face-centred constrained transport: as or_step, with the
// face field fB ([3][N3][N2][N1], sqrt(-g) B^(a+1) on the lower x^(a+1) face
// of each cell) advanced by the edge EMFs of each stage and the zones'
// sqrt(-g) B taken as its cell means. Faces of the interior cells are
// updated; other entries are kept. Returns the next dt, or -1 for a
// configuration it does not run (Flux-CT, or with the flux correction).
double or_step_face(const or_params* c, double* U, double* P, double* fB, double dt, const double* dir_lo,
                    const double* dir_hi, long* stats) {
  if (c->bfield != BFIELD_FACE || c->fofc) return -1.0;
  if (c->integrator != INT_VL2) return rk_step(c, U, P, fB, dt, dir_lo, dir_hi, stats);
  Grid gr;
  build_grid(*c, gr);
  const size_t n = gr.cells() * NVAR;
  std::vector<double> Pn(P, P + n), U0(U, U + n), Ps(Pn), Us(U0), Pnew, Unew;
  std::vector<double> fB0(fB, fB + 3 * gr.cells()), fBs(fB0), fBn(fB0);
  Fluxes fx;
  StageStats st;
  apply_bc(gr, Pn.data(), dir_lo, dir_hi);
  stage<double>(gr, U0.data(), Pn.data(), c->gam, 0.5 * dt, Us.data(), Ps.data(), fx, st, nullptr, nullptr,
                fB0.data(), fBs.data());
  apply_bc(gr, Ps.data(), dir_lo, dir_hi);
  Pnew = Ps;
  Unew = U0;
  stage<double>(gr, U0.data(), Ps.data(), c->gam, dt, Unew.data(), Pnew.data(), fx, st, nullptr, nullptr,
                fB0.data(), fBn.data());
  const double dtn = cfl_dt(gr, fx);
  for (int v = 0; v < NVAR; ++v)
    for (int k = gr.s3(); k < gr.e3(); ++k)
      for (int j = gr.s2(); j < gr.e2(); ++j)
        for (int i = gr.s1(); i < gr.e1(); ++i) {
          size_t q = gr.idx(v, k, j, i);
          U[q] = Unew[q];
          P[q] = Pnew[q];
        }
  std::memcpy(fB, fBn.data(), fBn.size() * sizeof(double));
  if (stats) {
    stats[0] = st.nfail;
    stats[1] = st.nfloor;
    stats[2] = st.nunfixed;
    stats[3] = st.nfofc;
  }
  return dtn;
}

// The edge EMFs of face-centred CT from a ghost-filled state ([3][cells],
// entries the interior faces need; others 0).
void or_face_emfs(const or_params* c, const double* Pin, double* E) {
  Grid gr;
  build_grid(*c, gr);
  Fluxes fx;
  compute_raw(gr, Pin, fx, c->gam);
  polar_zero(gr, fx);
  std::vector<double> Ev[3];
  face_emfs(gr, Pin, fx, Ev);
  for (int q = 0; q < 3; ++q) std::memcpy(E + q * gr.cells(), Ev[q].data(), gr.cells() * sizeof(double));
}

// One face-CT stage on a grid with caller-filled ghosts and caller-supplied
// edge EMFs E ([3][cells]): fBout = fB0 + cdt curl E on the interior cells'
// faces, then the zone update as or_stage with the zones' field from the new
// faces. ctop as or_stage.
void or_stage_face(const or_params* c, const double* U0, const double* Pin, double cdt, const double* E,
                   const double* fB0, double* fBout, double* Uout, double* Pout, double* ct1, double* ct2, double* ct3,
                   long* stats) {
  Grid gr;
  build_grid(*c, gr);
  Fluxes fx;
  StageStats st;
  stage<double>(gr, U0, Pin, c->gam, cdt, Uout, Pout, fx, st, nullptr, nullptr, fB0, fBout, nullptr, E);
  double* Co[3] = {ct1, ct2, ct3};
  for (int d = 0; d < 3; ++d)
    if (Co[d]) std::memcpy(Co[d], fx.ctop[d].data(), fx.ctop[d].size() * sizeof(double));
  if (stats) {
    stats[0] = st.nfail;
    stats[1] = st.nfloor;
    stats[2] = st.nunfixed;
    stats[3] = st.nfofc;
  }
}

// Face divergence of a face field: per interior cell sum_a (fB_a(upper) -
// fB_a(lower)) / dx_a (x1, x2 only on a 2-D grid); out = {max |div|, mean
// |div|}; div (nullable) gets the per-cell values.
void or_face_divb(const or_params* c, const double* fB, double* out, double* div) {
  Grid gr;
  build_grid(*c, gr);
  const GridInfo& g = gr.g;
  const double dx[3] = {g.dx1, g.dx2, g.dx3};
  double mx = 0.0, sum = 0.0;
  long cnt = 0;
  for (int k = gr.s3(); k < gr.e3(); ++k)
    for (int j = gr.s2(); j < gr.e2(); ++j)
      for (int i = gr.s1(); i < gr.e1(); ++i) {
        double d = (fB[gr.idx(0, k, j, i + 1)] - fB[gr.idx(0, k, j, i)]) / dx[0] +
                   (fB[gr.idx(1, k, j + 1, i)] - fB[gr.idx(1, k, j, i)]) / dx[1];
        if (g.ndim == 3) d += (fB[gr.idx(2, k + 1, j, i)] - fB[gr.idx(2, k, j, i)]) / dx[2];
        if (div) div[gr.idx(0, k, j, i)] = d;
        mx = std::max(mx, std::fabs(d));
        sum += std::fabs(d);
        ++cnt;
      }
  out[0] = mx;
  out[1] = cnt ? sum / cnt : 0.0;
}

// Cell-centred B^i of the interior cells from a face field (the face means
// over sqrt(-g) at the cell centre), written into P's field slots.
void or_face_to_cell(const or_params* c, const double* fB, double* P) {
  Grid gr;
  build_grid(*c, gr);
  for (int k = gr.s3(); k < gr.e3(); ++k)
    for (int j = gr.s2(); j < gr.e2(); ++j)
      for (int i = gr.s1(); i < gr.e1(); ++i) {
        double UB[3];
        face_to_cell_u<double>(gr, fB, k, j, i, UB);
        const double gd = gr.G(LOC_CENT, j, i).gdet;
        for (int b = 0; b < 3; ++b) P[gr.idx(B1 + b, k, j, i)] = UB[b] / gd;
      }
}

// The zones the first-order flux correction flags in one stage from the
// ghost-filled stage input Pin and U0 (cdt = c dt): flags [N3][N2][N1], 1 for
// a flagged interior zone. Returns their number.
long or_fofc_flags(const or_params* c, const double* U0, const double* Pin, double cdt, int* flags) {
  Grid gr;
  build_grid(*c, gr);
  Fluxes fx;
  compute_fluxes(gr, Pin, fx, c->gam);
  std::vector<char> flag(gr.cells(), 0);
  const long n = fofc_trial(gr, U0, Pin, c->gam, cdt, fx, flag.data());
  for (size_t q = 0; q < gr.cells(); ++q) flags[q] = flag[q];
  return n;
}

// Tangent of one step (forward-mode dual numbers through the same stages):
// U, P advance exactly as in or_step (same values); dU, dP (same layouts)
// and dgam carry a direction on entry, and on exit dU, dP hold the
// directional derivative of U^{n+1}, P^{n+1} (interior; dt held fixed).
// Derivative rules at the non-smooth points: the branch the values take
// (MC: slope 0 when the one-sided differences do not agree in sign, the
// first candidate on ties; ctop: the first of the maximal speeds), the
// implicit-function derivative of the inversion, floored components and
// fixed-up zones frozen, Dirichlet ghosts and clamped inflow constant.
// dF1 (nullable): the tangent of the stage-2 x1 fluxes, cell layout.
// zflag (nullable, [N3][N2][N1]): per zone, bit 1 = an inversion failed
// (either stage; the zone was fixed up), bit 2 = a floor or ceiling acted.
// stats as or_step. Returns the next CFL dt.
double or_step_jvp(const or_params* c, double* U, double* P, double* dU, double* dP, double dgam, double dt,
                   const double* dir_lo, const double* dir_hi, double* dF1, int* zflag, long* stats) {
  Grid gr;
  build_grid(*c, gr);
  const size_t n = gr.cells() * NVAR;
  std::vector<Dd> Pn(n), U0(n);
  for (size_t q = 0; q < n; ++q) {
    Pn[q] = mk<double>(P[q], dP[q]);
    U0[q] = mk<double>(U[q], dU[q]);
  }
  const Dd gam = mk<double>(c->gam, dgam);
  std::vector<Dd> Ps(Pn), Us(U0), Pnew, Unew;
  FluxesT<Dd> fx;
  StageStats st;
  std::vector<int> pf[2], ff[2];
  apply_bc(gr, Pn.data(), dir_lo, dir_hi);
  stage<Dd>(gr, U0.data(), Pn.data(), gam, 0.5 * dt, Us.data(), Ps.data(), fx, st, &pf[0], &ff[0]);
  apply_bc(gr, Ps.data(), dir_lo, dir_hi);
  Pnew = Ps;
  Unew = U0;
  stage<Dd>(gr, U0.data(), Ps.data(), gam, dt, Unew.data(), Pnew.data(), fx, st, &pf[1], &ff[1]);
  double dtn = cfl_dt(gr, fx);
  if (zflag)
    for (size_t q = 0; q < gr.cells(); ++q)
      zflag[q] = ((pf[0][q] || pf[1][q]) ? 1 : 0) | ((ff[0][q] || ff[1][q]) ? 2 : 0);
  for (int v = 0; v < NVAR; ++v)
    for (int k = gr.s3(); k < gr.e3(); ++k)
      for (int j = gr.s2(); j < gr.e2(); ++j)
        for (int i = gr.s1(); i < gr.e1(); ++i) {
          size_t q = gr.idx(v, k, j, i);
          U[q] = Unew[q].v;
          P[q] = Pnew[q].v;
          dU[q] = Unew[q].d;
          dP[q] = Pnew[q].d;
        }
  if (dF1)
    for (size_t q = 0; q < n; ++q) dF1[q] = fx.F[0][q].d;
  if (stats) {
    stats[0] = st.nfail;
    stats[1] = st.nfloor;
    stats[2] = st.nunfixed;
    stats[3] = st.nfofc;
  }
  return dtn;
}

// Run nsteps steps with a fixed dt (dt > 0) or with the CFL dt of the previous
// step (dt <= 0: the first step uses -dt, or the CFL dt of P if dt == 0),
// stopping at time t_end when t_end > 0 (the last step is clipped to land on it).
// Returns the time advanced. stats as or_step, accumulated.
double or_evolve(const or_params* c, double* U, double* P, int nsteps, double dt, double t_end, const double* dir_lo,
                 const double* dir_hi, long* stats) {
  double t = 0.0;
  double dtc = dt > 0.0 ? dt : -dt;
  long acc[4] = {0, 0, 0, 0};
  for (int s = 0; s < nsteps || (t_end > 0.0 && nsteps <= 0); ++s) {
    double step_dt = dtc;
    if (t_end > 0.0) {
      if (t >= t_end * (1.0 - 1e-14)) break;
      if (t + step_dt > t_end) step_dt = t_end - t;
    }
    long st[4];
    double next = or_step(c, U, P, step_dt, dir_lo, dir_hi, st);
    for (int q = 0; q < 4; ++q) acc[q] += st[q];
    t += step_dt;
    if (dt <= 0.0) dtc = next;
  }
  if (stats)
    for (int q = 0; q < 4; ++q) stats[q] = acc[q];
  return t;
}

// divB of sqrt(-g) B at the corners whose adjacent cells are all interior
// (Flux-CT's conserved corner divergence). out[0] = max |divB|, out[1] = mean
// |divB|; optional field div (cell layout [N3][N2][N1], corner (i-1/2,j-1/2,
// k-1/2) stored at (k,j,i), zero elsewhere).
void or_divb(const or_params* c, const double* P, double* out, double* div) {
  Grid gr;
  build_grid(*c, gr);
  const GridInfo& g = gr.g;
  const double dx[3] = {g.dx1, g.dx2, g.dx3};
  auto gB = [&](int d, int k, int j, int i) { return gr.G(LOC_CENT, j, i).gdet * P[gr.idx(B1 + d, k, j, i)]; };
  double mx = 0.0, sum = 0.0;
  long cnt = 0;
  if (div) std::memset(div, 0, gr.cells() * sizeof(double));
  int kl = g.ndim == 3 ? gr.s3() + 1 : 0, kh = g.ndim == 3 ? gr.e3() - 1 : 0;
  for (int k = kl; k <= kh; ++k)
    for (int j = gr.s2() + 1; j <= gr.e2() - 1; ++j)
      for (int i = gr.s1() + 1; i <= gr.e1() - 1; ++i) {
        double dv = 0.0;
        if (g.ndim == 2) {
          dv += (gB(0, k, j, i) + gB(0, k, j - 1, i) - gB(0, k, j, i - 1) - gB(0, k, j - 1, i - 1)) / (2.0 * dx[0]);
          dv += (gB(1, k, j, i) + gB(1, k, j, i - 1) - gB(1, k, j - 1, i) - gB(1, k, j - 1, i - 1)) / (2.0 * dx[1]);
        } else {
          double s1p = gB(0, k, j, i) + gB(0, k, j - 1, i) + gB(0, k - 1, j, i) + gB(0, k - 1, j - 1, i);
          double s1m = gB(0, k, j, i - 1) + gB(0, k, j - 1, i - 1) + gB(0, k - 1, j, i - 1) + gB(0, k - 1, j - 1, i - 1);
          double s2p = gB(1, k, j, i) + gB(1, k, j, i - 1) + gB(1, k - 1, j, i) + gB(1, k - 1, j, i - 1);
          double s2m = gB(1, k, j - 1, i) + gB(1, k, j - 1, i - 1) + gB(1, k - 1, j - 1, i) + gB(1, k - 1, j - 1, i - 1);
          double s3p = gB(2, k, j, i) + gB(2, k, j, i - 1) + gB(2, k, j - 1, i) + gB(2, k, j - 1, i - 1);
          double s3m = gB(2, k - 1, j, i) + gB(2, k - 1, j, i - 1) + gB(2, k - 1, j - 1, i) + gB(2, k - 1, j - 1, i - 1);
          dv = (s1p - s1m) / (4.0 * dx[0]) + (s2p - s2m) / (4.0 * dx[1]) + (s3p - s3m) / (4.0 * dx[2]);
        }
        if (div) div[gr.idx(0, k, j, i)] = dv;
        mx = std::max(mx, std::fabs(dv));
        sum += std::fabs(dv);
        ++cnt;
      }
  out[0] = mx;
  out[1] = cnt ? sum / cnt : 0.0;
}

// ---- point-level entry points for the pin tests ----

// Conserved U and the flux F^dir of one state at a given covariant metric.
void or_point_flux(double gam, const double* gcov16, const double* P, int dir, double* F) {
  Geo G;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) G.gcov[m][n] = gcov16[m * 4 + n];
  geo_from_gcov(G);
  FluidState<double> S;
  fluid_state(P, G, S);
  prim_to_flux<double>(P, S, G, gam, dir, F);
}

// u^mu, b^mu, b^2 of one state: out[0..3] ucon, out[4..7] bcon, out[8] bsq.
void or_point_state(const double* gcov16, const double* P, double* out) {
  Geo G;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) G.gcov[m][n] = gcov16[m * 4 + n];
  geo_from_gcov(G);
  FluidState<double> S;
  fluid_state(P, G, S);
  for (int m = 0; m < 4; ++m) {
    out[m] = S.ucon[m];
    out[4 + m] = S.bcon[m];
  }
  out[8] = S.bsq;
}

void or_point_speeds(double gam, const double* gcov16, const double* P, int dir, double* cmax, double* cmin) {
  Geo G;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) G.gcov[m][n] = gcov16[m * 4 + n];
  geo_from_gcov(G);
  FluidState<double> S;
  fluid_state(P, G, S);
  signal_speeds<double>(P, S, G, gam, dir, *cmax, *cmin);
}

void or_point_llf(double gam, const double* gcov16, const double* PL, const double* PR, int dir, double* F,
                  double* ctop) {
  Geo G;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) G.gcov[m][n] = gcov16[m * 4 + n];
  geo_from_gcov(G);
  llf_flux<double>(PL, PR, G, gam, dir, F, *ctop);
}

// Single-point inversion at a given metric; P: guess in, result out.
int or_point_c2p(double gam, const double* gcov16, const double* U, double* P) {
  Geo G;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) G.gcov[m][n] = gcov16[m * 4 + n];
  geo_from_gcov(G);
  return cons_to_prim_point(U, G, gam, P);
}

// Jacobians dF^dir/dP and dU/dP (8x8, row = output slot, column = primitive)
// of one state, by forward-mode differentiation.
void or_point_jacobians(double gam, const double* gcov16, const double* P, int dir, double* dF, double* dU) {
  Geo G;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) G.gcov[m][n] = gcov16[m * 4 + n];
  geo_from_gcov(G);
  for (int col = 0; col < NVAR; ++col) {
    Dual<double> Pd[NVAR];
    for (int v = 0; v < NVAR; ++v) Pd[v] = mk<double>(P[v], v == col ? 1.0 : 0.0);
    FluidState<Dual<double>> S;
    fluid_state(Pd, G, S);
    Dual<double> F[NVAR], U[NVAR];
    prim_to_flux(Pd, S, G, gam, dir, F);
    prim_to_flux(Pd, S, G, gam, 0, U);
    for (int r = 0; r < NVAR; ++r) {
      dF[r * NVAR + col] = F[r].d;
      dU[r * NVAR + col] = U[r].d;
    }
  }
}

// Floating-point operations of the method's per-item formulas, counted by
// running the oracle's own templated point physics on the counting type at
// one state (the counts do not depend on the values except through the
// clamps and branches the state takes): out[0] one WENO5 face value, out[1]
// one MC reconstruction of a cell (slope and both face values), out[2] the
// LLF flux of one face from its two states (two fluid states, four flux and
// conserved vectors, two speed pairs, the LLF combination), out[3] the
// connection source terms of one zone, out[4] the conserved variables of
// one zone from its primitives. P: 8 primitives; the metric is that of the
// cell centre at native (x1, x2).
void or_count_ops(const or_params* c, double x1, double x2, const double* P, double* out) {
  Geo G = geo_at(*c, x1, x2);
  double cn[4][4][4];
  connection_at(*c, x1, x2, cn);
  OpCounts& k = op_counts();
  // a monotone stencil: MC takes its full path (a nonzero slope)
  Cnt q[5] = {Cnt(P[0]), Cnt(1.1 * P[0]), Cnt(1.25 * P[0]), Cnt(1.3 * P[0]), Cnt(1.5 * P[0])};
  k = OpCounts();
  (void)weno5_upper<Cnt>(q);
  out[0] = (double)k.total();
  k = OpCounts();
  Cnt lo, hi;
  recon_cell<Cnt>(RECON_MC, q, lo, hi);
  out[1] = (double)k.total();
  Cnt Pc[NVAR], Pr[NVAR], F[NVAR], S[NVAR], U[NVAR], ct;
  for (int v = 0; v < NVAR; ++v) {
    Pc[v] = Cnt(P[v]);
    Pr[v] = Cnt(P[v] * (1.0 + 0.01 * (v + 1)));
  }
  const Cnt gam(c->gam);
  k = OpCounts();
  llf_flux<Cnt, Cnt>(Pc, Pr, G, gam, 1, F, ct);
  out[2] = (double)k.total();
  k = OpCounts();
  source_terms<Cnt, Cnt>(Pc, G, cn, gam, S);
  out[3] = (double)k.total();
  k = OpCounts();
  p2c_at<Cnt>(G, Pc, gam, U);
  out[4] = (double)k.total();
}

// Source terms of one state at a cell centre of the grid (j, i).
void or_point_source(const or_params* c, double x1, double x2, const double* P, double* S) {
  Geo G = geo_at(*c, x1, x2);
  double cn[4][4][4];
  connection_at(*c, x1, x2, cn);
  source_terms<double>(P, G, cn, c->gam, S);
}

// Floors of one state at native (x1, x2) (the radius as the grid's floors
// take it: r of the Kerr-Schild family, 1 in Minkowski). P: 8 primitives,
// floored in place; returns the floor bit mask of apply_floors.
int or_point_floors(const or_params* c, double x1, double x2, double* P) {
  Geo G = geo_at(*c, x1, x2);
  double r = 1.0, th = 0.0;
  if (c->kind != MINKOWSKI) native_to_ks<double>(*c, x1, x2, r, th);
  return apply_floors(*c, G, r, P);
}

// 1-D reconstruction of q[0..n-1]: lo[i], hi[i] = lower/upper face values of
// cell i for 2 <= i < n-2 (others untouched).
void or_recon(int recon, int n, const double* q, double* lo, double* hi) {
  for (int i = 2; i < n - 2; ++i) recon_cell(recon, q + i - 2, lo[i], hi[i]);
}

}  // extern "C"
