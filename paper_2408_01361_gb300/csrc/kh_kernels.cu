// Kernels of the FP64 HARM step on sm_103a (arXiv 2408.01361, "Algorithm"
// section) and their host launchers:
//   geometry cache, ghost fill, reconstruction + LLF fluxes, Flux-CT EMFs,
//   update + sources + Noble-2D inversion + floors, fixup, CFL reduction,
//   corner divB, and the stand-alone prim->cons / cons->prim kernels.
//
// Layout: structure of arrays [var][k][j][i] with padded rows; the thread
// index runs fastest along i so a warp reads consecutive doubles of a row.
// Every device loop has a fixed bound; no kernel waits on another.
#include "kh_zone.cuh"

namespace kh {

namespace {

constexpr int TPB = 128;    // default threads per block
constexpr int TPB_MAX = 256;


inline int nblocks(long long n, int tpb) { return (int)((n + tpb - 1) / tpb); }

// ---------------------------------------------------------------------------
// Geometry cache: one thread per (j, i) of the allocation. Metric, inverse,
// sqrt(-g), lapse at CENT, x1 face and x2 face; connection and r at CENT.
// ---------------------------------------------------------------------------
__global__ void k_geometry(CoordParams cp, double x1o, double x2o, FloorParams fl, Layout L, double* geo,
                           double* dgm, double* flo) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= L.gplane) return;
  const int i = (int)(p % L.n1s), j = (int)(p / L.n1s);
  const double x1c = x1o + (i - L.ng + 0.5) * L.dx[0];
  const double x1f = x1o + (i - L.ng) * L.dx[0];
  const double x2c = x2o + (j - L.ng + 0.5) * L.dx[1];
  const double x2f = x2o + (j - L.ng) * L.dx[1];
  for (int loc = 0; loc < 3; ++loc) {
    const double x1 = (loc == LOC_F1) ? x1f : x1c;
    const double x2 = (loc == LOC_F2) ? x2f : x2c;
    double g[4][4], gi[4][4], dg[4][4][4];
    native_metric(cp, x1, x2, g, loc == LOC_CENT ? dg : nullptr);
    const double det = inverse4_cofactor(g, gi);
    double* b = geo + (long long)loc * NGEO * L.gplane + p;
    for (int m = 0; m < 4; ++m)
      for (int n = m; n < 4; ++n) {
        b[sym_index(m, n) * L.gplane] = g[m][n];
        b[(10 + sym_index(m, n)) * L.gplane] = gi[m][n];
      }
    b[20 * L.gplane] = sqrt(fabs(det));
    b[21 * L.gplane] = 1.0 / sqrt(-gi[0][0]);
    if (loc == LOC_CENT) {
      // d_1 g_{mn}, d_2 g_{mn} (the metric does not depend on t or phi)
      for (int a = 1; a <= 2; ++a)
        for (int m = 0; m < 4; ++m)
          for (int n = m; n < 4; ++n) dgm[((a - 1) * 10 + sym_index(m, n)) * L.gplane + p] = dg[a][m][n];
      const double r = (cp.kind == COORD_MINKOWSKI) ? 1.0 : coord_map(cp, x1c, x2c).r;
      flo[p] = fmax(fl.rho_min * pow(r, -1.5), 1e-20);
      flo[L.gplane + p] = fmax(fl.u_min * pow(r, -2.5), 1e-20);
      flo[2 * L.gplane + p] = 1.0 / sqrt(fabs(det));
    }
  }
}

// ---------------------------------------------------------------------------
// Ghost fill of the 8 primitive slots. x1 ghosts over interior (j, k); x2
// ghosts over all i and interior k; x3 ghosts over all (i, j): edges and
// corners are compositions of the face rules (three launches, in order).
// ---------------------------------------------------------------------------
// One pass over every ghost cell: the x1 rule, then the x2 rule, then the x3
// rule (the order of the per-direction passes, in which a later direction's
// ghosts copy cells that an earlier direction filled) composed into one map
// from the ghost cell to an interior cell (or to the x1 Dirichlet data at the
// mapped (j, k)), with the per-component operations of the rules crossed on
// the way: u~1 clamped by an x1 outflow face (no inflow), u~2 and B2 negated
// by a polar x2 face. The two act on different components, so their order
// does not matter. Reads interior cells of src only and writes ghost cells of
// dst, so src == dst is allowed. Ghost cells are enumerated in three slabs:
// x1 ghosts of interior (j, k), x2 ghosts of interior k, x3 ghosts.

// Number of ghost cells in the three slabs.
__device__ __forceinline__ long long ghost_total(const Layout& L) {
  const long long nj = L.e[1] - L.s[1], nk = L.e[2] - L.s[2];
  const long long T1 = nj * nk * L.ng * 2, T2 = (long long)L.N1 * nk * L.ng * 2;
  const long long T3 = L.ndim == 3 ? (long long)L.N1 * L.N2 * L.ng3 * 2 : 0;
  return T1 + T2 + T3;
}

// Ghost cell number t (< ghost_total) -> (i, j, k).
__device__ __forceinline__ void ghost_cell(const Layout& L, long long t, int& i, int& j, int& k) {
  const long long nj = L.e[1] - L.s[1], nk = L.e[2] - L.s[2];
  const long long T1 = nj * nk * L.ng * 2, T2 = (long long)L.N1 * nk * L.ng * 2;
  if (t < T1) {
    const int side = (int)(t % 2), m = (int)((t / 2) % L.ng);
    j = L.s[1] + (int)((t / (2 * L.ng)) % nj);
    k = L.s[2] + (int)(t / (2LL * L.ng * nj));
    i = side == 0 ? L.ng - 1 - m : L.ng + L.n1 + m;
  } else if (t < T1 + T2) {
    const long long u = t - T1;
    i = (int)(u % L.N1);
    const int side = (int)((u / L.N1) % 2), m = (int)((u / (2LL * L.N1)) % L.ng);
    k = L.s[2] + (int)(u / (2LL * L.N1 * L.ng));
    j = side == 0 ? L.ng - 1 - m : L.ng + L.n2 + m;
  } else {
    const long long u = t - T1 - T2;
    i = (int)(u % L.N1);
    j = (int)((u / L.N1) % L.N2);
    const int side = (int)((u / ((long long)L.N1 * L.N2)) % 2), m = (int)(u / (2LL * L.N1 * L.N2));
    k = side == 0 ? L.ng3 - 1 - m : L.ng3 + L.n3 + m;
  }
}

// The composed ghost map of cell (i, j, k): its source cell (is, js, ks), or
// for dir != 0 (1: inner, 2: outer x1 Dirichlet face) the index (ks, js, is)
// into that face's ghost data; flip: u~2 and B2 change sign (polar x2 face);
// clamp 1: u~1 <= 0 (inner x1 outflow), 2: u~1 >= 0 (outer).
struct GhostSrc {
  int i, j, k;
  int dir, clamp;
  bool flip;
};

__device__ __forceinline__ GhostSrc ghost_source(const Layout& L, const Scheme& S, int i, int j, int k) {
  GhostSrc g{i, j, k, 0, 0, false};
  if (L.ndim == 3 && (k < L.s[2] || k >= L.e[2])) {
    const int side = k < L.s[2] ? 0 : 1;
    if (S.bc[4 + side] == KH_BC_PERIODIC) g.k = side == 0 ? k + L.n3 : k - L.n3;
    else g.k = side == 0 ? L.s[2] : L.e[2] - 1;
  }
  if (j < L.s[1] || j >= L.e[1]) {
    const int side = j < L.s[1] ? 0 : 1, bc = S.bc[2 + side];
    if (bc == KH_BC_PERIODIC) g.j = side == 0 ? j + L.n2 : j - L.n2;
    else if (bc == KH_BC_OUTFLOW) g.j = side == 0 ? L.ng : L.ng + L.n2 - 1;
    else g.j = side == 0 ? 2 * L.ng - 1 - j : 2 * (L.ng + L.n2) - 1 - j;
    g.flip = bc == KH_BC_POLAR;
  }
  if (i < L.s[0] || i >= L.e[0]) {
    const int side = i < L.s[0] ? 0 : 1, bc = S.bc[side];
    if (bc == KH_BC_DIRICHLET) {
      g.dir = side + 1;
      g.i = side == 0 ? i : i - (L.ng + L.n1);  // index into the ghost data
    } else if (bc == KH_BC_PERIODIC) {
      g.i = side == 0 ? i + L.n1 : i - L.n1;
    } else if (bc == KH_BC_OUTFLOW) {
      g.i = side == 0 ? L.ng : L.ng + L.n1 - 1;
      g.clamp = side + 1;
    } else {
      g.i = side == 0 ? 2 * L.ng - 1 - i : 2 * (L.ng + L.n1) - 1 - i;
    }
  }
  return g;
}

template <class TS, class TD>
__device__ __forceinline__ void bc_cell(const CVarsT<TS>& src, const VarsT<TD>& dst, const Layout& L, const Scheme& S,
                                        const TS* dlo, const TS* dhi, int i, int j, int k) {
  const GhostSrc g = ghost_source(L, S, i, j, k);
  const int ks = g.k, js = g.j, is = g.i, clamp = g.clamp;
  const bool flip = g.flip;
  const TS* D = g.dir == 1 ? dlo : (g.dir == 2 ? dhi : nullptr);
  if (KH_OOB(L, kh_in(L, i, j, k, 0) && (D != nullptr || kh_in(L, is, js, ks, 0)))) return;
  const long long d = L.at(k, j, i), sc = D ? 0 : L.at(ks, js, is);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    TS x = D ? D[(((long long)v * L.n3s + ks) * L.n2s + js) * L.ng + is] : src.v[v][sc];
    if (v == V_U1 && ((clamp == 1 && x > TS(0)) || (clamp == 2 && x < TS(0)))) x = TS(0);
    if (flip && (v == V_U2 || v == V_B2)) x = -x;
    if constexpr (sizeof(TS) == sizeof(TD)) dst.v[v][d] = x;
    else dst.v[v][d] = f32_of_f64(x);  // integer operations, not the FP64 pipe
  }
}

template <class TS, class TD>
__global__ void k_bc_fill(CVarsT<TS> src, VarsT<TD> dst, Layout L, Scheme S, const TS* dlo, const TS* dhi) {
  pdl_wait();
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ghost_total(L)) return;
  int i, j, k;
  ghost_cell(L, t, i, j, k);
  bc_cell<TS, TD>(src, dst, L, S, dlo, dhi, i, j, k);
}

// The FP32 copy of an FP64 state in one pass over the ghosted box (row
// padding skipped): interior cells converted, ghost cells by the ghost map
// from the FP64 interior (the mixed path's stage-1 input).
__global__ void k_fill_f32(CVarsT<double> src, VarsT<float> dst, Layout L, Scheme S, const double* dlo,
                           const double* dhi) {
  pdl_wait();
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)L.N1 * L.N2 * L.N3) return;
  int i, j, k;
  split3(t, L.N1, L.N2, i, j, k);
  if (KH_OOB(L, kh_in(L, i, j, k, 0))) return;
  if (i >= L.s[0] && i < L.e[0] && j >= L.s[1] && j < L.e[1] && k >= L.s[2] && k < L.e[2]) {
    const long long c = L.at(k, j, i);
    // all eight loads first (in flight together), then the conversions
    // (integer ops, not the FP64 pipe) and stores
    double q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = src.v[v][c];
#pragma unroll
    for (int v = 0; v < NV; ++v) dst.v[v][c] = f32_of_f64(q[v]);
  } else {
    bc_cell<double, float>(src, dst, L, S, dlo, dhi, i, j, k);
  }
}


// ---------------------------------------------------------------------------
// Reconstruction + LLF flux through the lower x^D face of cell (k, j, i),
// over the interior faces plus one transverse row on each side (Flux-CT).
// ---------------------------------------------------------------------------
template <int D, int RECON, class TIN, class R>
__global__ void __launch_bounds__(TPB_MAX) k_flux(CVarsT<TIN> P, Layout L, GeomT<R> G, Scheme S, FaceBox box, R* F,
                                                 R* ctop, int polar_lo, int polar_hi) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned tot = (unsigned)box.n[0] * box.n[1] * box.n[2];
  if (t >= tot) return;
  int i, j, k;
  split3(t, box.n[0], box.n[1], i, j, k);
  if (KH_OOB(L, kh_in_dir(L, D, i + box.lo[0], j + box.lo[1], k + box.lo[2], -3, 2))) return;
  flux_face<D, RECON, TIN, R>(P, L, G, S, i + box.lo[0], j + box.lo[1], k + box.lo[2], F, ctop, polar_lo, polar_hi);
}

// Corner EMFs of Flux-CT (Toth 2000) from the LLF field fluxes:
//   e3(i-1/2, j-1/2) = (F1_B2(j) + F1_B2(j-1) - F2_B1(i) - F2_B1(i-1)) / 4 and
//   cyclic e1 (x1-edges), e2 (x2-edges) in 3-D.
template <class R>
__global__ void k_emf(const R* F1, const R* F2, const R* F3, R* e1, R* e2, R* e3, Layout L) {
  pdl_wait();
  const int n0 = L.e[0] - L.s[0] + 1, n1 = L.e[1] - L.s[1] + 1, n2 = (L.ndim == 3) ? L.e[2] - L.s[2] + 1 : 1;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)n0 * n1 * n2) return;
  int i, j, k;
  split3(t, n0, n1, i, j, k);
  {
    const int ii = i + L.s[0], jj = j + L.s[1], kk = k + (L.ndim == 3 ? L.s[2] : 0);
    if (KH_OOB(L, kh_in(L, ii, jj, kk, 0) && kh_in(L, ii - 1, jj - 1, L.ndim == 3 ? kk - 1 : kk, 0))) return;
  }
  emf_at<R>(F1, F2, F3, e1, e2, e3, L, i + L.s[0], j + L.s[1], k + (L.ndim == 3 ? L.s[2] : 0));
}

template <class R>
__global__ void k_apply_ct(R* F1, R* F2, R* F3, const R* e1, const R* e2, const R* e3, Layout L) {
  const int n0 = L.e[0] - L.s[0] + 1, n1 = L.e[1] - L.s[1] + 1, n2 = (L.ndim == 3) ? L.e[2] - L.s[2] + 1 : 1;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)n0 * n1 * n2) return;
  int i, j, k;
  split3(t, n0, n1, i, j, k);
  apply_ct_at<R>(F1, F2, F3, e1, e2, e3, L, i + L.s[0], j + L.s[1], k + (L.ndim == 3 ? L.s[2] : 0));
}

// ---------------------------------------------------------------------------
// Update of one interior zone: U = U0 + cdt (-div F + S(Pin)), inversion with
// Pin as the guess, floors; writes Pout, pflag and (stage 2) U.
// ---------------------------------------------------------------------------

template <int INV>
__global__ void __launch_bounds__(TPB_MAX) k_update(const double* U0, CVars Pin, Vars Pout, double* Uout,
                                                   const double* F1, const double* F2, const double* F3, Layout L,
                                                   DevGeom G, Scheme S, const double* dtp, double coef, int8_t* pflag,
                                                   unsigned long long* cnt, FailList fl, const double* fBn,
                                                   double* dUout) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nzones(L)) return;
  int i, j, k;
  zone_ijk(L, t, i, j, k);
  if (KH_OOB(L, kh_in(L, i, j, k, 1))) return;
  update_zone<false, INV>(U0, Pin, Pout, Uout, F1, F2, F3, L, G, S, coef * __ldg(dtp), pflag, cnt, i, j, k, nullptr,
                          fl, fBn, dUout);
}

// out = sum_t a_t in_t over n values (Runge-Kutta stage bases; up to 4 terms).
struct LinComb {
  const double* in[4];
  double a[4];
  int n;
};
__global__ void k_lincomb(double* out, LinComb lc, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    double s = lc.a[0] * lc.in[0][q];
    for (int t = 1; t < lc.n; ++t) s += lc.a[t] * lc.in[t][q];
    out[q] = s;
  }
}

// four blocks of TPB_MAX per SM: 64 registers (the unconstrained kernel takes
// ~220; the spills go to L1). Measured on GB300 (192x96x96 torus, per launch):
// 300 us at 4 blocks, 308 us at 3 (80 registers), 334 us at 2 (128).
template <int INV>
__global__ void __launch_bounds__(TPB_MAX, 4) k_update_mixed(const double* U0, CVarsT<float> Pin, Vars Pout64,
                                                         VarsT<float> Pout32, double* Uout, const float* F1,
                                                         const float* F2, const float* F3, Layout L, DevGeom G,
                                                         GeomT<float> Gf, Scheme S, const double* dtp, double coef,
                                                         int8_t* pflag, unsigned long long* cnt, FailList fl,
                                                         const double* fBn, double* dUout, CtEmf ect) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nzones(L)) return;
  int i, j, k;
  zone_ijk(L, t, i, j, k);
  if (KH_OOB(L, kh_in(L, i, j, k, 1))) return;
  update_mixed_zone<false, INV>(U0, Pin, Pout64, Pout32, Uout, F1, F2, F3, L, G, Gf, S, df_of_f64(coef * __ldg(dtp)),
                                pflag, cnt, i, j, k, fl, fBn, dUout, ect);
}

template <class T>
__global__ void __launch_bounds__(TPB) k_fixup(VarsT<T> P, double* Uout, const int8_t* pflag, Layout L, DevGeom G,
                                              Scheme S, unsigned long long* cnt) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nzones(L)) return;
  int i, j, k;
  zone_ijk(L, t, i, j, k);
  if (KH_OOB(L, kh_in(L, i, j, k, 1))) return;
  fixup_zone<T>(P, Uout, pflag, L, G, S, cnt, i, j, k);
}

// The same over the stage's failed-zone list (its length read on the
// device), one warp per failed zone (fixup_warp).
template <class T>
__global__ void __launch_bounds__(TPB) k_fixup_list(VarsT<T> P, double* Uout, const int8_t* pflag, Layout L,
                                                   DevGeom G, Scheme S, unsigned long long* cnt, FailList fl) {
  pdl_wait();
  const unsigned long long n = *fl.n;
  const long long gs = L.gplane;
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long q = warp; q < n; q += nwarps) {
    const long long c = fl.idx[q];
    const int k = (int)(c / gs), j = (int)((c % gs) / L.n1s), i = (int)(c % L.n1s);
#ifdef KH_BOUNDS_CHECK
    if (!kh_in(L, i, j, k, 1)) {  // c is the warp's: the whole warp skips it, lane 0 counts it
      if (lane == 0 && L.oob) atomicAdd(L.oob, 1ULL);
      continue;
    }
#endif
    fixup_warp<T>(P, Uout, pflag, L, G, S, cnt, i, j, k, lane);
  }
}

// ---------------------------------------------------------------------------
// First-order flux correction (the paper's "Algorithm" section, after
// Beckwith & Stone 2011): trial flags, their ghosts, donor-cell face fluxes.
// ---------------------------------------------------------------------------
template <int INV>
__global__ void __launch_bounds__(TPB_MAX) k_fofc_trial(const double* U0, CVars Pin, const double* F1,
                                                       const double* F2, const double* F3, Layout L, DevGeom G,
                                                       Scheme S, const double* dtp, double coef, int8_t* flag,
                                                       unsigned long long* cnt) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nzones(L)) return;
  int i, j, k;
  zone_ijk(L, t, i, j, k);
  update_zone<true, INV>(U0, Pin, Vars{}, nullptr, F1, F2, F3, L, G, S, coef * __ldg(dtp), flag, cnt, i, j, k);
}

template <int INV>
__global__ void __launch_bounds__(TPB_MAX, 3) k_fofc_trial_mixed(const double* U0, CVarsT<float> Pin,
                                                                const float* F1, const float* F2, const float* F3,
                                                                Layout L, DevGeom G, GeomT<float> Gf, Scheme S,
                                                                const double* dtp, double coef, int8_t* flag,
                                                                unsigned long long* cnt, CtEmf ect) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nzones(L)) return;
  int i, j, k;
  zone_ijk(L, t, i, j, k);
  update_mixed_zone<true, INV>(U0, Pin, Vars{}, VarsT<float>{}, nullptr, F1, F2, F3, L, G, Gf, S,
                          df_of_f64(coef * __ldg(dtp)), flag, cnt, i, j, k, FailList{nullptr, nullptr, 0u}, nullptr,
                          nullptr, ect);
}

// Ghost flags follow the state's ghost map: a periodic image or an outflow or
// polar copy carries its source zone's flag; Dirichlet ghosts are not evolved.
__global__ void k_flag_ghosts(int8_t* flag, Layout L, Scheme S) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ghost_total(L)) return;
  int i, j, k;
  ghost_cell(L, t, i, j, k);
  const GhostSrc g = ghost_source(L, S, i, j, k);
  flag[L.at(k, j, i)] = g.dir ? 0 : flag[L.at(g.k, g.j, g.i)];
}

// The raw flux of every face of the box that borders a flagged cell becomes
// the LLF flux of the two cells' own (donor-cell) states.
template <int D, class TIN, class R>
__global__ void __launch_bounds__(TPB_MAX) k_fofc_faces(CVarsT<TIN> P, Layout L, GeomT<R> G, Scheme S, FaceBox box,
                                                       const int8_t* flag, R* F, R* ctop, int polar_lo,
                                                       int polar_hi) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned tot = (unsigned)box.n[0] * box.n[1] * box.n[2];
  if (t >= tot) return;
  int i, j, k;
  split3(t, box.n[0], box.n[1], i, j, k);
  i += box.lo[0];
  j += box.lo[1];
  k += box.lo[2];
  const long long c = L.at(k, j, i);
  const long long st = (D == 1) ? 1 : (D == 2 ? (long long)L.n1s : (long long)L.n1s * L.n2s);
  if (!(flag[c] | flag[c - st])) return;
  flux_face<D, RECON_DONOR, TIN, R>(P, L, G, S, i, j, k, F, ctop, polar_lo, polar_hi);
}

// ---------------------------------------------------------------------------
// Face-centred constrained transport: cell EMFs, edge EMFs, face update.
// ---------------------------------------------------------------------------
// Active-direction extents of the box [s - lo_pad, e] (inactive x3: one cell).
__device__ __forceinline__ void box_dims(const Layout& L, int pad, int n[3], int lo[3]) {
  for (int q = 0; q < 3; ++q) {
    const bool active = q < 2 || L.ndim == 3;
    lo[q] = active ? L.s[q] - pad : 0;
    n[q] = active ? L.e[q] - L.s[q] + 1 + pad : 1;
  }
}

// Cell-centred EMFs of the cells [s-1, e] along every active direction.
template <class R>
__global__ void __launch_bounds__(TPB) k_cell_emf(CVarsT<R> P, Layout L, GeomT<R> G, R* ecc) {
  int n[3], lo[3];
  box_dims(L, 1, n, lo);
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)n[0] * n[1] * n[2]) return;
  int i, j, k;
  split3(t, n[0], n[1], i, j, k);
  i += lo[0];
  j += lo[1];
  k += lo[2];
  const long long c = L.at(k, j, i);
  R Pc[NV], E[3];
#pragma unroll
  for (int v = 0; v < NV; ++v) Pc[v] = P.v[v][c];
  const Met<R> m = load_met(G, L.gplane, LOC_CENT, (long long)j * L.n1s + i);
  cell_emfs(Pc, m, E);
#pragma unroll
  for (int q = 0; q < 3; ++q) ecc[q * L.plane + c] = E[q];
}

// Edge EMFs of the edges the interior faces need (box [s, e]; along its own
// direction an edge stays inside [s, e)); zero on a polar axis.
template <class R>
__global__ void __launch_bounds__(TPB) k_face_emf(const R* F1, const R* F2, const R* F3, const R* ecc, R* e1, R* e2,
                                                 R* e3, Layout L, Scheme S, int emf) {
  int n[3], lo[3];
  box_dims(L, 0, n, lo);
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)n[0] * n[1] * n[2]) return;
  int i, j, k;
  split3(t, n[0], n[1], i, j, k);
  i += lo[0];
  j += lo[1];
  k += lo[2];
  const long long c = L.at(k, j, i);
  const R* F[3] = {F1, F2, F3};
  const bool axis = (S.bc[2] == KH_BC_POLAR && j == L.s[1]) || (S.bc[3] == KH_BC_POLAR && j == L.e[1]);
  if (L.ndim == 3) {
    if (k < L.e[2]) e3[c] = axis ? R(0) : edge_emf<R>(2, F, ecc, L, emf, i, j, k);
    if (i < L.e[0]) e1[c] = axis ? R(0) : edge_emf<R>(0, F, ecc, L, emf, i, j, k);
    if (j < L.e[1]) e2[c] = edge_emf<R>(1, F, ecc, L, emf, i, j, k);
  } else {
    // no x3 variation: E1 is the x2-face value F^2(B^3), E2 minus the x1-face value F^1(B^3)
    e3[c] = axis ? R(0) : edge_emf<R>(2, F, ecc, L, emf, i, j, k);
    if (i < L.e[0]) e1[c] = axis ? R(0) : F2[V_B3 * L.plane + c];
    if (j < L.e[1]) e2[c] = -F1[V_B3 * L.plane + c];
  }
}

// fBout = fB0 + c dt (d_b E_c - d_c E_b) on every face of the interior cells
// (box [s, e]: a face family keeps index e only along its normal). The curl
// is formed in FP64 also from FP32 EMFs (converted exactly, by integer
// operations): the face divergence of the increments then cancels to FP64
// rounding, as on the FP64 path (an FP32 curl would leave FP32-sized
// divergence each step). A few FP64 operations per face.
template <class R>
__global__ void __launch_bounds__(TPB) k_face_update(const double* fB0, double* fBout, const R* e1, const R* e2,
                                                    const R* e3, Layout L, const double* dtp, double coef) {
  int n[3], lo[3];
  box_dims(L, 0, n, lo);
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)n[0] * n[1] * n[2]) return;
  int x[3];
  split3(t, n[0], n[1], x[0], x[1], x[2]);
  for (int q = 0; q < 3; ++q) x[q] += lo[q];
  const long long c = L.at(x[2], x[1], x[0]);
  const long long st[3] = {1, (long long)L.n1s, (long long)L.n1s * L.n2s};
  const R* E[3] = {e1, e2, e3};
  const double cdt = coef * __ldg(dtp);
  const int nd = L.ndim;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, cc = (a + 2) % 3;
    bool in = true;
    for (int q = 0; q < nd; ++q)
      if (q != a && x[q] >= L.e[q]) in = false;
    if (!in) continue;
    auto f64 = [](R v) -> double {
      if constexpr (sizeof(R) == sizeof(double)) return v;
      else return f64_of_f32(v);
    };
    double rhs = 0.0;
    if (b < nd) rhs += (f64(E[cc][c + st[b]]) - f64(E[cc][c])) * L.idx[b];
    if (cc < nd) rhs -= (f64(E[b][c + st[cc]]) - f64(E[b][c])) * L.idx[cc];
    fBout[a * L.plane + c] = fB0[a * L.plane + c] + cdt * rhs;
  }
}

// Face divergence of the interior cells (max |div|, sum |div|) per block.
__global__ void __launch_bounds__(RED_THREADS) k_face_divb(const double* fB, Layout L, double* partial);

// B of the interior cells = face means / sqrt(-g).
__global__ void __launch_bounds__(TPB) k_face_to_cell(const double* fB, double* B, Layout L, DevGeom G) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nzones(L)) return;
  int i, j, k;
  zone_ijk(L, t, i, j, k);
  const long long c = L.at(k, j, i);
  double UB[3];
  face_means(fB, L, c, UB);
  const double gd = __ldg(G.g + (long long)LOC_CENT * NGEO * L.gplane + 20 * L.gplane + (long long)j * L.n1s + i);
#pragma unroll
  for (int q = 0; q < 3; ++q) B[q * L.plane + c] = UB[q] / gd;
}

// ---------------------------------------------------------------------------
// Reductions: warp shuffles, then shared memory, then one block over partials.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block-wide (max a, sum b) with RED_THREADS threads.
__device__ __forceinline__ void block_max_sum(double& a, double& b) {
  __shared__ double sa[RED_THREADS / 32], sb[RED_THREADS / 32];
  a = warp_max(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  if (w == 0) {
    a = (l < RED_THREADS / 32) ? sa[l] : 0.0;
    b = (l < RED_THREADS / 32) ? sb[l] : 0.0;
    a = warp_max(a);
    b = warp_sum(b);
  }
}

// CFL: inv = sum_d max(ctop_d(lower face), ctop_d(upper face)) / dx_d per zone;
// the grid-wide maximum gives dt = cfl / max(inv) = min over zones of cfl / inv.
template <class T>
__global__ void __launch_bounds__(RED_THREADS) k_cfl(const T* c1, const T* c2, const T* c3, Layout L,
                                                    double* partial) {
  pdl_wait();
  const unsigned nz = nzones(L);
  T m = T(0);  // per-thread maximum in the speeds' precision
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < nz; t += gridDim.x * blockDim.x) {
    int i, j, k;
    zone_ijk(L, t, i, j, k);
    if (KH_OOB(L, kh_in(L, i, j, k, 1))) continue;
    const T v = cfl_inv_zone(c1, c2, c3, L, i, j, k);
    m = v > m ? v : m;
  }
  double mx = (double)m, dummy = 0.0;
  block_max_sum(mx, dummy);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = mx;
    partial[2 * blockIdx.x + 1] = 0.0;
  }
}

__global__ void k_finish(const double* partial, int n, double cfl, int mode, double* out) {
  pdl_wait();
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    a = fmax(a, partial[2 * q]);
    b += partial[2 * q + 1];
  }
  block_max_sum(a, b);
  if (threadIdx.x == 0) {
    if (mode == 0) {
      out[0] = cfl / a;
    } else {
      out[0] = a;
      out[1] = b;
    }
  }
}

// Corner divB of sqrt(-g) B at corners whose adjacent cells are all interior.
__global__ void __launch_bounds__(RED_THREADS) k_divb(const double* B1, const double* B2, const double* B3,
                                                     Layout L, DevGeom G, double* partial) {
  const int n0 = L.e[0] - L.s[0] - 1, n1 = L.e[1] - L.s[1] - 1;
  const int n2 = L.ndim == 3 ? L.e[2] - L.s[2] - 1 : 1;
  const long long tot = (long long)(n0 > 0 ? n0 : 0) * (n1 > 0 ? n1 : 0) * (n2 > 0 ? n2 : 0);
  const double* gd = G.g + (long long)LOC_CENT * NGEO * L.gplane + 20 * L.gplane;
  double mx = 0.0, sm = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int i = L.s[0] + 1 + (int)(t % n0);
    const int j = L.s[1] + 1 + (int)((t / n0) % n1);
    const int k = (L.ndim == 3 ? L.s[2] + 1 : 0) + (int)(t / ((long long)n0 * n1));
    const double dv = divb_corner(B1, B2, B3, L, gd, i, j, k);
    mx = fmax(mx, fabs(dv));
    sm += fabs(dv);
  }
  block_max_sum(mx, sm);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = mx;
    partial[2 * blockIdx.x + 1] = sm;
  }
}

__global__ void __launch_bounds__(RED_THREADS) k_face_divb(const double* fB, Layout L, double* partial) {
  const long long tot = nzones(L);
  const long long P = L.plane, sj = L.n1s, sk = (long long)L.n1s * L.n2s;
  double mx = 0.0, sm = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    zone_ijk(L, (unsigned)t, i, j, k);
    const long long c = L.at(k, j, i);
    double d = (fB[c + 1] - fB[c]) * L.idx[0] + (fB[P + c + sj] - fB[P + c]) * L.idx[1];
    if (L.ndim == 3) d += (fB[2 * P + c + sk] - fB[2 * P + c]) * L.idx[2];
    mx = fmax(mx, fabs(d));
    sm += fabs(d);
  }
  block_max_sum(mx, sm);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = mx;
    partial[2 * blockIdx.x + 1] = sm;
  }
}

// Stand-alone P -> U and U -> P over every cell of the allocation's ghosted box.
__global__ void __launch_bounds__(TPB) k_p2c(CVars P, double* U, Layout L, DevGeom G, Scheme S) {
  const long long tot = (long long)L.N1 * L.N2 * L.N3;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= tot) return;
  const int i = (int)(t % L.N1), j = (int)((t / L.N1) % L.N2), k = (int)(t / ((long long)L.N1 * L.N2));
  const long long c = L.at(k, j, i);
  const Met<double> m = load_met(G, L.gplane, LOC_CENT, (long long)j * L.n1s + i);
  double p[NV], u[NV];
  for (int v = 0; v < NV; ++v) p[v] = P.v[v][c];
  FState<double> s;
  fluid_state(p, m, s);
  cons_only(p, s, m, S.gam, u);
  for (int v = 0; v < NV; ++v) U[v * L.plane + c] = u[v];
}

template <int INV>
__global__ void __launch_bounds__(TPB) k_c2p(const double* U, Vars P, int8_t* pflag, Layout L, DevGeom G, Scheme S,
                                            unsigned long long* cnt) {
  const long long tot = (long long)L.N1 * L.N2 * L.N3;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= tot) return;
  const int i = (int)(t % L.N1), j = (int)((t / L.N1) % L.N2), k = (int)(t / ((long long)L.N1 * L.N2));
  const long long c = L.at(k, j, i);
  const Met<double> m = load_met(G, L.gplane, LOC_CENT, (long long)j * L.n1s + i);
  double u[NV], p[NV];
  for (int v = 0; v < NV; ++v) {
    u[v] = U[v * L.plane + c];
    p[v] = P.v[v][c];
  }
  const double ig = __ldg(G.flo + 2 * L.gplane + (long long)j * L.n1s + i);  // 1 / sqrt(-g)
  const int flag = invert<INV>(u, m, ig, S.gam, S.igam, S.gfac, S.c2p, p);
  p[V_B1] = u[V_B1] * ig;
  p[V_B2] = u[V_B2] * ig;
  p[V_B3] = u[V_B3] * ig;
  for (int v = 0; v < NV; ++v) P.v[v][c] = p[v];
  if (pflag) pflag[c] = (int8_t)flag;
  if (flag) atomicAdd(cnt + CNT_FAIL, 1ULL);
}

__global__ void k_to_f32(const double* src, float* dst, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    dst[q] = (float)src[q];
}

__global__ void k_vars_to_f32(CVars src, VarsT<float> dst, long long plane) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < plane;
       q += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int v = 0; v < NV; ++v) dst.v[v][q] = f32_of_f64(src.v[v][q]);  // integer ops, not the FP64 pipe
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
int reduction_blocks(const Layout& L) {
  long long nz = (long long)L.n1 * L.n2 * L.n3;
  long long b = (nz + RED_THREADS - 1) / RED_THREADS;
  if (b > 152 * 8) b = 152 * 8;
  return b < 1 ? 1 : (int)b;
}

int launch_geometry(const CoordParams& cp, double x1o, double x2o, const FloorParams& fl, const Layout& L, double* geo,
                    double* dgm, double* flo, cudaStream_t s) {
  k_geometry<<<nblocks(L.gplane, TPB), TPB, 0, s>>>(cp, x1o, x2o, fl, L, geo, dgm, flo);
  return 1;
}

template <class T>
int launch_bc(const VarsT<T>& P, const Layout& L, const Scheme& S, const T* dlo, const T* dhi, cudaStream_t s) {
  return launch_bc_fill<T, T>(cviewT(P), P, L, S, dlo, dhi, s);
}

template <class TS, class TD>
int launch_bc_fill(const CVarsT<TS>& src, const VarsT<TD>& dst, const Layout& L, const Scheme& S, const TS* dlo,
                   const TS* dhi, cudaStream_t s) {
  const long long nj = L.e[1] - L.s[1], nk = L.e[2] - L.s[2];
  const long long tot = nj * nk * L.ng * 2 + (long long)L.N1 * nk * L.ng * 2 +
                        (L.ndim == 3 ? (long long)L.N1 * L.N2 * L.ng3 * 2 : 0);
  launch_pdl(k_bc_fill<TS, TD>, dim3((unsigned)nblocks(tot, TPB)), dim3(TPB), 0, s, src, dst, L, S, dlo, dhi);
  return 1;
}
template int launch_bc_fill<double, float>(const CVarsT<double>&, const VarsT<float>&, const Layout&, const Scheme&,
                                           const double*, const double*, cudaStream_t);
template int launch_bc<double>(const VarsT<double>&, const Layout&, const Scheme&, const double*, const double*,
                               cudaStream_t);
template int launch_bc<float>(const VarsT<float>&, const Layout&, const Scheme&, const float*, const float*,
                              cudaStream_t);

template <int D, class TIN, class R>
static int launch_flux_d(const CVarsT<TIN>& P, const Layout& L, const GeomT<R>& G, const Scheme& S, R* F, R* ctop,
                         int tpb, cudaStream_t s) {
  const FaceBox b = face_box(L, D);
  const long long tot = (long long)b.n[0] * b.n[1] * b.n[2];
  const int plo = S.bc[2] == KH_BC_POLAR, phi = S.bc[3] == KH_BC_POLAR;
  if (S.recon == KH_RECON_MC)
    k_flux<D, KH_RECON_MC, TIN, R><<<nblocks(tot, tpb), tpb, 0, s>>>(P, L, G, S, b, F, ctop, plo, phi);
  else
    k_flux<D, KH_RECON_WENO5, TIN, R><<<nblocks(tot, tpb), tpb, 0, s>>>(P, L, G, S, b, F, ctop, plo, phi);
  return 1;
}

template <class TIN, class R>
int launch_flux_dir(int D, const CVarsT<TIN>& P, const Layout& L, const GeomT<R>& G, const Scheme& S, R* F, R* ctop,
                    int tpb, cudaStream_t s) {
  if (D == 1) return launch_flux_d<1>(P, L, G, S, F, ctop, tpb, s);
  if (D == 2) return launch_flux_d<2>(P, L, G, S, F, ctop, tpb, s);
  return launch_flux_d<3>(P, L, G, S, F, ctop, tpb, s);
}
template int launch_flux_dir<double, double>(int, const CVarsT<double>&, const Layout&, const GeomT<double>&,
                                             const Scheme&, double*, double*, int, cudaStream_t);
template int launch_flux_dir<double, float>(int, const CVarsT<double>&, const Layout&, const GeomT<float>&,
                                            const Scheme&, float*, float*, int, cudaStream_t);
template int launch_flux_dir<float, float>(int, const CVarsT<float>&, const Layout&, const GeomT<float>&,
                                           const Scheme&, float*, float*, int, cudaStream_t);

int launch_fofc_trial(const double* U0, const CVars& Pin, double* const F[3], const Layout& L, const DevGeom& G,
                      const Scheme& S, const double* dtp, double coef, int8_t* flag, unsigned long long* cnt,
                      int tpb, cudaStream_t s) {
  const long long nz = (long long)L.n1 * L.n2 * L.n3;
  if (S.c2p.method == C2P_KASTAUN)
    k_fofc_trial<C2P_KASTAUN><<<nblocks(nz, tpb), tpb, 0, s>>>(U0, Pin, F[0], F[1], F[2], L, G, S, dtp, coef, flag,
                                                               cnt);
  else if (S.c2p.method == C2P_1DW)
    k_fofc_trial<C2P_1DW><<<nblocks(nz, tpb), tpb, 0, s>>>(U0, Pin, F[0], F[1], F[2], L, G, S, dtp, coef, flag, cnt);
  else
    k_fofc_trial<C2P_NOBLE2D><<<nblocks(nz, tpb), tpb, 0, s>>>(U0, Pin, F[0], F[1], F[2], L, G, S, dtp, coef, flag,
                                                               cnt);
  return 1;
}

int launch_fofc_trial_mixed(const double* U0, const CVarsT<float>& Pin, float* const F[3], const Layout& L,
                            const DevGeom& G, const GeomT<float>& Gf, const Scheme& S, const double* dtp, double coef,
                            int8_t* flag, unsigned long long* cnt, int tpb, cudaStream_t s, float* const* emf) {
  const long long nz = (long long)L.n1 * L.n2 * L.n3;
  const CtEmf ect{{emf ? emf[0] : nullptr, emf ? emf[1] : nullptr, emf ? emf[2] : nullptr}};
  auto go = [&](auto kern) {
    kern<<<nblocks(nz, tpb), tpb, 0, s>>>(U0, Pin, F[0], F[1], F[2], L, G, Gf, S, dtp, coef, flag, cnt, ect);
  };
  if (S.c2p.method == C2P_KASTAUN) go(k_fofc_trial_mixed<C2P_KASTAUN>);
  else if (S.c2p.method == C2P_1DW) go(k_fofc_trial_mixed<C2P_1DW>);
  else if (S.mixed_fp64) go(k_fofc_trial_mixed<C2P_NOBLE2D_FP64>);
  else go(k_fofc_trial_mixed<C2P_NOBLE2D>);
  return 1;
}

int launch_flag_ghosts(int8_t* flag, const Layout& L, const Scheme& S, cudaStream_t s) {
  const long long nj = L.e[1] - L.s[1], nk = L.e[2] - L.s[2];
  const long long tot = nj * nk * L.ng * 2 + (long long)L.N1 * nk * L.ng * 2 +
                        (L.ndim == 3 ? (long long)L.N1 * L.N2 * L.ng3 * 2 : 0);
  k_flag_ghosts<<<nblocks(tot, TPB), TPB, 0, s>>>(flag, L, S);
  return 1;
}

template <int D, class TIN, class R>
static int launch_fofc_d(const CVarsT<TIN>& P, const Layout& L, const GeomT<R>& G, const Scheme& S,
                         const int8_t* flag, R* F, R* ctop, int tpb, cudaStream_t s) {
  const FaceBox b = face_box(L, D);
  const long long tot = (long long)b.n[0] * b.n[1] * b.n[2];
  const int plo = S.bc[2] == KH_BC_POLAR, phi = S.bc[3] == KH_BC_POLAR;
  k_fofc_faces<D, TIN, R><<<nblocks(tot, tpb), tpb, 0, s>>>(P, L, G, S, b, flag, F, ctop, plo, phi);
  return 1;
}

template <class TIN, class R>
int launch_fofc_faces(int D, const CVarsT<TIN>& P, const Layout& L, const GeomT<R>& G, const Scheme& S,
                      const int8_t* flag, R* F, R* ctop, int tpb, cudaStream_t s) {
  if (D == 1) return launch_fofc_d<1>(P, L, G, S, flag, F, ctop, tpb, s);
  if (D == 2) return launch_fofc_d<2>(P, L, G, S, flag, F, ctop, tpb, s);
  return launch_fofc_d<3>(P, L, G, S, flag, F, ctop, tpb, s);
}
template int launch_fofc_faces<double, double>(int, const CVarsT<double>&, const Layout&, const GeomT<double>&,
                                               const Scheme&, const int8_t*, double*, double*, int, cudaStream_t);
template int launch_fofc_faces<float, float>(int, const CVarsT<float>&, const Layout&, const GeomT<float>&,
                                             const Scheme&, const int8_t*, float*, float*, int, cudaStream_t);

template <class R> int launch_ct(R* const F[3], R* const emf[3], const Layout& L, cudaStream_t s) {
  const long long tot = (long long)(L.e[0] - L.s[0] + 1) * (L.e[1] - L.s[1] + 1) * (L.ndim == 3 ? L.e[2] - L.s[2] + 1 : 1);
  k_emf<R><<<nblocks(tot, TPB), TPB, 0, s>>>(F[0], F[1], F[2], emf[0], emf[1], emf[2], L);
  k_apply_ct<R><<<nblocks(tot, TPB), TPB, 0, s>>>(F[0], F[1], F[2], emf[0], emf[1], emf[2], L);
  return 2;
}
template <class R> int launch_emf(R* const F[3], R* const emf[3], const Layout& L, cudaStream_t s) {
  const long long tot = (long long)(L.e[0] - L.s[0] + 1) * (L.e[1] - L.s[1] + 1) * (L.ndim == 3 ? L.e[2] - L.s[2] + 1 : 1);
  launch_pdl(k_emf<R>, dim3((unsigned)nblocks(tot, TPB)), dim3(TPB), 0, s, F[0], F[1], F[2], emf[0], emf[1], emf[2], L);
  return 1;
}
template int launch_emf<float>(float* const[3], float* const[3], const Layout&, cudaStream_t);
template int launch_ct<double>(double* const[3], double* const[3], const Layout&, cudaStream_t);
template int launch_ct<float>(float* const[3], float* const[3], const Layout&, cudaStream_t);

int launch_update(const double* U0, const CVars& Pin, const Vars& Pout, double* Uout, double* const F[3],
                  const Layout& L, const DevGeom& G, const Scheme& S, const double* dtp, double coef, int8_t* pflag,
                  unsigned long long* cnt, int tpb, cudaStream_t s, FailList fl, const double* fBn,
                  double* dUout) {
  const long long nz = (long long)L.n1 * L.n2 * L.n3;
  if (S.c2p.method == C2P_KASTAUN)
    k_update<C2P_KASTAUN><<<nblocks(nz, tpb), tpb, 0, s>>>(U0, Pin, Pout, Uout, F[0], F[1], F[2], L, G, S, dtp, coef,
                                                           pflag, cnt, fl, fBn, dUout);
  else if (S.c2p.method == C2P_1DW)
    k_update<C2P_1DW><<<nblocks(nz, tpb), tpb, 0, s>>>(U0, Pin, Pout, Uout, F[0], F[1], F[2], L, G, S, dtp, coef,
                                                       pflag, cnt, fl, fBn, dUout);
  else
    k_update<C2P_NOBLE2D><<<nblocks(nz, tpb), tpb, 0, s>>>(U0, Pin, Pout, Uout, F[0], F[1], F[2], L, G, S, dtp, coef,
                                                           pflag, cnt, fl, fBn, dUout);
  return 1;
}

int launch_update_mixed(const double* U0, const CVarsT<float>& Pin, const Vars& Pout64, const VarsT<float>& Pout32,
                        double* Uout, float* const F[3], const Layout& L, const DevGeom& G, const GeomT<float>& Gf,
                        const Scheme& S, const double* dtp, double coef, int8_t* pflag, unsigned long long* cnt,
                        int tpb, cudaStream_t s, FailList fl, const double* fBn, double* dUout,
                        float* const* emf) {
  const CtEmf ect{{emf ? emf[0] : nullptr, emf ? emf[1] : nullptr, emf ? emf[2] : nullptr}};
  auto go = [&](auto kern) {
    kern<<<nblocks((long long)L.n1 * L.n2 * L.n3, tpb), tpb, 0, s>>>(U0, Pin, Pout64, Pout32, Uout, F[0], F[1], F[2],
                                                                     L, G, Gf, S, dtp, coef, pflag, cnt, fl, fBn,
                                                                     dUout, ect);
  };
  if (S.c2p.method == C2P_KASTAUN) go(k_update_mixed<C2P_KASTAUN>);
  else if (S.c2p.method == C2P_1DW) go(k_update_mixed<C2P_1DW>);
  else if (S.mixed_fp64) go(k_update_mixed<C2P_NOBLE2D_FP64>);
  else go(k_update_mixed<C2P_NOBLE2D>);
  return 1;
}

template <class T>
int launch_fixup(const VarsT<T>& P, double* Uout, const int8_t* pflag, const Layout& L, const DevGeom& G,
                 const Scheme& S, unsigned long long* cnt, cudaStream_t s, FailList fl) {
  const long long nz = (long long)L.n1 * L.n2 * L.n3;
  if (fl.idx) {
    // the list is short in practice; its length is known only on the device
    long long b = nblocks(nz, TPB);
    if (b > 152) b = 152;
    launch_pdl(k_fixup_list<T>, dim3((unsigned)b), dim3(TPB), 0, s, P, Uout, pflag, L, G, S, cnt, fl);
  } else {
    k_fixup<T><<<nblocks(nz, TPB), TPB, 0, s>>>(P, Uout, pflag, L, G, S, cnt);
  }
  return 1;
}
template int launch_fixup<double>(const VarsT<double>&, double*, const int8_t*, const Layout&, const DevGeom&,
                                  const Scheme&, unsigned long long*, cudaStream_t, FailList);
template int launch_fixup<float>(const VarsT<float>&, double*, const int8_t*, const Layout&, const DevGeom&,
                                 const Scheme&, unsigned long long*, cudaStream_t, FailList);

template <class T>
int launch_cfl(T* const ctop[3], const Layout& L, double cfl, double* partial, int npartial, double* dt_out,
               cudaStream_t s) {
  launch_pdl(k_cfl<T>, dim3(npartial), dim3(RED_THREADS), 0, s, ctop[0], ctop[1], ctop[2], L, partial);
  launch_pdl(k_finish, dim3(1), dim3(RED_THREADS), 0, s, partial, npartial, cfl, 0, dt_out);
  return 2;
}
template int launch_cfl<double>(double* const[3], const Layout&, double, double*, int, double*, cudaStream_t);
template int launch_cfl<float>(float* const[3], const Layout&, double, double*, int, double*, cudaStream_t);

// The interior state in the compact order [16][n3][n2][n1] (U's 8 slots,
// then P's 5 and B's 3) from / to the padded layout.
__global__ void k_pack(const double* U, CVars PB, double* out, Layout L) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nz = nzones(L);
  if (t >= nz) return;
  int i, j, k;
  zone_ijk(L, t, i, j, k);
  const long long c = L.at(k, j, i);
  // all sixteen loads first (in flight together), then the stores
  double q[2 * NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    q[v] = U[v * L.plane + c];
    q[NV + v] = PB.v[v][c];
  }
#pragma unroll
  for (int v = 0; v < 2 * NV; ++v) out[(long long)v * nz + t] = q[v];
}

__global__ void k_unpack(const double* in, double* U, Vars PB, Layout L) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nz = nzones(L);
  if (t >= nz) return;
  int i, j, k;
  zone_ijk(L, t, i, j, k);
  const long long c = L.at(k, j, i);
  // all sixteen loads first (over the host link when `in` is pinned host
  // memory: their latencies overlap), then the stores
  double q[2 * NV];
#pragma unroll
  for (int v = 0; v < 2 * NV; ++v) q[v] = in[(long long)v * nz + t];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    U[v * L.plane + c] = q[v];
    PB.v[v][c] = q[NV + v];
  }
}

int launch_pack(const double* U, const CVars& PB, double* out, const Layout& L, cudaStream_t s) {
  const long long nz = (long long)L.n1 * L.n2 * L.n3;
  k_pack<<<nblocks(nz, TPB), TPB, 0, s>>>(U, PB, out, L);
  return 1;
}

int launch_unpack(const double* in, double* U, const Vars& PB, const Layout& L, cudaStream_t s) {
  const long long nz = (long long)L.n1 * L.n2 * L.n3;
  k_unpack<<<nblocks(nz, TPB), TPB, 0, s>>>(in, U, PB, L);
  return 1;
}

int launch_fill_f32(const CVars& src, const VarsT<float>& dst, const Layout& L, const Scheme& S, const double* dlo,
                    const double* dhi, cudaStream_t s) {
  const long long tot = (long long)L.N1 * L.N2 * L.N3;
  launch_pdl(k_fill_f32, dim3((unsigned)nblocks(tot, TPB)), dim3(TPB), 0, s, src, dst, L, S, dlo, dhi);
  return 1;
}

int launch_vars_to_f32(const CVars& src, const VarsT<float>& dst, const Layout& L, cudaStream_t s) {
  long long b = nblocks(L.plane, 256);
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  k_vars_to_f32<<<(int)b, 256, 0, s>>>(src, dst, L.plane);
  return 1;
}

__global__ void k_df_planes(const double* geo, const double* flo, float* df, long long gplane) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < gplane;
       p += (long long)gridDim.x * blockDim.x) {
    auto put = [&](int q, double x) {
      const df64 v = df_of_f64(x);
      df[2 * (q * gplane + p)] = v.hi;
      df[2 * (q * gplane + p) + 1] = v.lo;
    };
    // cell-centre planes: gcov pairs 0..9, gcon pairs 10..19, gdet 20, alpha 21
    const double* gc = geo + 10 * gplane + p;
    for (int q = 0; q < 4; ++q) put(DF_GCON0 + q, gc[q * gplane]);  // g^{0m}: pairs 00 01 02 03
    const int sp[6][2] = {{1, 1}, {1, 2}, {1, 3}, {2, 2}, {2, 3}, {3, 3}};
    for (int q = 0; q < 6; ++q) {  // gamma^{ij} = g^{ij} - g^{0i} g^{0j} / g^{00}, in FP64
      const int a = sp[q][0], b = sp[q][1];
      put(DF_GSP + q, gc[(4 + q) * gplane] - gc[a * gplane] * gc[b * gplane] / gc[0]);
    }
    for (int q = 0; q < 6; ++q) put(DF_GCOV + q, geo[(4 + q) * gplane + p]);  // pairs 11 12 13 22 23 33
    put(DF_ALPHA, geo[21 * gplane + p]);
    put(DF_IG, flo[2 * gplane + p]);
    put(DF_RHOFL, flo[p]);
    put(DF_UFL, flo[gplane + p]);
  }
}

int launch_df_planes(const double* geo, const double* flo, float* df, long long gplane, cudaStream_t s) {
  long long b = nblocks(gplane, 256);
  if (b > 152 * 4) b = 152 * 4;
  if (b < 1) b = 1;
  k_df_planes<<<(int)b, 256, 0, s>>>(geo, flo, df, gplane);
  return 1;
}

int launch_to_f32(const double* src, float* dst, long long n, cudaStream_t s) {
  long long b = nblocks(n, 256);
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  k_to_f32<<<(int)b, 256, 0, s>>>(src, dst, n);
  return 1;
}

int launch_divb(const double* const B[3], const Layout& L, const DevGeom& G, double* partial, int npartial,
                double* out2, cudaStream_t s) {
  k_divb<<<npartial, RED_THREADS, 0, s>>>(B[0], B[1], B[2], L, G, partial);
  k_finish<<<1, RED_THREADS, 0, s>>>(partial, npartial, 0.0, 1, out2);
  return 2;
}

static long long box_count(const Layout& L, int pad) {
  long long t = 1;
  for (int q = 0; q < 3; ++q) t *= (q < 2 || L.ndim == 3) ? (long long)(L.e[q] - L.s[q] + 1 + pad) : 1LL;
  return t;
}

template <class R>
int launch_face_ct(const CVarsT<R>& P, R* const F[3], R* ecc, R* const emf[3], const double* fB0, double* fBout,
                   const Layout& L, const GeomT<R>& G, const Scheme& S, const double* dtp, double coef,
                   cudaStream_t s) {
  int n = 0;
  if (S.emf == KH_EMF_GS05) {
    k_cell_emf<R><<<nblocks(box_count(L, 1), TPB), TPB, 0, s>>>(P, L, G, ecc);
    ++n;
  }
  const long long tot = box_count(L, 0);
  k_face_emf<R><<<nblocks(tot, TPB), TPB, 0, s>>>(F[0], F[1], F[2], ecc, emf[0], emf[1], emf[2], L, S, S.emf);
  k_face_update<R><<<nblocks(tot, TPB), TPB, 0, s>>>(fB0, fBout, emf[0], emf[1], emf[2], L, dtp, coef);
  return n + 2;
}
template int launch_face_ct<double>(const CVarsT<double>&, double* const[3], double*, double* const[3],
                                    const double*, double*, const Layout&, const GeomT<double>&, const Scheme&,
                                    const double*, double, cudaStream_t);
template int launch_face_ct<float>(const CVarsT<float>&, float* const[3], float*, float* const[3], const double*,
                                   double*, const Layout&, const GeomT<float>&, const Scheme&, const double*, double,
                                   cudaStream_t);

int launch_lincomb(double* out, int nterm, const double* const* in, const double* a, long long n, cudaStream_t s) {
  LinComb lc{};
  for (int t = 0; t < nterm; ++t) {
    lc.in[t] = in[t];
    lc.a[t] = a[t];
  }
  lc.n = nterm;
  long long b = nblocks(n, TPB);
  if (b > 152 * 16) b = 152 * 16;
  k_lincomb<<<(int)b, TPB, 0, s>>>(out, lc, n);
  return 1;
}

int launch_face_divb(const double* fB, const Layout& L, double* partial, int npartial, double* out2, cudaStream_t s) {
  k_face_divb<<<npartial, RED_THREADS, 0, s>>>(fB, L, partial);
  k_finish<<<1, RED_THREADS, 0, s>>>(partial, npartial, 0.0, 1, out2);
  return 2;
}

int launch_face_to_cell(const double* fB, double* B, const Layout& L, const DevGeom& G, cudaStream_t s) {
  const long long nz = (long long)L.n1 * L.n2 * L.n3;
  k_face_to_cell<<<nblocks(nz, TPB), TPB, 0, s>>>(fB, B, L, G);
  return 1;
}

int launch_p2c(const CVars& P, double* U, const Layout& L, const DevGeom& G, const Scheme& S, cudaStream_t s) {
  const long long tot = (long long)L.N1 * L.N2 * L.N3;
  k_p2c<<<nblocks(tot, TPB), TPB, 0, s>>>(P, U, L, G, S);
  return 1;
}

int launch_c2p(const double* U, const Vars& P, int8_t* pflag, const Layout& L, const DevGeom& G, const Scheme& S,
               unsigned long long* cnt, cudaStream_t s) {
  const long long tot = (long long)L.N1 * L.N2 * L.N3;
  if (S.c2p.method == C2P_KASTAUN)
    k_c2p<C2P_KASTAUN><<<nblocks(tot, TPB), TPB, 0, s>>>(U, P, pflag, L, G, S, cnt);
  else if (S.c2p.method == C2P_1DW)
    k_c2p<C2P_1DW><<<nblocks(tot, TPB), TPB, 0, s>>>(U, P, pflag, L, G, S, cnt);
  else
    k_c2p<C2P_NOBLE2D><<<nblocks(tot, TPB), TPB, 0, s>>>(U, P, pflag, L, G, S, cnt);
  return 1;
}

}  // namespace kh
