// Adjoint (vector-Jacobian product) of one FP64 step of the HARM scheme:
// given the gradient of an objective with respect to the step's outputs
// (U^{n+1}, P^{n+1}, and optionally the stage-2 x1 face fluxes), the gradient
// with respect to its inputs (U^n, P^n) and to the adiabatic index.
//
// The step is first re-run from its checkpoint (U^n, P^n) with the forward
// kernels, recording the ghost-filled stage inputs and each inversion's
// result before floors. The reverse pass then walks the stages backwards:
//   * inversion + floors: implicit-function adjoint of p2c(P) = U (a 5x5 FP64
//     solve per zone with the Jacobian of the conserved variables in the
//     fluid primitives; B = U_B / sqrt(-g)); floored components and zones
//     that were fixed up are frozen (zero derivative upstream); where stage
//     2 recomputed U from floored P, the gradient of that recomputation;
//   * update: transpose of the flux divergence, source-term gradient;
//   * Flux-CT: transpose of the (linear) EMF averaging; axis fluxes zero;
//   * LLF: the two states' fluxes, conserved vectors and the active signal
//     speed of ctop = max(0, c+_L, c+_R, -c-_L, -c-_R) (first argument on
//     ties); reconstruction through the branch the forward took (MC) or the
//     smooth WENO5 weights;
//   * ghost fill: transpose of the copies (sign flips, clamped inflow = 0).
// Local Jacobians come from forward-mode dual numbers (kh_dual.cuh) over the
// same templated physics the forward kernels run.
#include <math.h>

#include "kh_ctx.h"
#include "kh_dual.cuh"
#include "kh_face_vjp.cuh"
#include "kh_zone.cuh"

using namespace kh;

namespace {

constexpr int ATPB = 128;
constexpr int AFPB = 64;  // face kernels (large per-thread state)
using D9 = Dn<9>;         // 8 primitives + the adiabatic index

int adj_rc(cudaError_t e) { return e == cudaSuccess ? KH_OK : (e == cudaErrorMemoryAllocation ? KH_ENOMEM : KH_ECUDA); }
inline int nb(long long n, int t) { return (int)((n + t - 1) / t); }

// Warp-sum then one atomic per warp.
__device__ __forceinline__ void add_scalar(double* out, double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out, v);
}

__device__ __forceinline__ bool interior(const Layout& L, int i, int j, int k) {
  return i >= L.s[0] && i < L.e[0] && j >= L.s[1] && j < L.e[1] && k >= L.s[2] && k < L.e[2];
}

// ---- forward record: the FP64 update that also stores the pre-floor result ----
__global__ void __launch_bounds__(ATPB) k_update_rec(const double* U0, CVars Pin, Vars Pout, double* Uout,
                                                    const double* F1, const double* F2, const double* F3, Layout L,
                                                    DevGeom G, Scheme S, const double* dtp, double coef,
                                                    int8_t* pflag, unsigned long long* cnt, double* Praw) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nzones(L)) return;
  int i, j, k;
  zone_ijk(L, t, i, j, k);
  update_zone(U0, Pin, Pout, Uout, F1, F2, F3, L, G, S, coef * __ldg(dtp), pflag, cnt, i, j, k, Praw);
}

// Conserved vector of P with its Jacobian in (P, gamma): J[u][q] = dU_u/dx_q.
__device__ __forceinline__ void p2c_jacobian(const double* P, const Met<double>& m, double gam, double J[NV][9]) {
  D9 Pd[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Pd[v] = D9::var(P[v], v);
  const D9 g = D9::var(gam, 8);
  FState<D9> s;
  fluid_state(Pd, m, s);
  D9 Ud[NV];
  cons_only(Pd, s, m, g, Ud);
#pragma unroll
  for (int u = 0; u < NV; ++u)
#pragma unroll
    for (int q = 0; q < 9; ++q) J[u][q] = Ud[u].d[q];
}

// Solve A x = b (5x5, partial pivoting); returns false if singular.
__device__ bool solve5(double A[5][5], double b[5]) {
  for (int c = 0; c < 5; ++c) {
    int piv = c;
    double best = fabs(A[c][c]);
    for (int r = c + 1; r < 5; ++r)
      if (fabs(A[r][c]) > best) {
        best = fabs(A[r][c]);
        piv = r;
      }
    if (!(best > 0.0)) return false;
    if (piv != c) {
      for (int q = 0; q < 5; ++q) {
        const double t = A[c][q];
        A[c][q] = A[piv][q];
        A[piv][q] = t;
      }
      const double t = b[c];
      b[c] = b[piv];
      b[piv] = t;
    }
    const double ip = 1.0 / A[c][c];
    for (int r = c + 1; r < 5; ++r) {
      const double f = A[r][c] * ip;
      if (f == 0.0) continue;
      for (int q = c; q < 5; ++q) A[r][q] -= f * A[c][q];
      b[r] -= f * b[c];
    }
  }
  for (int c = 4; c >= 0; --c) {
    double acc = b[c];
    for (int q = c + 1; q < 5; ++q) acc -= A[c][q] * b[q];
    b[c] = acc / A[c][c];
  }
  return true;
}

// ---- reverse of inversion + floors (+ stage 2's recomputed U) ----
// gP: adjoint of the stage output P (8 slots, null slots = 0); gU: adjoint of
// the stage output U (stage 2 only, may be null). Writes lu = adjoint of U
// before the inversion.
__global__ void __launch_bounds__(ATPB) k_adj_out(CVars gP, const double* gU, const double* Praw, CVars Pout,
                                                 const int8_t* pflag, int recompute_u, Layout L, DevGeom G, Scheme S,
                                                 double* lu, double* gsum) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  double dg = 0.0;
  if (t < nzones(L)) {
    int i, j, k;
    zone_ijk(L, t, i, j, k);
    const long long c = L.at(k, j, i);
    const long long p = (long long)j * L.n1s + i;
    double lU[NV], lP[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      lU[v] = 0.0;
      lP[v] = gP.v[v] ? gP.v[v][c] : 0.0;
    }
    if (pflag[c] == 0) {  // a zone that was fixed up is frozen
      double po[NV], pr[NV];
      bool floored = false;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        po[v] = Pout.v[v][c];
        pr[v] = Praw[v * L.plane + c];
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) floored |= (po[v] != pr[v]);
      const Met<double> m = load_met(G, L.gplane, LOC_CENT, p);
      double J[NV][9];
      if (gU) {
        if (floored && recompute_u) {  // U = p2c(P_out): its gradient flows into P_out
          p2c_jacobian(po, m, S.gam, J);
          for (int q = 0; q < 9; ++q) {
            double acc = 0.0;
            for (int u = 0; u < NV; ++u) acc += gU[u * L.plane + c] * J[u][q];
            if (q < NV) lP[q] += acc; else dg += acc;
          }
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) lU[v] = gU[v * L.plane + c];
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v)
        if (po[v] != pr[v]) lP[v] = 0.0;  // floored component: frozen
      // implicit function p2c(P) = U at the pre-floor result
      p2c_jacobian(pr, m, S.gam, J);
      double A[5][5], mu[5];
      for (int a = 0; a < 5; ++a) {
        mu[a] = lP[a];
        for (int b = 0; b < 5; ++b) A[a][b] = J[b][a];  // J_ff^T
      }
      if (solve5(A, mu)) {
        const double ig = __ldg(G.flo + 2 * L.gplane + p);
        for (int f = 0; f < 5; ++f) lU[f] += mu[f];
        for (int b = 0; b < 3; ++b) {
          double acc = lP[5 + b];
          for (int f = 0; f < 5; ++f) acc -= J[f][5 + b] * mu[f];
          lU[5 + b] += acc * ig;
        }
        for (int f = 0; f < 5; ++f) dg -= mu[f] * J[f][8];
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) lu[v * L.plane + c] = lU[v];
  }
  add_scalar(gsum, dg);
}

// ---- reverse of the update's base and sources: gU_in += lu; sources ----
__global__ void __launch_bounds__(ATPB) k_adj_src(const double* lu, CVars Ph, Layout L, DevGeom G, Scheme S,
                                                 const double* dtp, double coef, double* gU_in, double* lp,
                                                 double* gsum, int has_sources) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  double dg = 0.0;
  if (t < nzones(L)) {
    int i, j, k;
    zone_ijk(L, t, i, j, k);
    const long long c = L.at(k, j, i);
    const long long p = (long long)j * L.n1s + i;
    const double cdt = coef * __ldg(dtp);
    double ls[NV];
    bool any = false;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double x = lu[v * L.plane + c];
      gU_in[v * L.plane + c] += x;
      ls[v] = cdt * x;
      any |= (v >= V_U && v <= V_U3 && x != 0.0);
    }
    if (any && has_sources) {
      D9 Pd[NV], Sd[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Pd[v] = D9::var(Ph.v[v][c], v);
        Sd[v] = D9(0.0);
      }
      const Met<double> m = load_met(G, L.gplane, LOC_CENT, p);
      source_terms(Pd, m, G.dgm, L.gplane, p, D9::var(S.gam, 8), Sd);
      for (int q = 0; q < 9; ++q) {
        double acc = 0.0;
        for (int v = V_U; v <= V_U3; ++v) acc += ls[v] * Sd[v].d[q];
        if (q < NV) lp[q * L.plane + c] += acc; else dg += acc;
      }
    }
  }
  add_scalar(gsum, dg);
}

// ---- transpose of the flux divergence: face adjoints (plus a seed) ----
template <int D>
__global__ void k_adj_div(const double* lu, double* lf, FaceBox box, Layout L, const double* dtp, double coef,
                          const double* seed) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)box.n[0] * box.n[1] * box.n[2]) return;
  int i, j, k;
  split3(t, box.n[0], box.n[1], i, j, k);
  i += box.lo[0];
  j += box.lo[1];
  k += box.lo[2];
  const long long c = L.at(k, j, i);
  const long long st = (D == 1) ? 1 : (D == 2 ? (long long)L.n1s : (long long)L.n1s * L.n2s);
  const bool up = interior(L, i, j, k);
  const bool dn = interior(L, i - (D == 1), j - (D == 2), k - (D == 3));
  const double f = coef * __ldg(dtp) * L.idx[D - 1];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double a = up ? lu[v * L.plane + c] : 0.0;
    const double b = dn ? lu[v * L.plane + c - st] : 0.0;
    lf[v * L.plane + c] = f * (a - b) + (seed ? seed[v * L.plane + c] : 0.0);
  }
}

// ---- transpose of Flux-CT ----
// Index ranges of the forward: EMFs e3 on i in [s0,e0], j in [s1,e1], k in
// [s2,e2) (3-D) or k = 0; e1 on i < e0; e2 on j < e1; face rewrites on x1
// faces with j < e1 (and k < e2 in 3-D), x2 faces with i < e0, x3 faces with
// i < e0 and j < e1.
struct CtRange {
  int s[3], e[3], nd;
  __device__ bool kin(int k, bool closed) const {
    return nd == 2 ? k == 0 : (k >= s[2] && (closed ? k <= e[2] : k < e[2]));
  }
  __device__ bool e3(int i, int j, int k) const {
    return i >= s[0] && i <= e[0] && j >= s[1] && j <= e[1] && kin(k, false);
  }
  __device__ bool e1(int i, int j, int k) const {
    return nd == 3 && i >= s[0] && i < e[0] && j >= s[1] && j <= e[1] && k >= s[2] && k <= e[2];
  }
  __device__ bool e2(int i, int j, int k) const {
    return nd == 3 && i >= s[0] && i <= e[0] && j >= s[1] && j < e[1] && k >= s[2] && k <= e[2];
  }
  __device__ bool x1(int i, int j, int k) const {
    return i >= s[0] && i <= e[0] && j >= s[1] && j < e[1] && kin(k, false);
  }
  __device__ bool x2(int i, int j, int k) const {
    return i >= s[0] && i < e[0] && j >= s[1] && j <= e[1] && kin(k, false);
  }
  __device__ bool x3(int i, int j, int k) const {
    return nd == 3 && i >= s[0] && i < e[0] && j >= s[1] && j < e[1] && k >= s[2] && k <= e[2];
  }
};

inline CtRange ct_range(const Layout& L) {
  CtRange r;
  for (int a = 0; a < 3; ++a) {
    r.s[a] = L.s[a];
    r.e[a] = L.e[a];
  }
  r.nd = L.ndim;
  return r;
}

__global__ void k_adj_emf(const double* lf1, const double* lf2, const double* lf3, double* le1, double* le2,
                          double* le3, Layout L, CtRange R) {
  const int n0 = L.e[0] - L.s[0] + 1, n1 = L.e[1] - L.s[1] + 1, n2 = (L.ndim == 3) ? L.e[2] - L.s[2] + 1 : 1;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)n0 * n1 * n2) return;
  int i, j, k;
  split3(t, n0, n1, i, j, k);
  i += L.s[0];
  j += L.s[1];
  k += (L.ndim == 3 ? L.s[2] : 0);
  const long long c = L.at(k, j, i), P = L.plane, sj = L.n1s, sk = (long long)L.n1s * L.n2s;
  auto at = [&](const double* f, int v, long long q) { return f[v * P + q]; };
  if (R.e3(i, j, k)) {
    double a = 0.0;
    if (R.x1(i, j, k)) a += 0.5 * at(lf1, V_B2, c);
    if (R.x1(i, j - 1, k)) a += 0.5 * at(lf1, V_B2, c - sj);
    if (R.x2(i, j, k)) a -= 0.5 * at(lf2, V_B1, c);
    if (R.x2(i - 1, j, k)) a -= 0.5 * at(lf2, V_B1, c - 1);
    le3[c] = a;
  }
  if (R.e1(i, j, k)) {
    double a = 0.0;
    if (R.x2(i, j, k)) a += 0.5 * at(lf2, V_B3, c);
    if (R.x2(i, j, k - 1)) a += 0.5 * at(lf2, V_B3, c - sk);
    if (R.x3(i, j, k)) a -= 0.5 * at(lf3, V_B2, c);
    if (R.x3(i, j - 1, k)) a -= 0.5 * at(lf3, V_B2, c - sj);
    le1[c] = a;
  }
  if (R.e2(i, j, k)) {
    double a = 0.0;
    if (R.x3(i, j, k)) a += 0.5 * at(lf3, V_B1, c);
    if (R.x3(i - 1, j, k)) a += 0.5 * at(lf3, V_B1, c - 1);
    if (R.x1(i, j, k)) a -= 0.5 * at(lf1, V_B3, c);
    if (R.x1(i, j, k - 1)) a -= 0.5 * at(lf1, V_B3, c - sk);
    le2[c] = a;
  }
}

// The field-flux adjoints before Flux-CT (faces of direction D's face box);
// axis faces of x2 get zero (the forward zeroed their fluxes).
template <int D>
__global__ void k_adj_ctf(double* lf, const double* le1, const double* le2, const double* le3, FaceBox box,
                          Layout L, CtRange R, int polar_lo, int polar_hi) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)box.n[0] * box.n[1] * box.n[2]) return;
  int i, j, k;
  split3(t, box.n[0], box.n[1], i, j, k);
  i += box.lo[0];
  j += box.lo[1];
  k += box.lo[2];
  const long long c = L.at(k, j, i), P = L.plane, sj = L.n1s, sk = (long long)L.n1s * L.n2s;
  if (D == 2 && ((polar_lo && j == L.s[1]) || (polar_hi && j == L.e[1]))) {
#pragma unroll
    for (int v = 0; v < NV; ++v) lf[v * P + c] = 0.0;
    return;
  }
  const bool app = D == 1 ? R.x1(i, j, k) : (D == 2 ? R.x2(i, j, k) : R.x3(i, j, k));
  double b[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const bool touched = app && (L.ndim == 3 || q < 2);  // 2-D: CT leaves the B3 fluxes
    b[q] = touched ? 0.0 : lf[(V_B1 + q) * P + c];
  }
  if (D == 1) {
    if (R.e3(i, j, k)) b[1] += 0.25 * le3[c];
    if (R.e3(i, j + 1, k)) b[1] += 0.25 * le3[c + sj];
    if (R.e2(i, j, k)) b[2] -= 0.25 * le2[c];
    if (R.e2(i, j, k + 1)) b[2] -= 0.25 * le2[c + sk];
  } else if (D == 2) {
    if (R.e3(i, j, k)) b[0] -= 0.25 * le3[c];
    if (R.e3(i + 1, j, k)) b[0] -= 0.25 * le3[c + 1];
    if (R.e1(i, j, k)) b[2] += 0.25 * le1[c];
    if (R.e1(i, j, k + 1)) b[2] += 0.25 * le1[c + sk];
  } else {
    if (R.e2(i, j, k)) b[0] += 0.25 * le2[c];
    if (R.e2(i + 1, j, k)) b[0] += 0.25 * le2[c + 1];
    if (R.e1(i, j, k)) b[1] -= 0.25 * le1[c];
    if (R.e1(i, j + 1, k)) b[1] -= 0.25 * le1[c + sj];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) lf[(V_B1 + q) * P + c] = b[q];
}

// ---- reverse of reconstruction + LLF at one face ----
// Each side's gradient comes from side_grad_rev (kh_face_vjp.cuh, written
// reverse mode); side_grad_dual there is the dual-number evaluation of the
// same quantity that a host test compares it with.
template <int D, int RECON>
__global__ void __launch_bounds__(AFPB) k_adj_face(CVars Ph, const double* lf, Layout L, DevGeom G, Scheme S,
                                                  FaceBox box, int polar_lo, int polar_hi, double* lp, double* gsum) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  double dg = 0.0;
  if (t < (unsigned)box.n[0] * box.n[1] * box.n[2]) {
    int i, j, k;
    // x1 faces run with x2 fastest, so that the lanes of a warp scatter into
    // different cells (with x1 fastest, neighbouring lanes' 6-cell stencils
    // overlap and their atomics serialise)
    if (D == 1) {
      split3(t, box.n[1], box.n[0], j, i, k);
    } else {
      split3(t, box.n[0], box.n[1], i, j, k);
    }
    i += box.lo[0];
    j += box.lo[1];
    k += box.lo[2];
    const long long c = L.at(k, j, i);
    const bool axis = (D == 2) && ((polar_lo && j == L.s[1]) || (polar_hi && j == L.e[1]));
    double lam[NV];
    bool any = false;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      lam[v] = lf[v * L.plane + c];
      any |= lam[v] != 0.0;
    }
    if (any && !axis) {
      const long long st = (D == 1) ? 1 : (D == 2 ? (long long)L.n1s : (long long)L.n1s * L.n2s);
      // reconstruction with its gradient in the stencil (offsets -3..+2 from c)
      double PL[NV], PR[NV], gL[NV][6], gR[NV][6];
      for (int v = 0; v < NV; ++v) {
        const double* q = Ph.v[v] + c;
        for (int o = 0; o < 6; ++o) gL[v][o] = gR[v][o] = 0.0;
        if (RECON == KH_RECON_MC) {
          using D3 = Dn<3>;
          D3 lo, hi;
          recon_mc(D3::var(q[-2 * st], 0), D3::var(q[-st], 1), D3::var(q[0], 2), lo, hi);
          PL[v] = hi.v;
          for (int a = 0; a < 3; ++a) gL[v][1 + a] = hi.d[a];  // offsets -2, -1, 0
          recon_mc(D3::var(q[-st], 0), D3::var(q[0], 1), D3::var(q[st], 2), lo, hi);
          PR[v] = lo.v;
          for (int a = 0; a < 3; ++a) gR[v][2 + a] = lo.d[a];  // offsets -1, 0, +1
        } else {
          using D5 = Dn<5>;
          const D5 l = weno5_plus_t(D5::var(q[-3 * st], 0), D5::var(q[-2 * st], 1), D5::var(q[-st], 2),
                                    D5::var(q[0], 3), D5::var(q[st], 4));
          PL[v] = l.v;
          for (int a = 0; a < 5; ++a) gL[v][a] = l.d[a];  // offsets -3..+1
          const D5 r = weno5_plus_t(D5::var(q[2 * st], 0), D5::var(q[st], 1), D5::var(q[0], 2),
                                    D5::var(q[-st], 3), D5::var(q[-2 * st], 4));
          PR[v] = r.v;
          for (int a = 0; a < 5; ++a) gR[v][5 - a] = r.d[a];  // offsets +2..-2
        }
      }
      const Met<double> m = load_met(G, L.gplane, D == 3 ? LOC_CENT : D, (long long)j * L.n1s + i);
      // plain pass: ctop, its active speed, and the gradient weight of ctop
      FState<double> sL, sR;
      fluid_state(PL, m, sL);
      fluid_state(PR, m, sR);
      double FL[NV], UL[NV], FR[NV], UR[NV];
      flux_cons(PL, sL, m, S.gam, D, FL, UL);
      flux_cons(PR, sR, m, S.gam, D, FR, UR);
      double cmaxL, cminL, cmaxR, cminR;
      signal_speeds(PL, sL, m, S.gam, D, cmaxL, cminL);
      signal_speeds(PR, sR, m, S.gam, D, cmaxR, cminR);
      // ctop = max(cm, cn), cm = max(0, max(c+L, c+R)), cn = max(0, max(-c-L, -c-R))
      int am = 0, an = 0;  // 0: the zero branch; 1: left; 2: right
      double cm = 0.0, cn = 0.0;
      {
        const double a = cmaxL >= cmaxR ? cmaxL : cmaxR;
        if (!(0.0 >= a)) { cm = a; am = cmaxL >= cmaxR ? 1 : 2; }
        const double b = -cminL >= -cminR ? -cminL : -cminR;
        if (!(0.0 >= b)) { cn = b; an = -cminL >= -cminR ? 1 : 2; }
      }
      const bool use_m = cm >= cn;
      const double ct = use_m ? cm : cn;
      const int side_act = use_m ? am : an;  // which side's speed is active (0: none)
      double lct = 0.0;
#pragma unroll
      for (int v = 0; v < NV; ++v) lct -= 0.5 * lam[v] * (UR[v] - UL[v]);
      double gl[9], gr[9];
      side_grad_rev(PL, m, S.gam, lam, 0.5 * ct, D, side_act == 1 ? (use_m ? 1 : -1) : 0, lct, gl);
      side_grad_rev(PR, m, S.gam, lam, -0.5 * ct, D, side_act == 2 ? (use_m ? 1 : -1) : 0, lct, gr);
      dg += gl[8] + gr[8];
      for (int v = 0; v < NV; ++v) {
        double* dst = lp + v * L.plane + c;
        for (int o = 0; o < 6; ++o) {
          const double a = gl[v] * gL[v][o] + gr[v] * gR[v][o];
          if (a != 0.0) atomicAdd(dst + (o - 3) * st, a);
        }
      }
    }
  }
  add_scalar(gsum, dg);
}

// ---- transpose of the ghost fill (x3, then x2, then x1: the reverse order) ----
__global__ void k_adj_bc_x3(double* lp, Layout L, Scheme S) {
  const long long tot = (long long)L.N1 * L.N2 * L.ng3 * 2;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= tot) return;
  const int i = (int)(t % L.N1);
  const int j = (int)((t / L.N1) % L.N2);
  const int side = (int)((t / ((long long)L.N1 * L.N2)) % 2);
  const int m = (int)(t / (2LL * L.N1 * L.N2));
  const int kg = side == 0 ? L.ng3 - 1 - m : L.ng3 + L.n3 + m;
  const int bc = S.bc[4 + side];
  const int src = (bc == KH_BC_PERIODIC) ? (side == 0 ? kg + L.n3 : kg - L.n3) : (side == 0 ? L.ng3 : L.ng3 + L.n3 - 1);
  const long long s = L.at(src, j, i), d = L.at(kg, j, i);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double x = lp[v * L.plane + d];
    if (x != 0.0) atomicAdd(lp + v * L.plane + s, x);
  }
}

__global__ void k_adj_bc_x2(double* lp, Layout L, Scheme S) {
  const int nk = L.e[2] - L.s[2];
  const long long tot = (long long)L.N1 * nk * L.ng * 2;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= tot) return;
  const int i = (int)(t % L.N1);
  const int side = (int)((t / L.N1) % 2);
  const int m = (int)((t / (2LL * L.N1)) % L.ng);
  const int k = L.s[2] + (int)(t / (2LL * L.N1 * L.ng));
  const int jg = side == 0 ? L.ng - 1 - m : L.ng + L.n2 + m;
  const int bc = S.bc[2 + side];
  int src;
  if (bc == KH_BC_PERIODIC)
    src = side == 0 ? jg + L.n2 : jg - L.n2;
  else if (bc == KH_BC_OUTFLOW)
    src = side == 0 ? L.ng : L.ng + L.n2 - 1;
  else
    src = side == 0 ? 2 * L.ng - 1 - jg : 2 * (L.ng + L.n2) - 1 - jg;
  const long long s = L.at(k, src, i), d = L.at(k, jg, i);
  const bool flip = (bc == KH_BC_POLAR);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double x = lp[v * L.plane + d];
    if (flip && (v == V_U2 || v == V_B2)) x = -x;
    if (x != 0.0) atomicAdd(lp + v * L.plane + s, x);
  }
}

__global__ void k_adj_bc_x1(double* lp, CVars Ph, Layout L, Scheme S) {
  const int nj = L.e[1] - L.s[1], nk = L.e[2] - L.s[2];
  const long long tot = (long long)nj * nk * L.ng * 2;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= tot) return;
  const int side = (int)(t % 2);
  const int m = (int)((t / 2) % L.ng);
  const int j = L.s[1] + (int)((t / (2 * L.ng)) % nj);
  const int k = L.s[2] + (int)(t / (2LL * L.ng * nj));
  const int ig = side == 0 ? L.ng - 1 - m : L.ng + L.n1 + m;
  const int bc = S.bc[side];
  if (bc == KH_BC_DIRICHLET) return;  // fixed values: no dependence
  int src;
  if (bc == KH_BC_PERIODIC)
    src = side == 0 ? ig + L.n1 : ig - L.n1;
  else if (bc == KH_BC_OUTFLOW)
    src = side == 0 ? L.ng : L.ng + L.n1 - 1;
  else
    src = side == 0 ? 2 * L.ng - 1 - ig : 2 * (L.ng + L.n1) - 1 - ig;
  const long long s = L.at(k, j, src), d = L.at(k, j, ig);
  bool clamped = false;
  if (bc == KH_BC_OUTFLOW) {
    const double u1 = Ph.v[V_U1][s];
    clamped = (side == 0 && u1 > 0.0) || (side == 1 && u1 < 0.0);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double x = (v == V_U1 && clamped) ? 0.0 : lp[v * L.plane + d];
    if (x != 0.0) atomicAdd(lp + v * L.plane + s, x);
  }
}

// Interior of the 8-plane adjoint into the caller's P (5 planes) and B (3).
__global__ void k_adj_extract(const double* lp, double* gP, double* gB, Layout L) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= L.plane) return;
  const int i = (int)(t % L.n1s), j = (int)((t / L.n1s) % L.n2s), k = (int)(t / ((long long)L.n1s * L.n2s));
  const bool in = interior(L, i, j, k);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double x = in ? lp[v * L.plane + t] : 0.0;
    if (v < 5) gP[v * L.plane + t] = x; else gB[(v - 5) * L.plane + t] = x;
  }
}

// Gradient of U = p2c(P) at every interior cell: gP = (dU/dP)^T gU (8 slots).
__global__ void __launch_bounds__(ATPB) k_p2c_adj(CVars P, const double* gU, Layout L, DevGeom G, Scheme S,
                                                 double* gP, double* gB, double* gsum) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double dg = 0.0;
  if (t < L.plane) {
    const int i = (int)(t % L.n1s), j = (int)((t / L.n1s) % L.n2s), k = (int)(t / ((long long)L.n1s * L.n2s));
    double g[NV] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (interior(L, i, j, k)) {
      double p[NV], J[NV][9];
      for (int v = 0; v < NV; ++v) p[v] = P.v[v][t];
      const Met<double> m = load_met(G, L.gplane, LOC_CENT, (long long)j * L.n1s + i);
      p2c_jacobian(p, m, S.gam, J);
      for (int q = 0; q < 9; ++q) {
        double acc = 0.0;
        for (int u = 0; u < NV; ++u) acc += gU[u * L.plane + t] * J[u][q];
        if (q < NV) g[q] = acc; else dg = acc;
      }
    }
    for (int v = 0; v < NV; ++v) {
      if (v < 5) gP[v * L.plane + t] = g[v]; else gB[(v - 5) * L.plane + t] = g[v];
    }
  }
  add_scalar(gsum, dg);
}

Vars planes(double* base, const Layout& L) {
  Vars v;
  for (int q = 0; q < NV; ++q) v.v[q] = base + q * L.plane;
  return v;
}
CVars cplanes(const double* base, const Layout& L) {
  CVars v;
  for (int q = 0; q < NV; ++q) v.v[q] = base + q * L.plane;
  return v;
}
CVars cview8(const Vars& a) {
  CVars c;
  for (int q = 0; q < NV; ++q) c.v[q] = a.v[q];
  return c;
}

template <int D>
void launch_face_adj(const kh_ctx* x, const CVars& Ph, const double* lf, double* lp, double* gsum, cudaStream_t s) {
  const Layout& L = x->L;
  const FaceBox b = face_box(L, D);
  const long long tot = (long long)b.n[0] * b.n[1] * b.n[2];
  const int plo = x->S.bc[2] == KH_BC_POLAR, phi = x->S.bc[3] == KH_BC_POLAR;
  const DevGeom G{x->geo, x->dgm, x->flo};
  if (x->S.recon == KH_RECON_MC)
    k_adj_face<D, KH_RECON_MC><<<nb(tot, AFPB), AFPB, 0, s>>>(Ph, lf, L, G, x->S, b, plo, phi, lp, gsum);
  else
    k_adj_face<D, KH_RECON_WENO5><<<nb(tot, AFPB), AFPB, 0, s>>>(Ph, lf, L, G, x->S, b, plo, phi, lp, gsum);
}

template <int D>
void launch_div_ct(const kh_ctx* x, const double* lu, double* lf, double coef, const double* seed, cudaStream_t s) {
  const Layout& L = x->L;
  const FaceBox b = face_box(L, D);
  const long long tot = (long long)b.n[0] * b.n[1] * b.n[2];
  k_adj_div<D><<<nb(tot, ATPB), ATPB, 0, s>>>(lu, lf, b, L, x->dscalar + 3, coef, seed);
}

template <int D>
void launch_ctf(const kh_ctx* x, double* lf, const double* le, cudaStream_t s) {
  const Layout& L = x->L;
  const FaceBox b = face_box(L, D);
  const long long tot = (long long)b.n[0] * b.n[1] * b.n[2];
  const int plo = x->S.bc[2] == KH_BC_POLAR, phi = x->S.bc[3] == KH_BC_POLAR;
  k_adj_ctf<D><<<nb(tot, ATPB), ATPB, 0, s>>>(lf, le, le + L.plane, le + 2 * L.plane, b, L, ct_range(L), plo, phi);
}

// Reverse of one stage: from lu (adjoint of U before the inversion, already
// in x->adj + ADJ_LU) to lp (adjoint of the ghost-filled stage input,
// ghosts folded back into the interior) and gU_in.
void reverse_stage(kh_ctx* x, const CVars& Ph, double coef, const double* seed, double* gU_in, cudaStream_t s) {
  const Layout& L = x->L;
  double* lu = x->adj + ADJ_LU * L.plane;
  double* lp = x->adj + ADJ_LP * L.plane;
  double* lf = x->adj + ADJ_LF * L.plane;
  double* le = x->adj + ADJ_LE * L.plane;
  const DevGeom G{x->geo, x->dgm, x->flo};
  const long long nz = (long long)L.n1 * L.n2 * L.n3;
  cudaMemsetAsync(lp, 0, NV * L.plane * sizeof(double), s);
  k_adj_src<<<nb(nz, ATPB), ATPB, 0, s>>>(lu, Ph, L, G, x->S, x->dscalar + 3, coef, gU_in, lp, x->adj_red,
                                          x->c.kind != KH_MINKOWSKI);
  cudaMemsetAsync(lf, 0, 3 * NV * L.plane * sizeof(double), s);
  cudaMemsetAsync(le, 0, 3 * L.plane * sizeof(double), s);
  launch_div_ct<1>(x, lu, lf, coef, seed, s);
  launch_div_ct<2>(x, lu, lf + NV * L.plane, coef, nullptr, s);
  if (L.ndim == 3) launch_div_ct<3>(x, lu, lf + 2 * NV * L.plane, coef, nullptr, s);
  const long long ne = (long long)(L.e[0] - L.s[0] + 1) * (L.e[1] - L.s[1] + 1) * (L.ndim == 3 ? L.e[2] - L.s[2] + 1 : 1);
  k_adj_emf<<<nb(ne, ATPB), ATPB, 0, s>>>(lf, lf + NV * L.plane, lf + 2 * NV * L.plane, le, le + L.plane,
                                          le + 2 * L.plane, L, ct_range(L));
  launch_ctf<1>(x, lf, le, s);
  launch_ctf<2>(x, lf + NV * L.plane, le, s);
  if (L.ndim == 3) launch_ctf<3>(x, lf + 2 * NV * L.plane, le, s);
  launch_face_adj<1>(x, Ph, lf, lp, x->adj_red, s);
  launch_face_adj<2>(x, Ph, lf + NV * L.plane, lp, x->adj_red, s);
  if (L.ndim == 3) launch_face_adj<3>(x, Ph, lf + 2 * NV * L.plane, lp, x->adj_red, s);
  // ghost fill, transposed
  if (L.ndim == 3) {
    const long long t3 = (long long)L.N1 * L.N2 * L.ng3 * 2;
    k_adj_bc_x3<<<nb(t3, ATPB), ATPB, 0, s>>>(lp, L, x->S);
  }
  const long long t2 = (long long)L.N1 * (L.e[2] - L.s[2]) * L.ng * 2;
  k_adj_bc_x2<<<nb(t2, ATPB), ATPB, 0, s>>>(lp, L, x->S);
  const long long t1 = (long long)(L.e[1] - L.s[1]) * (L.e[2] - L.s[2]) * L.ng * 2;
  k_adj_bc_x1<<<nb(t1, ATPB), ATPB, 0, s>>>(lp, Ph, L, x->S);
}

}  // namespace

extern "C" {

int kh_step_adjoint(kh_ctx* x, const double* U, const double* P, const double* B, double dt, const double* gU,
                    const double* gP, const double* gB, const double* gF1, double* gU_in, double* gP_in,
                    double* gB_in, double* g_gamma) {
  if (!x || !U || !P || !B || !gU_in || !gP_in || !gB_in || !(dt > 0.0) || !isfinite(dt)) return KH_EINVAL;
  if (x->c.precision != KH_FP64 || x->S.fofc || x->S.bfield != KH_B_FLUXCT || x->S.c2p.method != C2P_NOBLE2D ||
      x->S.integrator != KH_INT_VL2)
    return KH_EINVAL;
  const Layout& L = x->L;
  cudaStream_t s = x->stream;
  if (!x->adj) {
    int rc = adj_rc(cudaMalloc((void**)&x->adj, (size_t)ADJ_PLANES * L.plane * sizeof(double)));
    if (rc == KH_OK) rc = adj_rc(cudaMalloc((void**)&x->adj_i8, (size_t)4 * L.plane));
    if (rc == KH_OK) rc = adj_rc(cudaMalloc((void**)&x->adj_red, sizeof(double)));
    if (rc != KH_OK) return rc;
  }
  const size_t pl = (size_t)L.plane * sizeof(double);
  int rc = adj_rc(cudaMemcpyAsync(x->dscalar + 3, &dt, sizeof(double), cudaMemcpyHostToDevice, s));
  if (rc != KH_OK) return rc;
  double* ph1 = x->adj + ADJ_PH1 * L.plane;
  double* raw1 = x->adj + ADJ_RAW1 * L.plane;
  double* pn1 = x->adj + ADJ_PN1 * L.plane;
  double* raw2 = x->adj + ADJ_RAW2 * L.plane;
  double* un1 = x->adj + ADJ_UN1 * L.plane;
  int8_t* pflag1 = x->adj_i8;
  const DevGeom G{x->geo, x->dgm, x->flo};
  const long long nz = (long long)L.n1 * L.n2 * L.n3;

  // ---- forward record from the checkpoint (the kernels of kh_step) ----
  cudaMemcpyAsync(ph1, P, 5 * pl, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(ph1 + 5 * L.plane, B, 3 * pl, cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(x->counters, 0, NCNT * sizeof(unsigned long long), s);
  const Vars Ph1 = planes(ph1, L), Pst = planes(x->pstar, L), Pn1 = planes(pn1, L);
  for (int st = 0; st < 2; ++st) {
    const Vars& Pin = st == 0 ? Ph1 : Pst;
    const Vars& Pout = st == 0 ? Pst : Pn1;
    launch_bc<double>(Pin, L, x->S, x->dirichlet[0], x->dirichlet[1], s);
    for (int d = 1; d <= L.ndim; ++d)
      launch_flux_dir<double, double>(d, cview8(Pin), L, G, x->S, x->F[d - 1], x->ctop[d - 1], x->tpb_flux, s);
    launch_ct<double>(x->F, x->emf, L, s);
    k_update_rec<<<nb(nz, ATPB), ATPB, 0, s>>>(U, cview8(Pin), Pout, st == 0 ? nullptr : un1, x->F[0], x->F[1],
                                               x->F[2], L, G, x->S, x->dscalar + 3, st == 0 ? 0.5 : 1.0, x->pflag,
                                               x->counters, st == 0 ? raw1 : raw2);
    launch_fixup<double>(Pout, st == 0 ? nullptr : un1, x->pflag, L, G, x->S, x->counters, s);
    if (st == 0) cudaMemcpyAsync(pflag1, x->pflag, (size_t)L.plane, cudaMemcpyDeviceToDevice, s);
  }
  rc = adj_rc(cudaGetLastError());
  if (rc != KH_OK) return rc;

  // ---- reverse ----
  cudaMemsetAsync(gU_in, 0, 8 * pl, s);
  cudaMemsetAsync(x->adj_red, 0, sizeof(double), s);
  double* lu = x->adj + ADJ_LU * L.plane;
  double* lp = x->adj + ADJ_LP * L.plane;
  CVars gPv;
  for (int q = 0; q < 5; ++q) gPv.v[q] = gP ? gP + q * L.plane : nullptr;
  for (int q = 0; q < 3; ++q) gPv.v[5 + q] = gB ? gB + q * L.plane : nullptr;
  // stage 2: outputs P^{n+1} (with U recomputed where floored) and U^{n+1}
  k_adj_out<<<nb(nz, ATPB), ATPB, 0, s>>>(gPv, gU, raw2, cview8(Pn1), x->pflag, 1, L, G, x->S, lu, x->adj_red);
  reverse_stage(x, cview8(Pst), 1.0, gF1, gU_in, s);
  // stage 1: output P* only
  k_adj_out<<<nb(nz, ATPB), ATPB, 0, s>>>(cplanes(lp, L), nullptr, raw1, cview8(Pst), pflag1, 0, L, G, x->S, lu,
                                          x->adj_red);
  reverse_stage(x, cview8(Ph1), 0.5, nullptr, gU_in, s);
  k_adj_extract<<<nb(L.plane, ATPB), ATPB, 0, s>>>(lp, gP_in, gB_in, L);
  double gg = 0.0;
  rc = adj_rc(cudaGetLastError());
  if (rc == KH_OK) rc = adj_rc(cudaMemcpyAsync(&gg, x->adj_red, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (rc == KH_OK) rc = adj_rc(cudaStreamSynchronize(s));
  if (rc != KH_OK) return rc;
  if (g_gamma) *g_gamma = gg;
  return KH_OK;
}

int kh_prim_to_cons_adjoint(kh_ctx* x, const double* P, const double* B, const double* gU, double* gP, double* gB,
                            double* g_gamma) {
  if (!x || !P || !B || !gU || !gP || !gB) return KH_EINVAL;
  if (x->c.precision != KH_FP64) return KH_EINVAL;
  const Layout& L = x->L;
  cudaStream_t s = x->stream;
  if (!x->adj_red) {
    const int rc = adj_rc(cudaMalloc((void**)&x->adj_red, sizeof(double)));
    if (rc != KH_OK) return rc;
  }
  CVars Pv;
  for (int q = 0; q < 5; ++q) Pv.v[q] = P + q * L.plane;
  for (int q = 0; q < 3; ++q) Pv.v[5 + q] = B + q * L.plane;
  cudaMemsetAsync(x->adj_red, 0, sizeof(double), s);
  k_p2c_adj<<<nb(L.plane, ATPB), ATPB, 0, s>>>(Pv, gU, L, DevGeom{x->geo, x->dgm, x->flo}, x->S, gP, gB,
                                               x->adj_red);
  double gg = 0.0;
  int rc = adj_rc(cudaGetLastError());
  if (rc == KH_OK) rc = adj_rc(cudaMemcpyAsync(&gg, x->adj_red, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (rc == KH_OK) rc = adj_rc(cudaStreamSynchronize(s));
  if (rc != KH_OK) return rc;
  if (g_gamma) *g_gamma = gg;
  return KH_OK;
}

int kh_get_stage_flux(kh_ctx* x, int dir, double* F) {
  if (!x || !F || dir < 1 || dir > x->L.ndim || x->c.precision != KH_FP64) return KH_EINVAL;
  const size_t n = (size_t)NV * x->L.plane * sizeof(double);
  return adj_rc(cudaMemcpyAsync(F, x->F[dir - 1], n, cudaMemcpyDeviceToDevice, x->stream));
}

}  // extern "C"
