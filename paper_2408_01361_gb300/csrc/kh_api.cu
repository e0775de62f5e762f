// C ABI of the library (declared in include/kharma_gb300.h): context,
// device buffers, the step driver and the diagnostics.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>

#include <nvtx3/nvToolsExt.h>

#include "kh_ctx.h"

using namespace kh;

extern "C" int kh_get_stats(kh_ctx* x, kh_stats* out);


namespace {

int cuda_fail(cudaError_t e) {
  if (e == cudaSuccess) return KH_OK;
  return e == cudaErrorMemoryAllocation ? KH_ENOMEM : KH_ECUDA;
}

#define KH_TRY(call)                      \
  do {                                    \
    int _rc = cuda_fail(call);            \
    if (_rc != KH_OK) return _rc;         \
  } while (0)

DevGeom devgeom(const kh_ctx* x) { return DevGeom{x->geo, x->dgm, x->flo}; }

Vars vars_of(const kh_ctx* x, double* P, double* B) {
  Vars v;
  for (int q = 0; q < 5; ++q) v.v[q] = P + q * x->L.plane;
  for (int q = 0; q < 3; ++q) v.v[5 + q] = B + q * x->L.plane;
  return v;
}

CVars cvars_of(const kh_ctx* x, const double* P, const double* B) {
  CVars v;
  for (int q = 0; q < 5; ++q) v.v[q] = P + q * x->L.plane;
  for (int q = 0; q < 3; ++q) v.v[5 + q] = B + q * x->L.plane;
  return v;
}

CVars cview(const Vars& v) {
  CVars c;
  for (int q = 0; q < NV; ++q) c.v[q] = v.v[q];
  return c;
}

// NVTX range names of the kernel groups (visible to Nsight tools; a no-op
// when no tool is attached).
const char* const kGroupName[KH_NTIMERS] = {"kh ghost fill", "kh faces x1", "kh faces x2", "kh faces x3",
                                            "kh flux-CT",    "kh update",   "kh fixup",    "kh CFL",
                                            "kh flux correction"};

void mark(kh_ctx* x, int group, int stage, int which) {
  if (which == 0)
    nvtxRangePushA(kGroupName[group]);
  else
    nvtxRangePop();
  if (!x->profiling) return;
  // inside a stream capture the event becomes an external event record node:
  // every replay of the graph records it
  cudaEventRecordWithFlags(x->ev[group][stage][which], x->stream,
                           x->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  if (which == 1) x->ev_used[group][stage] = 1;
}

// Accumulate the recorded intervals (the stream must be synchronised).
void harvest(kh_ctx* x) {
  if (!x->profiling) return;
  for (int g = 0; g < KH_NTIMERS; ++g)
    for (int st = 0; st < 2; ++st)
      if (x->ev_used[g][st]) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, x->ev[g][st][0], x->ev[g][st][1]) == cudaSuccess) {
          x->prof_ms[g] += ms;
          x->prof_n[g] += 1;
        }
        x->ev_used[g][st] = 0;
      }
}

int check_launch(kh_ctx* x, int n) {
  x->launches += n;
  return cuda_fail(cudaGetLastError());
}

void free_all(kh_ctx* x) {
  void* ptrs[] = {x->geo, x->dgm, x->flo, x->pstar, x->F[0], x->F[1], x->F[2], x->ctop[0], x->ctop[1],
                  x->ctop[2], x->emf[0], x->emf[1], x->emf[2], x->pflag, x->partial, x->dscalar,
                  x->counters, x->dirichlet[0], x->dirichlet[1], x->geof, x->dgmf, x->pstarf, x->pnf, x->Ff[0],
                  x->Ff[1], x->Ff[2], x->ctopf[0], x->ctopf[1], x->ctopf[2], x->emff[0], x->emff[1],
                  x->emff[2], x->dirichletf[0], x->dirichletf[1], x->adj, x->adj_i8, x->adj_red, x->geodf, x->flist,
                  x->fflag, x->fsave, x->fsavef, x->fBstar, x->ecc, x->eccf, x->rk, x->rkf};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

GeomT<float> geomf(const kh_ctx* x) { return GeomT<float>{x->geof, x->dgmf, x->flo, x->geodf}; }

// One FP64 stage: ghost fill, fluxes per direction, Flux-CT, update, fixup.
int run_stage(kh_ctx* x, int st, const double* U0, const Vars& Pin, const Vars& Pout, double* Uout, double coef,
              double* dUout = nullptr) {
  const Layout& L = x->L;
  const DevGeom G = devgeom(x);
  cudaStream_t s = x->stream;
  int n = 0;
  mark(x, KH_T_BC, st, 0);
  n += launch_bc<double>(Pin, L, x->S, x->dirichlet[0], x->dirichlet[1], s);
  mark(x, KH_T_BC, st, 1);
  for (int d = 1; d <= L.ndim; ++d) {
    mark(x, KH_T_FLUX1 + d - 1, st, 0);
    n += launch_flux_dir<double, double>(d, cview(Pin), L, G, x->S, x->F[d - 1], x->ctop[d - 1], x->tpb_flux, s);
    mark(x, KH_T_FLUX1 + d - 1, st, 1);
  }
  const size_t b3 = 3 * (size_t)L.plane * sizeof(double);
  if (x->S.fofc) {
    // Flux-CT overwrites the raw field fluxes; the correction needs them again
    for (int d = 0; d < L.ndim; ++d)
      cudaMemcpyAsync(x->fsave + 3 * d * L.plane, x->F[d] + V_B1 * L.plane, b3, cudaMemcpyDeviceToDevice, s);
  }
  double* fBn = nullptr;
  if (x->S.bfield == KH_B_FACE) {
    // face-centred CT: edge EMFs from the raw fluxes move the face field;
    // the update takes the zones' field from the new faces
    fBn = x->fb_out ? x->fb_out : (st == 0 ? x->fBstar : x->fB);
    const double* fB0 = x->fb_in ? x->fb_in : x->fB;
    mark(x, KH_T_CT, st, 0);
    n += launch_face_ct<double>(cview(Pin), x->F, x->ecc, x->emf, fB0, fBn, L, G, x->S, x->dscalar + 3, coef, s);
    mark(x, KH_T_CT, st, 1);
  } else {
    mark(x, KH_T_CT, st, 0);
    n += launch_ct<double>(x->F, x->emf, L, s);
    mark(x, KH_T_CT, st, 1);
  }
  if (x->S.fofc) {
    // first-order flux correction: trial update with the high-order fluxes,
    // donor-cell fluxes on the faces of the flagged zones, Flux-CT again
    mark(x, KH_T_FOFC, st, 0);
    n += launch_fofc_trial(U0, cview(Pin), x->F, L, G, x->S, x->dscalar + 3, coef, x->fflag, x->counters,
                           x->tpb_update, s);
    n += launch_flag_ghosts(x->fflag, L, x->S, s);
    for (int d = 0; d < L.ndim; ++d)
      cudaMemcpyAsync(x->F[d] + V_B1 * L.plane, x->fsave + 3 * d * L.plane, b3, cudaMemcpyDeviceToDevice, s);
    for (int d = 1; d <= L.ndim; ++d)
      n += launch_fofc_faces<double, double>(d, cview(Pin), L, G, x->S, x->fflag, x->F[d - 1], x->ctop[d - 1],
                                             x->tpb_flux, s);
    n += launch_ct<double>(x->F, x->emf, L, s);
    mark(x, KH_T_FOFC, st, 1);
  }
  mark(x, KH_T_UPDATE, st, 0);
  const FailList fl{x->flist, x->counters + CNT_LIST0 + st, 0u};
  n += launch_update(U0, cview(Pin), Pout, Uout, x->F, L, G, x->S, x->dscalar + 3, coef, x->pflag, x->counters,
                     x->tpb_update, s, fl, fBn, dUout);
  mark(x, KH_T_UPDATE, st, 1);
  mark(x, KH_T_FIXUP, st, 0);
  n += launch_fixup<double>(Pout, Uout, x->pflag, L, G, x->S, x->counters, s, fl);
  mark(x, KH_T_FIXUP, st, 1);
  return n;
}


// One mixed stage. Stage 1 (st = 0): FP64 input, converted to FP32 with its
// ghost cells filled in FP32, read by the FP32 flux pass, output to the FP32
// shadow P*. Stage 2 (st = 1): the FP32 shadow (ghost-filled in FP32) as
// input, FP64 output and U.
template <class TIN>
int run_stage_mixed(kh_ctx* x, int st, const double* U0, const VarsT<TIN>& Pin, const TIN* dlo, const TIN* dhi,
                    const Vars& Pout64, const VarsT<float>& Pout32, double* Uout, double coef,
                    double* dUout = nullptr) {
  const Layout& L = x->L;
  const DevGeom G = devgeom(x);
  const GeomT<float> Gf = geomf(x);
  cudaStream_t s = x->stream;
  int n = 0;
  mark(x, KH_T_BC, st, 0);
  // The stencil pass reads FP32: an FP64 input is converted once per cell
  // (by integer operations; GB300 issues FP64 conversions at 1/64 the FP32
  // rate), then its ghost cells are filled from the FP64 interior straight
  // into the FP32 copy (the caller's FP64 ghosts are not needed).
  VarsT<float> Pf;
  if constexpr (sizeof(TIN) == sizeof(double)) {
    for (int q = 0; q < NV; ++q) Pf.v[q] = x->pnf + q * L.plane;
    n += launch_fill_f32(cviewT(Pin), Pf, L, x->S, dlo, dhi, s);
  } else {
    n += launch_bc<TIN>(Pin, L, x->S, dlo, dhi, s);
    Pf = Pin;
  }
  mark(x, KH_T_BC, st, 1);
  for (int d = 1; d <= L.ndim; ++d) {
    mark(x, KH_T_FLUX1 + d - 1, st, 0);
    // the stage input's 8 FP32 planes are contiguous (pnf or pstarf); a grid
    // too small for the tile's tensor box takes the per-face kernel
    int r = launch_flux_dir_tma(d, Pf.v[0], L, Gf, x->S, x->Ff[d - 1], x->ctopf[d - 1], x->counters,
                                x->wait_limit, s);
    if (r < 0)
      r = launch_flux_dir<float, float>(d, cviewT(Pf), L, Gf, x->S, x->Ff[d - 1], x->ctopf[d - 1], x->tpb_flux, s);
    n += r;
    mark(x, KH_T_FLUX1 + d - 1, st, 1);
  }
  // Flux-CT: the edge EMFs only; the update (and the correction's trial)
  // form the field fluxes from them, so the raw field fluxes stay in Ff
  const bool fct = x->S.bfield == KH_B_FLUXCT;
  double* fBn = nullptr;
  mark(x, KH_T_CT, st, 0);
  if (!fct) {
    // face-centred CT: FP32 EMFs, FP64 face field
    fBn = x->fb_out ? x->fb_out : (st == 0 ? x->fBstar : x->fB);
    const double* fB0 = x->fb_in ? x->fb_in : x->fB;
    n += launch_face_ct<float>(cviewT(Pf), x->Ff, x->eccf, x->emff, fB0, fBn, L, Gf, x->S, x->dscalar + 3, coef,
                               s);
  } else {
    n += launch_emf<float>(x->Ff, x->emff, L, s);
  }
  mark(x, KH_T_CT, st, 1);
  if (x->S.fofc) {
    // first-order flux correction (as in run_stage), FP32 fluxes; the raw
    // field fluxes were never overwritten, so the EMFs are simply redone
    mark(x, KH_T_FOFC, st, 0);
    n += launch_fofc_trial_mixed(U0, cviewT(Pf), x->Ff, L, G, Gf, x->S, x->dscalar + 3, coef, x->fflag,
                                 x->counters, x->tpb_update, s, x->emff);
    n += launch_flag_ghosts(x->fflag, L, x->S, s);
    for (int d = 1; d <= L.ndim; ++d)
      n += launch_fofc_faces<float, float>(d, cviewT(Pf), L, Gf, x->S, x->fflag, x->Ff[d - 1], x->ctopf[d - 1],
                                           x->tpb_flux, s);
    n += launch_emf<float>(x->Ff, x->emff, L, s);
    mark(x, KH_T_FOFC, st, 1);
  }
  mark(x, KH_T_UPDATE, st, 0);
  const FailList fl{x->flist, x->counters + CNT_LIST0 + st, 0u};
  // 3-D Flux-CT stages stage their inputs by TMA; otherwise (2-D, face CT,
  // or no tensor map) the update reads them itself
  int ru = -1;
  if (fct && L.ndim == 3)
    ru = launch_update_mixed_tma(U0, Pf.v[0], Pout64, Pout32, Uout, x->Ff, x->emff, L, G, Gf, x->S, x->dscalar + 3,
                                 coef, x->pflag, x->counters, fl, dUout, x->wait_limit, s);
  if (ru < 0)
    ru = launch_update_mixed(U0, cviewT(Pf), Pout64, Pout32, Uout, x->Ff, L, G, Gf, x->S, x->dscalar + 3, coef,
                             x->pflag, x->counters, x->tpb_update, s, fl, fBn, dUout, fct ? x->emff : nullptr);
  n += ru;
  mark(x, KH_T_UPDATE, st, 1);
  mark(x, KH_T_FIXUP, st, 0);
  if (Pout64.v[0])
    n += launch_fixup<double>(Pout64, Uout, x->pflag, L, G, x->S, x->counters, s, fl);
  else
    n += launch_fixup<float>(Pout32, Uout, x->pflag, L, G, x->S, x->counters, s, fl);
  mark(x, KH_T_FIXUP, st, 1);
  return n;
}

}  // namespace

extern "C" {

const char* kh_strerror(int code) {
  switch (code) {
    case KH_OK: return "success";
    case KH_EINVAL: return "invalid argument";
    case KH_ECUDA: return "CUDA runtime error";
    case KH_ENOMEM: return "device allocation failed";
    case KH_ETIMEOUT: return "bounded device wait timed out";
    case KH_ENAN: return "non-finite time step";
    default: return code > 0 ? "completed with failed inversions (repaired)" : "unknown error";
  }
}

int kh_geometry_init(double a, const kh_coords* c, double gamma, kh_ctx** out) {
  if (!c || !out) return KH_EINVAL;
  if (c->kind < KH_MINKOWSKI || c->kind > KH_FMKS) return KH_EINVAL;
  if (c->n1 < 4 || c->n2 < 4 || c->n3 < 1) return KH_EINVAL;
  if (c->recon != KH_RECON_MC && c->recon != KH_RECON_WENO5) return KH_EINVAL;
  if (c->precision != KH_FP64 && c->precision != KH_MIXED) return KH_EINVAL;
  if (c->fofc != 0 && c->fofc != 1) return KH_EINVAL;
  if (c->inverter < KH_INV_NOBLE2D || c->inverter > KH_INV_KASTAUN) return KH_EINVAL;
  if (c->integrator < KH_INT_VL2 || c->integrator > KH_INT_SSPRK54) return KH_EINVAL;
  if (c->bfield != KH_B_FLUXCT && c->bfield != KH_B_FACE) return KH_EINVAL;
  if (c->emf != KH_EMF_AVERAGE && c->emf != KH_EMF_GS05) return KH_EINVAL;
  if (c->bfield == KH_B_FACE && c->fofc) return KH_EINVAL;
  if (c->mixed_inversion != KH_MIXINV_DF && c->mixed_inversion != KH_MIXINV_FP64) return KH_EINVAL;
  if (!(gamma > 1.0) || !(c->cfl > 0.0) || !(fabs(a) < 1.0)) return KH_EINVAL;
  if (!(c->x1max > c->x1min) || !(c->x2max > c->x2min) || !(c->x3max > c->x3min)) return KH_EINVAL;
  for (int q = 0; q < 6; ++q) {
    const int b = c->bc[q];
    if (b < KH_BC_PERIODIC || b > KH_BC_DIRICHLET) return KH_EINVAL;
    if (b == KH_BC_DIRICHLET && q >= 2) return KH_EINVAL;
    if (b == KH_BC_POLAR && (q < 2 || q >= 4)) return KH_EINVAL;
  }
  if (c->kind == KH_FMKS && (c->poly_alpha != floor(c->poly_alpha) || !(c->poly_xt > 0.0))) return KH_EINVAL;
  if (c->kind == KH_MKS || c->kind == KH_FMKS) {
    if (c->x2min < -1e-12 || c->x2max > 1.0 + 1e-12) return KH_EINVAL;
  }

  kh_ctx* x = (kh_ctx*)calloc(1, sizeof(kh_ctx));
  if (!x) return KH_ENOMEM;
  x->c = *c;
  x->a = a;
  x->gam = gamma;
  x->stream = 0;
  Layout& L = x->L;
  L.n1 = c->n1; L.n2 = c->n2; L.n3 = c->n3;
  L.ng = NGHOST;
  L.ndim = c->n3 > 1 ? 3 : 2;
  L.ng3 = L.ndim == 3 ? NGHOST : 0;
  L.N1 = L.n1 + 2 * L.ng;
  L.N2 = L.n2 + 2 * L.ng;
  L.N3 = L.n3 + 2 * L.ng3;
  L.n1s = (L.N1 + 15) / 16 * 16;
  L.n2s = L.N2;
  L.n3s = L.N3;
  L.gplane = (long long)L.n1s * L.n2s;
  L.plane = L.gplane * L.n3s;
  if (L.plane >= (1LL << 31)) {  // kernels index cells with 32-bit arithmetic
    free(x);
    return KH_EINVAL;
  }
  x->tpb_flux = 128;
  x->tpb_update = 128;
  x->wait_limit = KH_WAIT_POLLS;
  L.dx[0] = (c->x1max - c->x1min) / c->n1;
  L.dx[1] = (c->x2max - c->x2min) / c->n2;
  L.dx[2] = (c->x3max - c->x3min) / c->n3;
  for (int q = 0; q < 3; ++q) {
    L.idx[q] = 1.0 / L.dx[q];
    L.idxf[q] = (float)L.idx[q];
  }
  L.s[0] = L.ng; L.e[0] = L.ng + L.n1;
  L.s[1] = L.ng; L.e[1] = L.ng + L.n2;
  L.s[2] = L.ng3; L.e[2] = L.ng3 + L.n3;

  Scheme& S = x->S;
  S.gam = gamma;
  S.igam = 1.0 / gamma;
  S.gfac = (gamma - 1.0) / gamma;
  S.cfl = c->cfl;
  S.recon = c->recon;
  S.fofc = c->fofc;
  S.integrator = c->integrator;
  S.bfield = c->bfield;
  S.emf = c->emf;
  for (int q = 0; q < 6; ++q) S.bc[q] = c->bc[q];
  S.fl.rho_min = c->rho_min;
  S.fl.u_min = c->u_min;
  S.fl.bsq_rho_max = c->bsq_rho_max;
  S.fl.bsq_u_max = c->bsq_u_max;
  S.fl.u_rho_max = c->u_rho_max;
  S.fl.gamma_max = c->gamma_max;
  S.fl.ibsq_rho_max = 1.0 / c->bsq_rho_max;
  S.fl.ibsq_u_max = 1.0 / c->bsq_u_max;
  S.c2p.max_iter = c->newton_max_iter > 0 ? c->newton_max_iter : 30;
  S.c2p.tol = c->newton_tol > 0.0 ? c->newton_tol : 1e-14;
  S.c2p.method = c->inverter;
  S.mixed_fp64 = c->precision == KH_MIXED && c->inverter == KH_INV_NOBLE2D && c->mixed_inversion == KH_MIXINV_FP64;
  set_mixed(S);

  x->cp = CoordParams{c->kind, a, c->x1min, c->hslope, c->poly_xt, c->poly_alpha, c->mks_smooth};

  const size_t pl = (size_t)L.plane * sizeof(double);
  const size_t gp = (size_t)L.gplane * sizeof(double);
  x->npartial = reduction_blocks(L);
  int rc = KH_OK;
#define KH_ALLOC(ptr, bytes)                                          \
  if (rc == KH_OK) {                                                  \
    rc = cuda_fail(cudaMalloc((void**)&(ptr), (bytes)));              \
  }
  KH_ALLOC(x->geo, 3 * NGEO * gp);
  KH_ALLOC(x->dgm, NDG * gp);
  KH_ALLOC(x->flo, 3 * gp);
  const bool mixed = c->precision == KH_MIXED;
  const size_t plf = (size_t)L.plane * sizeof(float);
  const size_t gpf = (size_t)L.gplane * sizeof(float);
  KH_ALLOC(x->pstar, NV * pl);
  if (!mixed) {
    for (int d = 0; d < L.ndim; ++d) {
      KH_ALLOC(x->F[d], NV * pl);
      KH_ALLOC(x->ctop[d], pl);
    }
    KH_ALLOC(x->emf[2], pl);
    if (L.ndim == 3 || c->bfield == KH_B_FACE) {
      KH_ALLOC(x->emf[0], pl);
      KH_ALLOC(x->emf[1], pl);
    }
  } else {
    KH_ALLOC(x->geof, 3 * NGEO * gpf);
    KH_ALLOC(x->dgmf, NDG * gpf);
    KH_ALLOC(x->geodf, 2 * NDF * gpf);
    KH_ALLOC(x->pstarf, NV * plf);
    KH_ALLOC(x->pnf, NV * plf);
    for (int d = 0; d < L.ndim; ++d) {
      KH_ALLOC(x->Ff[d], NV * plf);
      KH_ALLOC(x->ctopf[d], plf);
    }
    KH_ALLOC(x->emff[2], plf);
    if (L.ndim == 3 || c->bfield == KH_B_FACE) {
      KH_ALLOC(x->emff[0], plf);
      KH_ALLOC(x->emff[1], plf);
    }
    for (int f = 0; f < 2; ++f)
      if (c->bc[f] == KH_BC_DIRICHLET)
        KH_ALLOC(x->dirichletf[f], (size_t)NV * L.n3s * L.n2s * L.ng * sizeof(float));
  }
  KH_ALLOC(x->pflag, (size_t)L.plane);
  if (c->integrator != KH_INT_VL2) {
    // stage states, the stage base and SSPRK(5,4)'s stage-4 increment
    const int nrk = c->integrator == KH_INT_SSPRK54 ? 6 : (c->integrator == KH_INT_RK2 ? 2 : 0);
    if (nrk) KH_ALLOC(x->rk, (size_t)nrk * NV * pl);
    const int nrkf = c->integrator == KH_INT_SSPRK54 ? 5 : (c->integrator == KH_INT_RK2 ? 2 : 0);
    if (nrkf && c->bfield == KH_B_FACE) KH_ALLOC(x->rkf, (size_t)nrkf * 3 * pl);
  }
  if (c->bfield == KH_B_FACE) {
    KH_ALLOC(x->fBstar, 3 * pl);
    if (c->emf == KH_EMF_GS05) {
      if (mixed) {
        KH_ALLOC(x->eccf, 3 * plf);
      } else {
        KH_ALLOC(x->ecc, 3 * pl);
      }
    }
  }
  if (c->fofc) {
    KH_ALLOC(x->fflag, (size_t)L.plane);
    if (!mixed) KH_ALLOC(x->fsave, 3 * (size_t)L.ndim * pl);  // the mixed path keeps its raw field fluxes
  }
  KH_ALLOC(x->flist, (size_t)L.n1 * L.n2 * L.n3 * sizeof(unsigned));
  KH_ALLOC(x->partial, 2 * (size_t)x->npartial * sizeof(double));
  KH_ALLOC(x->dscalar, 4 * sizeof(double));
  KH_ALLOC(x->counters, (NCNT + 1) * sizeof(unsigned long long));  // + the bounds-check count
  for (int f = 0; f < 2; ++f)
    if (c->bc[f] == KH_BC_DIRICHLET) KH_ALLOC(x->dirichlet[f], (size_t)NV * L.n3s * L.n2s * L.ng * sizeof(double));
#undef KH_ALLOC
  if (rc == KH_OK) {
    // zero-initialise scratch so that never-written face entries are finite
    for (int d = 0; d < 3 && rc == KH_OK; ++d) {
      if (x->F[d]) rc = cuda_fail(cudaMemset(x->F[d], 0, NV * pl));
      if (rc == KH_OK && x->ctop[d]) rc = cuda_fail(cudaMemset(x->ctop[d], 0, pl));
      if (rc == KH_OK && x->emf[d]) rc = cuda_fail(cudaMemset(x->emf[d], 0, pl));
      if (rc == KH_OK && x->Ff[d]) rc = cuda_fail(cudaMemset(x->Ff[d], 0, NV * plf));
      if (rc == KH_OK && x->ctopf[d]) rc = cuda_fail(cudaMemset(x->ctopf[d], 0, plf));
      if (rc == KH_OK && x->emff[d]) rc = cuda_fail(cudaMemset(x->emff[d], 0, plf));
    }
    if (rc == KH_OK) rc = cuda_fail(cudaMemset(x->pstar, 0, NV * pl));
    if (rc == KH_OK) rc = cuda_fail(cudaMemset(x->counters, 0, (NCNT + 1) * sizeof(unsigned long long)));
    L.oob = x->counters + NCNT;
    if (rc == KH_OK && x->rkf) {
      const int nrkf = c->integrator == KH_INT_SSPRK54 ? 5 : 2;
      rc = cuda_fail(cudaMemset(x->rkf, 0, (size_t)nrkf * 3 * pl));
    }
    if (rc == KH_OK && x->pstarf) rc = cuda_fail(cudaMemset(x->pstarf, 0, NV * plf));
  }
  if (rc == KH_OK) {
    x->launches += launch_geometry(x->cp, c->x1min, c->x2min, S.fl, L, x->geo, x->dgm, x->flo, 0);
    if (mixed) {
      x->launches += launch_to_f32(x->geo, x->geof, 3LL * NGEO * L.gplane, 0);
      x->launches += launch_to_f32(x->dgm, x->dgmf, (long long)NDG * L.gplane, 0);
      x->launches += launch_df_planes(x->geo, x->flo, x->geodf, L.gplane, 0);
    }
    rc = cuda_fail(cudaGetLastError());
    if (rc == KH_OK) rc = cuda_fail(cudaDeviceSynchronize());
  }
  if (rc != KH_OK) {
    free_all(x);
    free(x);
    return rc;
  }
  *out = x;
  return KH_OK;
}

int kh_shape(const kh_ctx* x, int* n1s, int* n2s, int* n3s, int* ng) {
  if (!x) return KH_EINVAL;
  if (n1s) *n1s = x->L.n1s;
  if (n2s) *n2s = x->L.n2s;
  if (n3s) *n3s = x->L.n3s;
  if (ng) *ng = x->L.ng;
  return KH_OK;
}

int kh_set_stream(kh_ctx* x, void* s) {
  if (!x) return KH_EINVAL;
  x->stream = (cudaStream_t)s;
  return KH_OK;
}

int kh_set_dirichlet(kh_ctx* x, int face, const double* PB) {
  if (!x || face < 0 || face > 1 || !PB || !x->dirichlet[face]) return KH_EINVAL;
  const size_t bytes = (size_t)NV * x->L.n3s * x->L.n2s * x->L.ng * sizeof(double);
  KH_TRY(cudaMemcpyAsync(x->dirichlet[face], PB, bytes, cudaMemcpyDeviceToDevice, x->stream));
  if (x->dirichletf[face]) {
    x->launches += launch_to_f32(x->dirichlet[face], x->dirichletf[face],
                                 (long long)NV * x->L.n3s * x->L.n2s * x->L.ng, x->stream);
    KH_TRY(cudaGetLastError());
  }
  return KH_OK;
}

int kh_prim_to_cons(kh_ctx* x, const double* P, const double* B, double* U) {
  if (!x || !P || !B || !U) return KH_EINVAL;
  return check_launch(x, launch_p2c(cvars_of(x, P, B), U, x->L, devgeom(x), x->S, x->stream));
}

int kh_cons_to_prim(kh_ctx* x, const double* U, double* P, double* B, int8_t* pflag, int64_t* nfail) {
  if (!x || !U || !P || !B) return KH_EINVAL;
  KH_TRY(cudaMemsetAsync(x->counters, 0, NCNT * sizeof(unsigned long long), x->stream));
  int rc = check_launch(x, launch_c2p(U, vars_of(x, P, B), pflag, x->L, devgeom(x), x->S, x->counters, x->stream));
  if (rc != KH_OK) return rc;
  if (nfail) {
    unsigned long long h[NCNT];
    KH_TRY(cudaMemcpyAsync(h, x->counters, sizeof(h), cudaMemcpyDeviceToHost, x->stream));
    KH_TRY(cudaStreamSynchronize(x->stream));
    *nfail = (int64_t)h[CNT_FAIL];
    return (int)(h[CNT_FAIL] > 0x7fffffffULL ? 0x7fffffff : h[CNT_FAIL]);
  }
  return KH_OK;
}

int kh_fill_ghosts(kh_ctx* x, double* P, double* B) {
  if (!x || !P || !B) return KH_EINVAL;
  return check_launch(x, launch_bc<double>(vars_of(x, P, B), x->L, x->S, x->dirichlet[0], x->dirichlet[1], x->stream));
}

int kh_fluxes(kh_ctx* x, const double* P, const double* B, double* F1, double* F2, double* F3) {
  if (!x || !P || !B || !F1 || !F2 || (x->L.ndim == 3 && !F3)) return KH_EINVAL;
  if (x->c.precision != KH_FP64) return KH_EINVAL;  // FP64 diagnostic
  double* const F[3] = {F1, F2, x->L.ndim == 3 ? F3 : x->F[2]};
  int n = 0;
  for (int d = 1; d <= x->L.ndim; ++d)
    n += launch_flux_dir<double, double>(d, cvars_of(x, P, B), x->L, devgeom(x), x->S, F[d - 1], x->ctop[d - 1],
                                         x->tpb_flux, x->stream);
  n += launch_ct<double>(F, x->emf, x->L, x->stream);
  return check_launch(x, n);
}

}  // extern "C"

namespace {

// One Runge-Kutta step (FP64, Flux-CT) in Shu-Osher form: stage s forms its
// base sum_j a_sj U_j (k_lincomb) and runs the predictor-corrector's stage
// with coefficient c_s (run_stage: U_s = base + c_s dt L(P), inversion in
// place on P -- every kernel that reads the stage input runs before the
// update overwrites it). Stage states live in x->rk (8 planes each), then
// the base (8 planes) and SSPRK(5,4)'s stage-4 increment (8 planes).
//   RK1: U1 = U0 + dt L.  RK2: U1 = U0 + dt L; U2 = (U0 + U1)/2 + dt/2 L.
//   SSPRK(5,4) (Spiteri & Ruuth 2002): the published five-stage table, the
//   fifth stage reusing stage 4's raw increment c4 dt L(P3).
int issue_rk(kh_ctx* x, double* U, const Vars& Pn) {
  const Layout& L = x->L;
  cudaStream_t s = x->stream;
  const long long n8 = (long long)NV * L.plane;
  double* st[5] = {U, x->rk, x->rk + n8, x->rk + 2 * n8, x->rk + 3 * n8};
  const int nst = x->S.integrator == KH_INT_SSPRK54 ? 4 : (x->S.integrator == KH_INT_RK2 ? 1 : 0);
  double* base = x->rk + nst * n8;
  double* dU4 = base + n8;
  int n = 0;
  const int nstage = x->S.integrator == KH_INT_SSPRK54 ? 5 : (x->S.integrator == KH_INT_RK2 ? 2 : 1);
  auto stage = [&](int q, const double* U0, double* Uout, double c, double* dUout) {
    // each stage appends to the failed-zone list of slot q % 2: start it empty
    cudaMemsetAsync(x->counters + CNT_LIST0 + (q % 2), 0, sizeof(unsigned long long), s);
    if (x->c.precision == KH_FP64) {
      n += run_stage(x, q % 2, U0, Pn, Pn, Uout, c, dUout);
      return;
    }
    // mixed: the FP64 P^n enters the first stage, the FP32 shadow the later
    // ones (in place); the last stage writes the FP64 P^{n+1}
    VarsT<float> Psf, nof;
    Vars no64;
    for (int v = 0; v < NV; ++v) {
      Psf.v[v] = x->pstarf + v * L.plane;
      nof.v[v] = nullptr;
      no64.v[v] = nullptr;
    }
    const bool last = q == nstage - 1;
    if (q == 0)
      n += run_stage_mixed<double>(x, 0, U0, Pn, x->dirichlet[0], x->dirichlet[1], last ? Pn : no64,
                                   last ? nof : Psf, Uout, c, dUout);
    else
      n += run_stage_mixed<float>(x, q % 2, U0, Psf, x->dirichletf[0], x->dirichletf[1], last ? Pn : no64,
                                  last ? nof : Psf, Uout, c, dUout);
  };
  auto comb = [&](int nt, const double* const* in, const double* a) {
    n += launch_lincomb(base, nt, in, a, n8, s);
  };
  // face-centred CT: the face field's stage states (fs[0] = the caller's
  // field, the last stage writes it) and base, combined with the same
  // weights; SSPRK(5,4)'s fifth stage takes stage 4's face increment as
  // stage 4's output minus its base
  const bool face = x->S.bfield == KH_B_FACE;
  const long long n3 = 3 * (long long)L.plane;
  double* fs[5] = {x->fB, nullptr, nullptr, nullptr, nullptr};
  double* fbase = nullptr;
  if (face && x->rkf) {
    for (int q = 1; q <= nst; ++q) fs[q] = x->rkf + (q - 1) * n3;
    fbase = x->rkf + nst * n3;
  }
  auto fcomb = [&](int nt, const double* const* in, const double* a) {
    if (face) n += launch_lincomb(fbase, nt, in, a, n3, s);
  };
  auto faces = [&](const double* in, double* out) {
    x->fb_in = face ? in : nullptr;
    x->fb_out = face ? out : nullptr;
  };
  if (x->S.integrator == KH_INT_RK1) {
    faces(x->fB, x->fB);
    stage(0, U, U, 1.0, nullptr);
  } else if (x->S.integrator == KH_INT_RK2) {
    faces(x->fB, fs[1]);
    stage(0, U, st[1], 1.0, nullptr);
    const double* in[2] = {U, st[1]};
    const double a[2] = {0.5, 0.5};
    comb(2, in, a);
    const double* fin[2] = {fs[0], fs[1]};
    fcomb(2, fin, a);
    faces(fbase, x->fB);
    stage(1, base, U, 0.5, nullptr);
  } else {
    using T = Ssprk54;
    faces(x->fB, fs[1]);
    stage(0, U, st[1], T::c1, nullptr);
    // stages 2-4 combine U (and fB) with the previous stage's state
    for (int q = 1; q <= 3; ++q) {
      const double* in[2] = {U, st[q]};
      comb(2, in, T::a[q - 1]);
      const double* fin[2] = {fs[0], fs[q]};
      fcomb(2, fin, T::a[q - 1]);
      faces(fbase, fs[q + 1]);
      stage(q, base, st[q + 1], T::c[q - 1], q == 3 ? dU4 : nullptr);
    }
    {
      const double a[4] = {T::a5[0], T::a5[1], T::a5[2], T::c53 / T::c[2]};
      const double* in[4] = {st[2], st[3], st[4], dU4};
      comb(4, in, a);
      // fbase still holds stage 4's base: fs4 - fbase is stage 4's increment
      const double fa[4] = {a[0], a[1], a[2] + a[3], -a[3]};
      const double* fin[4] = {fs[2], fs[3], fs[4], fbase};
      fcomb(4, fin, fa);
      faces(fbase, x->fB);
      stage(4, base, U, T::c5, nullptr);
    }
  }
  faces(nullptr, nullptr);
  return n;
}

// Issue the launches of one full step on x->stream (dt is read from
// x->dscalar[3] by the update kernels).
int issue_step(kh_ctx* x, double* U, double* P, double* B) {
  const Layout& L = x->L;
  cudaStream_t s = x->stream;
  if (cudaMemsetAsync(x->counters, 0, NCNT * sizeof(unsigned long long), s) != cudaSuccess) return -1;
  Vars Pn = vars_of(x, P, B);
  Vars Ps;
  for (int q = 0; q < NV; ++q) Ps.v[q] = x->pstar + q * L.plane;
  int n = 0;
  if (x->c.precision == KH_FP64) {
    // stage 1: P^n -> P* (U* is not stored); stage 2: P* -> P^{n+1}, U^{n+1} in place
    if (x->S.integrator != KH_INT_VL2) {
      const int r = issue_rk(x, U, Pn);
      if (r < 0) return r;
      n += r;
    } else {
      n += run_stage(x, 0, U, Pn, Ps, nullptr, 0.5);
      n += run_stage(x, 1, U, Ps, Pn, U, 1.0);
    }
    mark(x, KH_T_CFL, 1, 0);
    n += launch_cfl<double>(x->ctop, L, x->S.cfl, x->partial, x->npartial, x->dscalar, s);
    mark(x, KH_T_CFL, 1, 1);
  } else {
    // stage 1: FP64 P^n -> FP32 shadow P*; stage 2: FP32 P* -> FP64 P^{n+1}, U^{n+1}
    VarsT<float> Psf, nof;
    Vars no64;
    for (int q = 0; q < NV; ++q) {
      Psf.v[q] = x->pstarf + q * L.plane;
      nof.v[q] = nullptr;
      no64.v[q] = nullptr;
    }
    if (x->S.integrator != KH_INT_VL2) {
      const int r = issue_rk(x, U, Pn);
      if (r < 0) return r;
      n += r;
    } else {
      n += run_stage_mixed<double>(x, 0, U, Pn, x->dirichlet[0], x->dirichlet[1], no64, Psf, nullptr, 0.5);
      n += run_stage_mixed<float>(x, 1, U, Psf, x->dirichletf[0], x->dirichletf[1], Pn, nof, U, 1.0);
    }
    mark(x, KH_T_CFL, 1, 0);
    n += launch_cfl<float>(x->ctopf, L, x->S.cfl, x->partial, x->npartial, x->dscalar, s);
    mark(x, KH_T_CFL, 1, 1);
  }
  return n;
}

void drop_graph(kh_ctx* x) {
  if (x->gexec) cudaGraphExecDestroy(x->gexec);
  x->gexec = nullptr;
  x->gkey[0] = x->gkey[1] = x->gkey[2] = nullptr;
}

// Capture the step for these pointers (once) and replay it. A step captured
// while profiling records the group events on every replay (their set is
// handed to harvest after each launch).
int step_graph(kh_ctx* x, double* U, double* P, double* B) {
  if (!(x->gexec && x->gkey[0] == U && x->gkey[1] == P && x->gkey[2] == B && x->gprof == x->profiling)) {
    drop_graph(x);
    if (!x->cap_stream && cudaStreamCreateWithFlags(&x->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return KH_ECUDA;
    cudaStream_t user = x->stream;
    x->stream = x->cap_stream;
    if (cudaStreamBeginCapture(x->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      x->stream = user;
      return KH_ECUDA;
    }
    x->capturing = 1;
    const int n = issue_step(x, U, P, B);
    x->capturing = 0;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(x->cap_stream, &g);
    x->stream = user;
    for (int q = 0; q < KH_NTIMERS; ++q)
      for (int st = 0; st < 2; ++st) {
        x->gev_used[q][st] = x->ev_used[q][st];
        x->ev_used[q][st] = 0;
      }
    if (n < 0 || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      return KH_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&x->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      x->gexec = nullptr;
      return KH_ECUDA;
    }
    x->gkey[0] = U;
    x->gkey[1] = P;
    x->gkey[2] = B;
    x->gprof = x->profiling;
    x->graph_launches = n;
  }
  if (cudaGraphLaunch(x->gexec, x->stream) != cudaSuccess) return KH_ECUDA;
  x->launches += x->graph_launches;
  if (x->profiling)
    for (int q = 0; q < KH_NTIMERS; ++q)
      for (int st = 0; st < 2; ++st) x->ev_used[q][st] = x->gev_used[q][st];
  return KH_OK;
}

}  // namespace

extern "C" {

int kh_step(kh_ctx* x, double* U, double* P, double* B, double dt, double* dt_cfl) {
  if (!x || !U || !P || !B || !(dt > 0.0) || !isfinite(dt)) return KH_EINVAL;
  if (x->S.bfield == KH_B_FACE && !x->fB) return KH_EINVAL;  // no face field registered
  // dt enters through device memory (a pageable copy: the host value may be
  // reused as soon as the call returns)
  KH_TRY(cudaMemcpyAsync(x->dscalar + 3, &dt, sizeof(double), cudaMemcpyHostToDevice, x->stream));
  int rc;
  if (x->graph_on) {
    rc = step_graph(x, U, P, B);
    if (rc != KH_OK) return rc;
    rc = cuda_fail(cudaGetLastError());
  } else {
    const int n = issue_step(x, U, P, B);
    if (n < 0) return KH_ECUDA;
    rc = check_launch(x, n);
  }
  if (rc != KH_OK) return rc;
  if (!dt_cfl && !x->profiling) return KH_OK;
  kh_stats st;
  rc = kh_get_stats(x, &st);
  if (rc != KH_OK) return rc;
  harvest(x);
  if (!dt_cfl) return KH_OK;
  *dt_cfl = st.dt_cfl;
  if (!isfinite(st.dt_cfl)) return KH_ENAN;
  return (int)(st.nfail > 0x7fffffffLL ? 0x7fffffff : st.nfail);
}

int kh_pack_state(kh_ctx* x, const double* U, const double* P, const double* B, double* out) {
  if (!x || !U || !P || !B || !out) return KH_EINVAL;
  return check_launch(x, launch_pack(U, cvars_of(x, P, B), out, x->L, x->stream));
}

int kh_unpack_state(kh_ctx* x, const double* in, double* U, double* P, double* B) {
  if (!x || !in || !U || !P || !B) return KH_EINVAL;
  return check_launch(x, launch_unpack(in, U, vars_of(x, P, B), x->L, x->stream));
}

int kh_set_face_field(kh_ctx* x, double* fB) {
  if (!x || !fB || x->S.bfield != KH_B_FACE) return KH_EINVAL;
  if (x->fB != fB) drop_graph(x);  // a captured step holds the old pointer
  x->fB = fB;
  if (cudaMemsetAsync(x->fBstar, 0, 3 * (size_t)x->L.plane * sizeof(double), x->stream) != cudaSuccess)
    return KH_ECUDA;
  return KH_OK;
}

int kh_face_to_cell(kh_ctx* x, const double* fB, double* B) {
  if (!x || !fB || !B) return KH_EINVAL;
  return check_launch(x, launch_face_to_cell(fB, B, x->L, devgeom(x), x->stream));
}

int kh_face_divb(kh_ctx* x, const double* fB, double* max_abs, double* l1) {
  if (!x || !fB) return KH_EINVAL;
  const Layout& L = x->L;
  int rc = check_launch(x, launch_face_divb(fB, L, x->partial, x->npartial, x->dscalar + 1, x->stream));
  if (rc != KH_OK) return rc;
  double h[2];
  KH_TRY(cudaMemcpyAsync(h, x->dscalar + 1, sizeof(h), cudaMemcpyDeviceToHost, x->stream));
  KH_TRY(cudaStreamSynchronize(x->stream));
  const double nz = (double)L.n1 * L.n2 * L.n3;
  if (max_abs) *max_abs = h[0];
  if (l1) *l1 = h[1] / nz;
  return KH_OK;
}

int kh_set_graph(kh_ctx* x, int enable) {
  if (!x) return KH_EINVAL;
  if (!enable) drop_graph(x);
  x->graph_on = enable ? 1 : 0;
  return KH_OK;
}

int kh_set_launch(kh_ctx* x, int tpb_flux, int tpb_update) {
  if (!x) return KH_EINVAL;
  const int ok[4] = {32, 64, 128, 256};
  bool f = false, u = false;
  for (int q = 0; q < 4; ++q) {
    f = f || tpb_flux == ok[q];
    u = u || tpb_update == ok[q];
  }
  if (!f || !u) return KH_EINVAL;
  x->tpb_flux = tpb_flux;
  x->tpb_update = tpb_update;
  drop_graph(x);
  return KH_OK;
}

int kh_get_launch(const kh_ctx* x, int* tpb_flux, int* tpb_update) {
  if (!x) return KH_EINVAL;
  if (tpb_flux) *tpb_flux = x->tpb_flux;
  if (tpb_update) *tpb_update = x->tpb_update;
  return KH_OK;
}

int kh_autotune(kh_ctx* x, const double* U, const double* P, const double* B, double dt, int* tpb_flux,
                int* tpb_update) {
  if (!x || !U || !P || !B || !(dt > 0.0)) return KH_EINVAL;
  // process-wide cache: one search per (grid, coordinates, reconstruction, precision)
  static std::mutex lock;
  static std::map<std::tuple<int, int, int, int, int, int>, std::pair<int, int>> cache;
  const auto key = std::make_tuple(x->L.n1, x->L.n2, x->L.n3, x->c.kind, x->c.recon, x->c.precision);
  {
    std::lock_guard<std::mutex> g(lock);
    auto it = cache.find(key);
    if (it != cache.end()) {
      const int rc = kh_set_launch(x, it->second.first, it->second.second);
      if (tpb_flux) *tpb_flux = x->tpb_flux;
      if (tpb_update) *tpb_update = x->tpb_update;
      return rc;
    }
  }
  const Layout& L = x->L;
  const size_t pl = (size_t)L.plane * sizeof(double);
  double *Us = nullptr, *Ps = nullptr, *Bs = nullptr;
  int rc = cuda_fail(cudaMalloc((void**)&Us, 8 * pl));
  if (rc == KH_OK) rc = cuda_fail(cudaMalloc((void**)&Ps, 5 * pl));
  if (rc == KH_OK) rc = cuda_fail(cudaMalloc((void**)&Bs, 3 * pl));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == KH_OK) rc = cuda_fail(cudaEventCreate(&e0));
  if (rc == KH_OK) rc = cuda_fail(cudaEventCreate(&e1));
  const int graph = x->graph_on, prof = x->profiling;
  x->graph_on = 0;
  x->profiling = 0;
  const int cand[3] = {64, 128, 256};
  float best = 1e30f;
  int bf = x->tpb_flux, bu = x->tpb_update;
  for (int a = 0; a < 3 && rc == KH_OK; ++a)
    for (int b = 0; b < 3 && rc == KH_OK; ++b) {
      x->tpb_flux = cand[a];
      x->tpb_update = cand[b];
      float ms = 0.0f;
      // one untimed step, then two timed steps, each from the caller's state
      for (int rep = 0; rep < 3 && rc == KH_OK; ++rep) {
        rc = cuda_fail(cudaMemcpyAsync(Us, U, 8 * pl, cudaMemcpyDeviceToDevice, x->stream));
        if (rc == KH_OK) rc = cuda_fail(cudaMemcpyAsync(Ps, P, 5 * pl, cudaMemcpyDeviceToDevice, x->stream));
        if (rc == KH_OK) rc = cuda_fail(cudaMemcpyAsync(Bs, B, 3 * pl, cudaMemcpyDeviceToDevice, x->stream));
        if (rc == KH_OK) rc = cuda_fail(cudaEventRecord(e0, x->stream));
        if (rc == KH_OK) {
          const int r = kh_step(x, Us, Ps, Bs, dt, nullptr);
          rc = r < 0 ? r : KH_OK;
        }
        if (rc == KH_OK) rc = cuda_fail(cudaEventRecord(e1, x->stream));
        if (rc == KH_OK) rc = cuda_fail(cudaEventSynchronize(e1));
        float t = 0.0f;
        if (rc == KH_OK && rep > 0 && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms += t;
      }
      if (rc == KH_OK && ms < best) {
        best = ms;
        bf = cand[a];
        bu = cand[b];
      }
    }
  x->tpb_flux = bf;
  x->tpb_update = bu;
  x->graph_on = graph;
  x->profiling = prof;
  drop_graph(x);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (Us) cudaFree(Us);
  if (Ps) cudaFree(Ps);
  if (Bs) cudaFree(Bs);
  if (rc != KH_OK) return rc;
  {
    std::lock_guard<std::mutex> g(lock);
    cache[key] = std::make_pair(bf, bu);
  }
  if (tpb_flux) *tpb_flux = bf;
  if (tpb_update) *tpb_update = bu;
  return KH_OK;
}

int kh_profile(kh_ctx* x, int enable) {
  if (!x) return KH_EINVAL;
  if ((enable ? 1 : 0) != x->profiling) drop_graph(x);  // a captured step holds the events (or none)
  if (enable && !x->profiling) {
    for (int g = 0; g < KH_NTIMERS; ++g)
      for (int st = 0; st < 2; ++st)
        for (int w = 0; w < 2; ++w) KH_TRY(cudaEventCreate(&x->ev[g][st][w]));
  }
  if (!enable && x->profiling) {
    for (int g = 0; g < KH_NTIMERS; ++g)
      for (int st = 0; st < 2; ++st)
        for (int w = 0; w < 2; ++w) cudaEventDestroy(x->ev[g][st][w]);
  }
  x->profiling = enable ? 1 : 0;
  for (int g = 0; g < KH_NTIMERS; ++g) {
    x->prof_ms[g] = 0.0;
    x->prof_n[g] = 0;
    x->ev_used[g][0] = x->ev_used[g][1] = 0;
  }
  return KH_OK;
}

int kh_profile_read(const kh_ctx* x, double* ms, int64_t* count) {
  if (!x) return KH_EINVAL;
  for (int g = 0; g < KH_NTIMERS; ++g) {
    if (ms) ms[g] = x->prof_ms[g];
    if (count) count[g] = x->prof_n[g];
  }
  return KH_OK;
}

int kh_get_stats(kh_ctx* x, kh_stats* out) {
  if (!x || !out) return KH_EINVAL;
  unsigned long long h[NCNT + 1];
  double dt;
  KH_TRY(cudaMemcpyAsync(h, x->counters, sizeof(h), cudaMemcpyDeviceToHost, x->stream));
  KH_TRY(cudaMemcpyAsync(&dt, x->dscalar, sizeof(double), cudaMemcpyDeviceToHost, x->stream));
  KH_TRY(cudaStreamSynchronize(x->stream));
  out->nfail = (int64_t)h[CNT_FAIL];
  out->nfloor = (int64_t)h[CNT_FLOOR];
  out->nunfixed = (int64_t)h[CNT_UNFIXED];
  out->nfp64 = (int64_t)h[CNT_FP64];
  out->nfofc = (int64_t)h[CNT_FOFC];
  out->nbounds = (int64_t)h[NCNT];
  out->dt_cfl = dt;
  x->last = *out;
  return h[CNT_TIMEOUT] ? KH_ETIMEOUT : KH_OK;
}

int kh_cfl_dt(kh_ctx* x, const double* P, const double* B, double* dt_cfl) {
  if (!x || !P || !B || !dt_cfl) return KH_EINVAL;
  const Layout& L = x->L;
  cudaStream_t s = x->stream;
  const size_t pl = (size_t)L.plane * sizeof(double);
  KH_TRY(cudaMemcpyAsync(x->pstar, P, 5 * pl, cudaMemcpyDeviceToDevice, s));
  KH_TRY(cudaMemcpyAsync(x->pstar + 5 * L.plane, B, 3 * pl, cudaMemcpyDeviceToDevice, s));
  Vars Ps;
  for (int q = 0; q < NV; ++q) Ps.v[q] = x->pstar + q * L.plane;
  int n = launch_bc<double>(Ps, L, x->S, x->dirichlet[0], x->dirichlet[1], s);
  if (x->c.precision == KH_FP64) {
    for (int d = 1; d <= L.ndim; ++d)
      n += launch_flux_dir<double, double>(d, cview(Ps), L, devgeom(x), x->S, x->F[d - 1], x->ctop[d - 1],
                                           x->tpb_flux, s);
    n += launch_cfl<double>(x->ctop, L, x->S.cfl, x->partial, x->npartial, x->dscalar, s);
  } else {
    for (int d = 1; d <= L.ndim; ++d)
      n += launch_flux_dir<double, float>(d, cview(Ps), L, geomf(x), x->S, x->Ff[d - 1], x->ctopf[d - 1],
                                          x->tpb_flux, s);
    n += launch_cfl<float>(x->ctopf, L, x->S.cfl, x->partial, x->npartial, x->dscalar, s);
  }
  int rc = check_launch(x, n);
  if (rc != KH_OK) return rc;
  KH_TRY(cudaMemcpyAsync(dt_cfl, x->dscalar, sizeof(double), cudaMemcpyDeviceToHost, s));
  KH_TRY(cudaStreamSynchronize(s));
  return isfinite(*dt_cfl) ? KH_OK : KH_ENAN;
}

int kh_divb(kh_ctx* x, const double* B, double* max_abs, double* l1) {
  if (!x || !B) return KH_EINVAL;
  const Layout& L = x->L;
  const double* Bp[3] = {B, B + L.plane, B + 2 * L.plane};
  int rc = check_launch(x, launch_divb(Bp, L, devgeom(x), x->partial, x->npartial, x->dscalar + 1, x->stream));
  if (rc != KH_OK) return rc;
  double h[2];
  KH_TRY(cudaMemcpyAsync(h, x->dscalar + 1, sizeof(h), cudaMemcpyDeviceToHost, x->stream));
  KH_TRY(cudaStreamSynchronize(x->stream));
  long long ncorner = (long long)(L.n1 - 1) * (L.n2 - 1) * (L.ndim == 3 ? (L.n3 - 1) : 1);
  if (max_abs) *max_abs = h[0];
  if (l1) *l1 = ncorner > 0 ? h[1] / (double)ncorner : 0.0;
  return KH_OK;
}

int64_t kh_launch_count(const kh_ctx* x) { return x ? (int64_t)x->launches : 0; }

int kh_set_wait_limit(kh_ctx* x, unsigned polls) {
  if (!x) return KH_EINVAL;
  if (polls != x->wait_limit) drop_graph(x);  // a captured step holds the old limit
  x->wait_limit = polls;
  return KH_OK;
}

int kh_destroy(kh_ctx* x) {
  if (!x) return KH_EINVAL;
  cudaStreamSynchronize(x->stream);
  drop_graph(x);
  if (x->cap_stream) cudaStreamDestroy(x->cap_stream);
  if (x->profiling) kh_profile(x, 0);
  free_all(x);
  free(x);
  return KH_OK;
}

}  // extern "C"
