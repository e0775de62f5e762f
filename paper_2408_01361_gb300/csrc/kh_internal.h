// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kh_mixed.cuh"  // kh_physics.cuh and the double-float update
#include "kharma_gb300.h"

namespace kh {

constexpr int NGHOST = 3;
// Piecewise-constant (donor-cell) reconstruction: the first-order fluxes of
// the flux correction (not a user-selectable scheme)
constexpr int RECON_DONOR = 2;
constexpr int NGEO = 22;  // per location: gcov (10 symmetric), gcon (10), gdet, alpha
constexpr int NDG = 20;  // d_1 g_{mn}, d_2 g_{mn}: 2 x 10 symmetric pairs (cell centres)
enum { LOC_CENT = 0, LOC_F1 = 1, LOC_F2 = 2 };

struct Layout {
  int n1, n2, n3, ng, ng3, ndim;
  int n1s, n2s, n3s;  // allocation extents
  int N1, N2, N3;     // ghosted extents (N1 <= n1s)
  long long plane;    // n1s * n2s * n3s
  long long gplane;   // n1s * n2s
  double dx[3];
  double idx[3];      // 1 / dx
  float idxf[3];      // the same, FP32 (mixed update)
  int s[3], e[3];     // interior [s, e) per direction (i, j, k)
  // bounds-checked builds (KH_BOUNDS_CHECK): counter of refused accesses
  unsigned long long* oob = nullptr;
  KH_HD long long at(int k, int j, int i) const { return ((long long)k * n2s + j) * n1s + i; }
};

// Bounds-checked builds (-DKH_BOUNDS_CHECK; the variant the tests build
// beside the release library, standing in for a memory checker): before a
// kernel touches the cells of its work item it checks them against the
// allocation; on a violation it counts it in *L.oob (kh_stats.nbounds) and
// skips the item instead of reading or writing out of bounds. Release builds
// compile the checks away (KH_OOB is false).
#ifdef KH_BOUNDS_CHECK
#define KH_OOB(L, ok) (!(ok) ? (((L).oob ? atomicAdd((L).oob, 1ULL) : 0ULL), true) : false)
#else
#define KH_OOB(L, ok) false
#endif

// The box [i - r, i + r] x [j - r, j + r] x [k - r, k + r] (k only in 3-D)
// lies inside the allocation.
KH_HD bool kh_in(const Layout& L, int i, int j, int k, int r) {
  const int r3 = L.ndim == 3 ? r : 0;
  return i - r >= 0 && i + r < L.n1s && j - r >= 0 && j + r < L.n2s && k - r3 >= 0 && k + r3 < L.n3s;
}

// The stencil [lo, hi] cells along x^D of cell (i, j, k) lies inside the
// allocation.
KH_HD bool kh_in_dir(const Layout& L, int D, int i, int j, int k, int lo, int hi) {
  const int a[3] = {D == 1 ? lo : 0, D == 2 ? lo : 0, D == 3 ? lo : 0};
  const int b[3] = {D == 1 ? hi : 0, D == 2 ? hi : 0, D == 3 ? hi : 0};
  return i + a[0] >= 0 && i + b[0] < L.n1s && j + a[1] >= 0 && j + b[1] < L.n2s && k + a[2] >= 0 &&
         k + b[2] < L.n3s;
}

// Pointers to the 8 primitive planes (5 fluid + 3 field) of one state.
template <class T> struct VarsT {
  T* v[NV];
};
template <class T> struct CVarsT {
  const T* v[NV];
};
using Vars = VarsT<double>;
using CVars = CVarsT<double>;

// Geometry cache in precision T (the FP64 cache and its FP32 copy).
template <class T> struct GeomT {
  const T* g;          // [3][NGEO][n2s][n1s]
  const T* dgm;        // [NDG][n2s][n1s]: metric derivatives in x1 and x2 at cell centres
  const double* flo;   // [3][n2s][n1s]: geometric floors of rho and u, and 1/sqrt(-g), at cell centres
  const float* df;     // FP32 copy only: [NDF][n2s][n1s] double-float (hi, lo) pairs (above)
};
using DevGeom = GeomT<double>;

struct Scheme {
  double gam;
  double igam;  // 1 / gam
  double gfac;  // (gam - 1) / gam
  double cfl;
  int recon;
  int fofc;  // first-order flux correction on
  int bfield; // KH_B_FLUXCT | KH_B_FACE
  int integrator;  // KH_INT_*
  int emf;    // KH_EMF_AVERAGE | KH_EMF_GS05 (face CT)
  int bc[6];
  FloorParams fl;
  C2POpts c2p;
  MixedConsts mx;
  int mixed_fp64;  // KH_MIXED, Noble-2D: every zone inverted in FP64 (kh_coords.mixed_inversion)
};

// Kernel template id of the mixed update's FP64 Noble-2D for every zone (not a
// solver of its own: the FP64 noble2d, entered without the double-float try).
constexpr int C2P_NOBLE2D_FP64 = 3;

// Host: fill S.mx from the FP64 fields.
inline void set_mixed(Scheme& S) { S.mx = mixed_consts(S.gam, S.fl); }

// Counters kept on the device for one step.
// CNT_FP64: zones of the mixed update whose inversion fell back to FP64;
// CNT_LIST0/1: lengths of the failed-zone lists of stages 1 and 2
// CNT_FOFC: zones flagged by the first-order flux correction's trials
// CNT_TIMEOUT: CTAs whose bounded wait for their TMA tile gave up;
// CNT_DRAIN: ... of those, CTAs whose copy had not landed after the drain wait
// (the slot after the NCNT per-step counters holds the bounds-checked
// build's count of refused accesses, kept for the context's life)
enum { CNT_FAIL = 0, CNT_FLOOR = 1, CNT_UNFIXED = 2, CNT_TIMEOUT = 3, CNT_FP64 = 4, CNT_LIST0 = 5, CNT_LIST1 = 6,
       CNT_FOFC = 7, CNT_DRAIN = 8, NCNT = 9 };

// Cells (L.at index) whose inversion failed in one stage, appended by the
// update (idx == nullptr: not recorded) as tag | cell; the fixup then visits
// these only. The single grid's tag is 0; the refined mesh's carries the
// block (block << 20, every block's allocation holding fewer than 2^20 cells).
struct FailList {
  unsigned* idx;
  unsigned long long* n;
  unsigned tag;
};

// SSPRK(5,4) of Spiteri & Ruuth (2002) in Shu-Osher form (the paper's
// "Algorithm" section lists it beside RK1, RK2 and the predictor-corrector):
// U1 = U + c1 dt L(P); U_{q+1} = a[q-1][0] U + a[q-1][1] U_q + c[q-1] dt L(P_q)
// for q = 1..3; U5 = a5[0] U2 + a5[1] U3 + a5[2] U4 + (c53 / c[2]) dU4 + c5 dt
// L(P4), where dU4 = c[2] dt L(P3) is stage 4's raw increment.
struct Ssprk54 {
  static constexpr double c1 = 0.391752226571890;
  static constexpr double a[3][2] = {{0.444370493651235, 0.555629506348765},
                                     {0.620101851488403, 0.379898148511597},
                                     {0.178079954393132, 0.821920045606868}};
  static constexpr double c[3] = {0.368410593050371, 0.251891774271694, 0.544974750228521};
  static constexpr double a5[3] = {0.517231671970585, 0.096059710526147, 0.386708617503269};
  static constexpr double c53 = 0.063692468666290;
  static constexpr double c5 = 0.226007483236906;
};

// ---- launchers (kh_kernels.cu); each returns the number of kernels launched ----
// Geometry of a grid whose first interior cell starts at native (x1o, x2o);
// cp.x1min is the FMKS blending reference (the x1 start of the whole domain).
int launch_geometry(const CoordParams& cp, double x1o, double x2o, const FloorParams& fl, const Layout& L, double* geo,
                    double* dgm, double* flo, cudaStream_t s);
template <class T> inline CVarsT<T> cviewT(const VarsT<T>& v) {
  CVarsT<T> c;
  for (int q = 0; q < NV; ++q) c.v[q] = v.v[q];
  return c;
}

// Ghost fill in place (one kernel: the x1, x2, x3 rules composed per cell).
template <class T>
int launch_bc(const VarsT<T>& P, const Layout& L, const Scheme& S, const T* dlo, const T* dhi, cudaStream_t s);
// The same map reading interior cells of src and writing the ghost cells of
// dst (FP64 -> FP32 for the mixed path's stage-1 input).
template <class TS, class TD>
int launch_bc_fill(const CVarsT<TS>& src, const VarsT<TD>& dst, const Layout& L, const Scheme& S, const TS* dlo,
                   const TS* dhi, cudaStream_t s);
// Reconstruction + LLF through x^D faces: stencil read in TIN, arithmetic and
// outputs in R (FP64 path: double/double; mixed: double or float in, float out).
// FP32 face fluxes from TMA-staged shared-memory tiles (kh_flux_tma.cu): P8
// is the 8-plane FP32 stage input; wlim bounds the polls of a CTA's wait for
// its tile (0: give up before the first poll); returns -1 if the tensor map
// cannot be encoded.
int launch_flux_dir_tma(int D, const float* P8, const Layout& L, const GeomT<float>& G, const Scheme& S, float* F,
                        float* ctop, unsigned long long* cnt, unsigned wlim, cudaStream_t s);
template <class TIN, class R>
int launch_flux_dir(int D, const CVarsT<TIN>& P, const Layout& L, const GeomT<R>& G, const Scheme& S, R* F, R* ctop,
                    int tpb, cudaStream_t s);
template <class R> int launch_ct(R* const F[3], R* const emf[3], const Layout& L, cudaStream_t s);
// Flux-CT's edge EMFs only (the field fluxes left raw; the mixed update forms
// its field fluxes from the EMFs).
template <class R> int launch_emf(R* const F[3], R* const emf[3], const Layout& L, cudaStream_t s);
// First-order flux correction (after Beckwith & Stone 2011). The trial: the
// FP64 update of every interior zone with the post-CT fluxes, writing only
// flag[c] (1: inversion failed or a floor acted); then the flags' ghost
// cells by the ghost map of the state (Dirichlet ghosts 0).
int launch_fofc_trial(const double* U0, const CVars& Pin, double* const F[3], const Layout& L, const DevGeom& G,
                      const Scheme& S, const double* dtp, double coef, int8_t* flag, unsigned long long* cnt,
                      int tpb, cudaStream_t s);
// The same trial with the mixed update (FP32 fluxes; Gf the FP32 geometry).
int launch_fofc_trial_mixed(const double* U0, const CVarsT<float>& Pin, float* const F[3], const Layout& L,
                            const DevGeom& G, const GeomT<float>& Gf, const Scheme& S, const double* dtp, double coef,
                            int8_t* flag, unsigned long long* cnt, int tpb, cudaStream_t s,
                            float* const* emf = nullptr);
int launch_flag_ghosts(int8_t* flag, const Layout& L, const Scheme& S, cudaStream_t s);
// Donor-cell LLF fluxes (with polar zeroing) through every x^D face of the
// flux pass's face box that borders a flagged cell, over the raw fluxes.
template <class TIN, class R>
int launch_fofc_faces(int D, const CVarsT<TIN>& P, const Layout& L, const GeomT<R>& G, const Scheme& S,
                      const int8_t* flag, R* F, R* ctop, int tpb, cudaStream_t s);
// The update reads its time increment as coef * dtp[0] (device memory), so a
// captured step keeps working when dt changes.
int launch_update(const double* U0, const CVars& Pin, const Vars& Pout, double* Uout, double* const F[3],
                  const Layout& L, const DevGeom& G, const Scheme& S, const double* dtp, double coef, int8_t* pflag,
                  unsigned long long* cnt, int tpb, cudaStream_t s, FailList fl = FailList{nullptr, nullptr},
                  const double* fBn = nullptr, double* dUout = nullptr);
// out = sum_t a[t] in[t] over n values (nterm <= 4).
int launch_lincomb(double* out, int nterm, const double* const* in, const double* a, long long n, cudaStream_t s);
// Face-centred CT of one stage (S.emf: KH_EMF_AVERAGE | KH_EMF_GS05): cell
// EMFs into ecc (GS05 only), edge EMFs from the raw fluxes F into emf[3],
// then fBout = fB0 + coef dtp[0] curl E on the interior cells' faces.
// R = float (mixed): FP32 stage input, fluxes and EMFs, FP64 face field.
template <class R>
int launch_face_ct(const CVarsT<R>& P, R* const F[3], R* ecc, R* const emf[3], const double* fB0, double* fBout,
                   const Layout& L, const GeomT<R>& G, const Scheme& S, const double* dtp, double coef,
                   cudaStream_t s);
int launch_face_divb(const double* fB, const Layout& L, double* partial, int npartial, double* out2, cudaStream_t s);
int launch_face_to_cell(const double* fB, double* B, const Layout& L, const DevGeom& G, cudaStream_t s);
// Mixed update: FP32 fluxes and sources, FP64 accumulation of U and FP64
// inversion; the stage input (sources, inversion guess) is read in FP32.
// Writes the FP64 output (Pout64.v[0] may be null) and/or its FP32 shadow
// (Pout32.v[0] may be null), and U when Uout is given (stage 2).
int launch_update_mixed(const double* U0, const CVarsT<float>& Pin, const Vars& Pout64, const VarsT<float>& Pout32,
                        double* Uout, float* const F[3], const Layout& L, const DevGeom& G, const GeomT<float>& Gf,
                        const Scheme& S, const double* dtp, double coef, int8_t* pflag, unsigned long long* cnt,
                        int tpb, cudaStream_t s, FailList fl = FailList{nullptr, nullptr},
                        const double* fBn = nullptr, double* dUout = nullptr, float* const* emf = nullptr);
// The same update (3-D grids, Flux-CT EMFs, no face field) with its inputs --
// P8 the 8-plane FP32 stage input, U0, the FP32 fluxes F and edge EMFs emf --
// staged per tile in shared memory by TMA (kh_update_tma.cu); wlim bounds the
// polls of a CTA's wait for its tiles. Returns -1 (nothing launched) where it
// does not apply or the tensor maps cannot be encoded.
int launch_update_mixed_tma(const double* U0, const float* P8, const Vars& Pout64, const VarsT<float>& Pout32,
                            double* Uout, float* const F[3], float* const emf[3], const Layout& L, const DevGeom& G,
                            const GeomT<float>& Gf, const Scheme& S, const double* dtp, double coef, int8_t* pflag,
                            unsigned long long* cnt, FailList fl, double* dUout, unsigned wlim, cudaStream_t s);
// Fixup over every zone, or (fl.idx != nullptr) over the stage's failed-zone list.
template <class T>
int launch_fixup(const VarsT<T>& P, double* Uout, const int8_t* pflag, const Layout& L, const DevGeom& G,
                 const Scheme& S, unsigned long long* cnt, cudaStream_t s, FailList fl = FailList{nullptr, nullptr});
template <class T>
int launch_cfl(T* const ctop[3], const Layout& L, double cfl, double* partial, int npartial, double* dt_out,
               cudaStream_t s);
int launch_divb(const double* const B[3], const Layout& L, const DevGeom& G, double* partial, int npartial,
                double* out2, cudaStream_t s);
int launch_p2c(const CVars& P, double* U, const Layout& L, const DevGeom& G, const Scheme& S, cudaStream_t s);
int launch_c2p(const double* U, const Vars& P, int8_t* pflag, const Layout& L, const DevGeom& G, const Scheme& S,
               unsigned long long* cnt, cudaStream_t s);
// Element-wise FP64 -> FP32 copy of n values.
int launch_to_f32(const double* src, float* dst, long long n, cudaStream_t s);
// The double-float planes of one grid's cell-centre geometry and floors.
int launch_df_planes(const double* geo, const double* flo, float* df, long long gplane, cudaStream_t s);
// FP64 -> FP32 copy of the 8 primitive planes (every cell of the allocation).
int launch_vars_to_f32(const CVars& src, const VarsT<float>& dst, const Layout& L, cudaStream_t s);
// The interior state (U, then P and B) in the compact order [16][n3][n2][n1].
int launch_pack(const double* U, const CVars& PB, double* out, const Layout& L, cudaStream_t s);
int launch_unpack(const double* in, double* U, const Vars& PB, const Layout& L, cudaStream_t s);
// The FP32 copy of an FP64 state with its ghost cells filled, in one pass:
// interior converted, ghosts by the ghost map from the FP64 interior.
int launch_fill_f32(const CVars& src, const VarsT<float>& dst, const Layout& L, const Scheme& S, const double* dlo,
                    const double* dhi, cudaStream_t s);

// Blocks used by the reductions (partial buffers hold 2 doubles per block).
constexpr int RED_THREADS = 256;
int reduction_blocks(const Layout& L);

#ifdef __CUDACC__
// Programmatic dependent launch for the kernels of the mixed step (fill,
// faces, EMFs, update, fixup, CFL): a kernel launched with launch_pdl is
// scheduled while the previous kernel on the stream drains, its CTAs
// resident and waiting in pdl_wait, which every such kernel calls before its
// first global access; it returns once the previous kernel has completed and
// its writes are visible (for a kernel launched without the attribute it
// returns at once). The step then loses no launch latency between its
// dependent kernels when launched kernel by kernel: 1430 -> 1477 M
// zone-cycles/s on the 192x96x96 torus; a captured graph of the same launches
// replays at 1461 M with or without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <class... P, class... A>
cudaError_t launch_pdl(void (*kern)(P...), dim3 g, dim3 b, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}
#endif

}  // namespace kh
