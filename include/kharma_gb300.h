/*
 * kharma_gb300.h -- C ABI of the GB300 (sm_103a) implementation of the HARM
 * finite-volume step for ideal GRMHD on a stationary Kerr spacetime
 * (arXiv 2408.01361, "KHARMA": "Algorithm" section for the scheme, "Extended
 * GRMHD" section for the ideal-MHD stress-energy tensor, "Requirements"
 * section for the funky-MKS coordinates, "Performance" section for the
 * zone-cycles/s metric).
 *
 * Memory: every array argument is a DEVICE pointer owned by the caller,
 * double precision, structure of arrays [var][n3s][n2s][n1s] with ghost
 * zones included; (n1s, n2s, n3s, ng) come from kh_shape(). Interior zone
 * (i, j, k) (0-based) lives at (ng + i, ng + j, ng3 + k) where ng3 = ng for
 * 3-D problems and 0 when n3 == 1. The row length n1s is n1 + 2 ng rounded
 * up to a multiple of 16 elements; the padding is never read or written.
 *   P: 5 fluid primitives rho, u, u~1, u~2, u~3 (u~ = velocity relative to the
 *      normal observer, McKinney & Gammie 2004);
 *   B: 3 cell-centred field components B^1..B^3;
 *   U: 8 conserved variables sqrt(-g) (rho u^t, T^t_t + rho u^t, T^t_i, B^i).
 * The library owns its geometry cache, scratch fluxes and reductions; it
 * allocates them in kh_geometry_init and frees them in kh_destroy.
 *
 * Streams: all calls are ordered on the context's stream (kh_set_stream;
 * default stream 0). A context is not thread-safe.
 *
 * Errors: 0 on success; negative KH_E* codes on failure (kh_strerror). A
 * positive return from kh_step / kh_cons_to_prim means "completed, with that
 * many zones whose inversion failed" (they were repaired by the fixup). No
 * call traps or asserts on the device; every device loop is bounded.
 */
#ifndef KHARMA_GB300_H
#define KHARMA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { KH_MINKOWSKI = 0, KH_KS = 1, KH_MKS = 2, KH_FMKS = 3 };
enum { KH_BC_PERIODIC = 0, KH_BC_OUTFLOW = 1, KH_BC_POLAR = 2, KH_BC_DIRICHLET = 3 };
enum { KH_RECON_MC = 0, KH_RECON_WENO5 = 1 };
enum { KH_FP64 = 0, KH_MIXED = 1 };
enum { KH_B_FLUXCT = 0, KH_B_FACE = 1 };
enum { KH_EMF_AVERAGE = 0, KH_EMF_GS05 = 1 };
enum { KH_INV_NOBLE2D = 0, KH_INV_1DW = 1, KH_INV_KASTAUN = 2 };
enum { KH_INT_VL2 = 0, KH_INT_RK1 = 1, KH_INT_RK2 = 2, KH_INT_SSPRK54 = 3 };
enum {
  KH_OK = 0,
  KH_EINVAL = -1,   /* bad argument or unsupported combination */
  KH_ECUDA = -2,    /* a CUDA runtime call failed */
  KH_ENOMEM = -3,   /* device allocation failed */
  KH_ETIMEOUT = -4, /* a bounded device wait gave up */
  KH_ENAN = -5      /* non-finite time step */
};

/* Problem description (coordinates, grid, boundaries, scheme options). */
typedef struct {
  int kind;               /* KH_MINKOWSKI | KH_KS | KH_MKS | KH_FMKS */
  int n1, n2, n3;         /* interior zones; n3 == 1 => 2-D (x1, x2) problem */
  int recon;              /* KH_RECON_MC | KH_RECON_WENO5 */
  int precision;          /* KH_FP64: every step of the path in FP64.
                             KH_MIXED: reconstruction, face fluxes, signal speeds,
                             Flux-CT EMFs and the connection sources in FP32 (FP32
                             stencil copies of P and of the geometry); U stored in
                             FP64 (U^n + the FP32 increment is an FP64 add); the
                             Noble-2D inversion in double-float (two FP32 numbers,
                             ~48 bits) with an FP64 fallback for zones it does not
                             converge (or in FP64 for every zone: mixed_inversion),
                             floors with FP32 decisions and double-float values;
                             1D_W and Kastaun invert in FP64; divB in FP64. */
  int bc[6];              /* x1 in, x1 out, x2 in, x2 out, x3 in, x3 out: KH_BC_* */
  double x1min, x1max, x2min, x2max, x3min, x3max; /* native coordinate box */
  double hslope;          /* MKS / FMKS theta concentration h */
  double poly_xt, poly_alpha, mks_smooth; /* FMKS parameters (alpha: even integer) */
  double cfl;             /* Courant number of the returned dt */
  double rho_min, u_min;  /* floor coefficients of r^-3/2 and r^-5/2 (>= 1e-20 each) */
  double bsq_rho_max, bsq_u_max; /* magnetisation ceilings b^2/rho, b^2/u */
  double u_rho_max;       /* temperature ceiling u/rho */
  double gamma_max;       /* Lorentz-factor ceiling */
  int newton_max_iter;    /* inversion iteration cap (<= 0: 30) */
  double newton_tol;      /* inversion tolerance on |dW/W| + |dv^2| (<= 0: 1e-14) */
  int fofc;               /* 1: first-order flux correction ("Algorithm" section, after
                             Beckwith & Stone 2011): each stage first runs a trial
                             update with its high-order fluxes; every face of a zone
                             whose trial inversion fails or whose floors act takes the
                             donor-cell (first-order) LLF flux, and polar zeroing and
                             Flux-CT are applied again before the stage's update. The
                             flags' ghost zones follow the state's ghost map (Dirichlet
                             ghosts unflagged; on a refined mesh a ghost takes the
                             flag of the cell it copies or is prolonged from, or the
                             largest flag of the fine cells it restricts). 0: off.
                             With Flux-CT, any integrator, single grids and meshes
                             (face CT and the adjoint refuse it). */
  int bfield;             /* KH_B_FLUXCT: cell-centred field, Flux-CT (Toth 2000);
                             KH_B_FACE: face-centred constrained transport
                             ("Algorithm" section: Stone & Gardiner 2009). The face
                             field sqrt(-g) B^a lives on the lower x^a face of each
                             cell (kh_set_face_field); the edge EMFs advance it by
                             d_b E_c - d_c E_b, which keeps every cell's face
                             divergence; B of a zone is the mean of its two faces
                             over sqrt(-g). Edge EMFs on a polar axis are zero.
                             Single grids and the refined mesh (kh_mesh_*: coarse
                             edges on a level interface take the finer block's EMFs),
                             FP64 and KH_MIXED (FP32 EMFs, the curl formed in FP64,
                             the face field in FP64); no flux correction, no
                             adjoint. Single grids run it with any integrator (the
                             face field is a stage state like U); the mesh with the
                             predictor-corrector. */
  int emf;                /* KH_B_FACE edge EMFs: KH_EMF_AVERAGE (mean of the four
                             face values; with face means as the zone field this is
                             Flux-CT) or KH_EMF_GS05 (Gardiner & Stone 2005: plus the
                             half-zone derivative terms, each taken from the cell
                             upwind of the mass flux through its face) */
  int inverter;           /* FP64 primitive recovery ("Algorithm" section): KH_INV_NOBLE2D
                             (Noble et al. 2006, Newton on (W, v^2); default),
                             KH_INV_1DW (Noble et al.'s one-unknown scheme: v^2(W) in
                             closed form, Newton on the energy equation) or
                             KH_INV_KASTAUN (Kastaun, Kalinani & Ciolfi 2021:
                             bracketed root of a master function of 1/(h gamma)).
                             All find the same root; newton_max_iter / newton_tol
                             apply to each (KASTAUN: up to 4x the iterations, tol
                             on the bracket width). Single-grid contexts, FP64 and
                             KH_MIXED (there Noble-2D runs in double-float with an
                             FP64 fallback, the others in FP64), single grids and
                             the refined mesh; the adjoint carries Noble-2D and
                             refuses the others; used by the update and
                             kh_cons_to_prim. */
  int integrator;         /* time integrator ("Algorithm" section): KH_INT_VL2 (the
                             predictor-corrector, default), KH_INT_RK1, KH_INT_RK2
                             (Heun) or KH_INT_SSPRK54 (Spiteri & Ruuth's five-stage
                             fourth-order SSP scheme), in Shu-Osher form: each stage
                             U_s = sum_j a_sj U_j + c_s dt L(P_{s-1}) with the
                             stage operator, inversion, floors and fixup of a
                             predictor-corrector stage. Single-grid contexts, FP64 or
                             KH_MIXED (the FP32 shadow carries the intermediate stage
                             primitives), with Flux-CT (and the flux correction in
                             every stage) or face CT (the face field combined with
                             the same weights; SSPRK(5,4)'s fifth stage takes stage
                             4's face increment as its output minus its base); 8 to
                             48 extra planes of scratch, plus 6 to 15 with face CT. */
  int mixed_inversion;    /* KH_MIXED with KH_INV_NOBLE2D: KH_MIXINV_DF (default) runs the
                             inversion in double-float with the FP64 fallback above;
                             KH_MIXINV_FP64 keeps the whole inversion in FP64 for every
                             zone: the conserved variables entering it are the FP64
                             U^n + increment, the Noble-2D Newton iteration starts from
                             the FP32 stage input, and the floors act in FP64 as on the
                             FP64 path. Ignored by KH_FP64 contexts and the other
                             solvers; single grids and the refined mesh. */
} kh_coords;
enum { KH_MIXINV_DF = 0, KH_MIXINV_FP64 = 1 };

/* Counters of the last kh_step (both stages summed). */
typedef struct {
  int64_t nfail;    /* zones whose inversion failed (repaired by the fixup) */
  int64_t nfloor;   /* zones where a floor or ceiling was applied */
  int64_t nunfixed; /* failed zones with no good neighbour (kept the stage input) */
  double dt_cfl;    /* CFL time step for the next step */
  int64_t nfp64;    /* KH_MIXED: zones whose inversion fell back to the FP64 Newton iteration */
  int64_t nfofc;    /* zones flagged by the first-order flux correction's trials */
  int64_t nbounds;  /* a library built with -DKH_BOUNDS_CHECK: work items whose cells fell
                       outside the allocation and were skipped, since the context was
                       created (0 in release builds, which have no checks) */
} kh_stats;

typedef struct kh_ctx kh_ctx;

/* Create a context: validates c, allocates the library's device buffers and
 * fills the FP64 geometry cache (metric, inverse, sqrt(-g), lapse at cell
 * centres and x1/x2 faces; connection at cell centres) for Kerr spin a and
 * the ideal-gas adiabatic index gamma ("Code Structure": GRCoordinates).
 * Geometry: Kerr-Schild (t, r, theta, phi); MKS r = e^x1, theta = pi x2 +
 * (1-h)/2 sin(2 pi x2); FMKS adds the polynomial theta of Wong et al. 2022
 * blended by exp(mks_smooth (x1min - x1)); theta is continued past the poles
 * by reflection. Requires n1, n2 >= 4, n3 >= 1, ng = 3 ghost zones.
 * Returns KH_EINVAL, KH_ENOMEM or KH_ECUDA on failure (*out untouched). */
int kh_geometry_init(double a, const kh_coords* c, double gamma, kh_ctx** out);

/* Allocation shape of every array: [var][*n3s][*n2s][*n1s], *ng ghosts. */
int kh_shape(const kh_ctx* ctx, int* n1s, int* n2s, int* n3s, int* ng);

/* Order all later calls on this cudaStream_t (NULL = legacy default stream). */
int kh_set_stream(kh_ctx* ctx, void* cuda_stream);

/* Ghost values for a KH_BC_DIRICHLET face (face 0: x1 inner, 1: x1 outer).
 * PB: device pointer, [8][n3s][n2s][ng] (P slots then B slots; ghost index
 * 0 is the ghost nearest the inner face of the array, i.e. cell ng - 3 for
 * face 0 and cell ng + n1 for face 1). Copied into the context. */
int kh_set_dirichlet(kh_ctx* ctx, int face, const double* PB);

/* U = sqrt(-g) (rho u^t, T^t_t + rho u^t, T^t_i, B^i) at every cell
 * (ghosts included), T^mu_nu the ideal-MHD stress-energy tensor of the
 * "Extended GRMHD" section (the conserved variables of the "Algorithm"
 * section's update). */
int kh_prim_to_cons(kh_ctx* ctx, const double* P, const double* B, double* U);

/* Primitive recovery at every cell (ghosts included) by the Noble et al.
 * (2006) two-unknown Newton iteration on (W, v^2), FP64. P holds the initial
 * guess on entry and the result on exit (unchanged where the inversion
 * failed); B = U_B / sqrt(-g). No floors, no fixup. pflag (device int8,
 * nullable): 0 ok, 1 no convergence, 2 v^2 >= 1, 3 W <= 0, 4 rho <= 0,
 * 5 u < 0. *nfail (host, nullable) = number of failed cells (synchronises). */
int kh_cons_to_prim(kh_ctx* ctx, const double* U, double* P, double* B, int8_t* pflag, int64_t* nfail);

/* One two-stage predictor-corrector step of length dt ("Algorithm" section;
 * conserved-synchronised). On entry U is U^n (authoritative) and (P, B) is
 * the matching P^n (stage-1 input and inversion guess). Stage 1: ghost fill,
 * fluxes from P^n (reconstruction, LLF, polar zeroing, Flux-CT), sources,
 * U* = U^n + dt/2 (-div F + S), inversion, floors, fixup -> P*. Stage 2: the
 * same from P* with dt applied to U^n -> U^{n+1}, P^{n+1}. Interior zones of
 * U, P, B are overwritten; ghost zones of P, B hold the stage-1 fill.
 * dt_cfl (host, nullable): if given, the stream is synchronised and the CFL
 * dt of the new state (from stage-2 signal speeds) is written; otherwise no
 * host synchronisation happens and the value is kept for kh_get_stats.
 * Returns the number of failed inversions (>= 0) when dt_cfl is given, 0
 * otherwise, or a negative KH_E* code. */
int kh_step(kh_ctx* ctx, double* U, double* P, double* B, double dt, double* dt_cfl);

/* CFL dt of a state (P, B): ghost fill on a scratch copy, fluxes, then
 * dt = cfl min_zones 1 / sum_d (ctop_d / dx_d). Synchronises. */
int kh_cfl_dt(kh_ctx* ctx, const double* P, const double* B, double* dt_cfl);

/* Corner divergence of sqrt(-g) B at corners whose adjacent cells are all
 * interior (the quantity the "Algorithm" section's Flux-CT conserves, and
 * the divergence the "Readiness and Testing" section monitors): *max_abs =
 * max |divB|, *l1 = mean |divB| over those corners (host pointers;
 * synchronises). */
int kh_divb(kh_ctx* ctx, const double* B, double* max_abs, double* l1);

/* Diagnostics: the fluxes kh_step uses, from (P, B) with ghosts filled by the
 * caller: F1, F2, F3 (device, [8][n3s][n2s][n1s], the flux through the lower
 * face of each cell, after polar zeroing and Flux-CT; F3 unused when
 * n3 == 1; the first-order flux correction, which needs a trial update, is
 * not applied). Entries outside the computed face ranges are left untouched. */
int kh_fluxes(kh_ctx* ctx, const double* P, const double* B, double* F1, double* F2, double* F3);

/* KH_B_FACE contexts: register the face field fB (device, caller-owned,
 * [3][n3s][n2s][n1s], plane a = sqrt(-g) B^(a+1) on the lower x^(a+1) face of
 * each cell; on a 2-D grid plane 2 holds the cell's sqrt(-g) B^3) that every
 * later kh_step advances together with (U, P, B). kh_step updates the faces
 * of the interior cells (both bounding faces along the normal) and leaves
 * other entries alone. The zone field B must be the face means over sqrt(-g)
 * (kh_face_to_cell) when stepping starts. KH_EINVAL for other contexts. */
int kh_set_face_field(kh_ctx* ctx, double* fB);

/* B (3 planes) of the interior cells = the face means of fB over sqrt(-g)
 * (ghost cells untouched). Any context. */
int kh_face_to_cell(kh_ctx* ctx, const double* fB, double* B);

/* Face divergence sum_a (fB_a(upper) - fB_a(lower)) / dx_a of the interior
 * cells (x1, x2 only on a 2-D grid): *max_abs = max |div|, *l1 = mean |div|
 * (host pointers; synchronises). Any context. */
int kh_face_divb(kh_ctx* ctx, const double* fB, double* max_abs, double* l1);

/* The interior state in a compact order, for moving it to and from the host
 * with the ghost cells and row padding left out: kh_pack_state writes
 * out[16][n3][n2][n1] = U's 8 slots, then P's 5 and B's 3, of the interior
 * zones; kh_unpack_state writes them back into the padded layout (interior
 * cells only). out / in may be device memory or page-locked host memory
 * (cudaHostAlloc, or cudaHostRegister'ed; under unified addressing it is
 * mapped into the device address space at the same address): the kernels
 * then read or write it over the host link directly, with no separate copy.
 * Asynchronous on the context stream (synchronise before the host reads a
 * packed host buffer, or reuses one being unpacked). */
int kh_pack_state(kh_ctx* ctx, const double* U, const double* P, const double* B, double* out);
int kh_unpack_state(kh_ctx* ctx, const double* in, double* U, double* P, double* B);

/* Ghost fill of (P, B) in place with the context's boundary rules. */
int kh_fill_ghosts(kh_ctx* ctx, double* P, double* B);

/* Counters of the last kh_step (synchronises). */
int kh_get_stats(kh_ctx* ctx, kh_stats* out);

/* CUDA-graph replay: enable != 0 captures the launches of one kh_step into a
 * graph (on a private capture stream) the first time kh_step is called with a
 * given (U, P, B) triple and replays it on the context stream afterwards;
 * dt reaches the captured update kernels through device memory, so every
 * call may use a new dt. New pointers or launch settings re-capture.
 * With profiling on (kh_profile) the captured step holds the group events
 * as external event record nodes, recorded on every replay; switching
 * profiling re-captures. enable == 0 frees the graph. */
int kh_set_graph(kh_ctx* ctx, int enable);

/* Threads per block of the stencil (reconstruction + LLF) kernels and of the
 * update kernels: each one of 32, 64, 128, 256 (default 128, 128). */
int kh_set_launch(kh_ctx* ctx, int tpb_flux, int tpb_update);
int kh_get_launch(const kh_ctx* ctx, int* tpb_flux, int* tpb_update);

/* Autotuner: times kh_step of the state (U, P, B) with step dt (on scratch
 * copies; the inputs are not modified) for every pair of threads per block in
 * {64, 128, 256} x {64, 128, 256}, keeps the fastest in the context and in a
 * process-wide cache keyed by (n1, n2, n3, coordinates, reconstruction,
 * precision), and writes the choice to the host pointers (nullable). The
 * scratch copies are allocated and freed inside the call. Synchronises. */
int kh_autotune(kh_ctx* ctx, const double* U, const double* P, const double* B, double dt, int* tpb_flux,
                int* tpb_update);

/* Per-kernel-group timing. Groups: */
enum {
  KH_T_BC = 0,     /* ghost fill (3 kernels in 3-D) */
  KH_T_FLUX1 = 1,  /* reconstruction + LLF through x1 faces */
  KH_T_FLUX2 = 2,  /* ... x2 faces */
  KH_T_FLUX3 = 3,  /* ... x3 faces */
  KH_T_CT = 4,     /* Flux-CT EMFs and field fluxes (2 kernels) */
  KH_T_UPDATE = 5, /* sources + update + inversion + floors */
  KH_T_FIXUP = 6,  /* neighbour-average repair of failed zones */
  KH_T_CFL = 7,    /* CFL reduction (2 kernels) */
  KH_T_FOFC = 8,   /* first-order flux correction: trial, flag ghosts, donor-cell
                      faces and the second Flux-CT (kh_coords.fofc) */
  KH_NTIMERS = 9
};
/* enable != 0: record CUDA events on the context stream around each group of
 * every later kh_step (each step then synchronises its stream; with a CUDA
 * graph, kh_set_graph, the events are nodes of the captured step and are
 * recorded by every replay) and reset the accumulators; enable == 0 stops
 * and resets. */
int kh_profile(kh_ctx* ctx, int enable);
/* Accumulated milliseconds and timed intervals per group (host arrays of
 * KH_NTIMERS entries; either may be NULL). One interval per stage. */
int kh_profile_read(const kh_ctx* ctx, double* ms, int64_t* count);

/* Number of kernel launches issued by this context since creation. */
int64_t kh_launch_count(const kh_ctx* ctx);

/* Bounded device wait of the KH_MIXED face kernels: each CTA stages its
 * tile in shared memory by one TMA tensor copy and polls the copy's mbarrier
 * at most `polls` times (default KH_WAIT_POLLS; each poll may suspend the
 * thread for a short hardware-defined interval). A CTA that gives up counts
 * a timeout, keeps waiting (at most KH_WAIT_POLLS more polls) until its
 * copy has landed, so that no copy outlives the CTA's shared memory, and
 * leaves its faces unwritten; the next kh_get_stats (and kh_step with a
 * dt_cfl pointer) returns KH_ETIMEOUT, and the step's result is not valid.
 * polls = 0 gives up before the first poll (to exercise the path). The
 * context stays usable: set the limit back and step again. Drops a captured
 * graph. KH_EINVAL for a null context. */
#define KH_WAIT_POLLS (1u << 22)
int kh_set_wait_limit(kh_ctx* ctx, unsigned polls);

/* ---------------------------------------------------------------------------
 * Adjoint of one step (FP64 contexts). Given the gradient of an objective
 * with respect to the outputs of kh_step(U, P, B, dt) -- gU (8 planes), gP
 * (5), gB (3), each nullable (= 0), and gF1, nullable, the gradient with
 * respect to the stage-2 x1 face fluxes (8 planes, the flux through the lower
 * x1 face of each cell, after Flux-CT) -- writes the gradient with respect to
 * the step's inputs U (gU_in, 8 planes), P (gP_in, 5) and B (gB_in, 3), and
 * with respect to the adiabatic index (*g_gamma). Interior cells carry the
 * gradient; ghost cells are written as 0. U, P, B are the step's input
 * (the checkpoint; read only): the step is re-run from it to record the
 * stage states, then reversed (see the reverse rules below). All arrays are
 * device pointers in the kh_shape layout; the call synchronises the context
 * stream. Scratch (~83 planes of doubles) is allocated on the first call and
 * kept until kh_destroy. KH_EINVAL for a mixed-precision context, a
 * context with the first-order flux correction on, or bad arguments.
 *
 * Reverse rules: limiter and max branches as taken by the
 * forward (ties: the first argument), LLF with ctop differentiated through
 * its active speed, Flux-CT and the ghost fill transposed exactly, the
 * inversion by the implicit-function theorem (a 5x5 FP64 solve per zone),
 * floored components and fixed-up zones frozen (zero derivative upstream).
 * The initial guess of the inversion carries no derivative. */
int kh_step_adjoint(kh_ctx* ctx, const double* U, const double* P, const double* B, double dt, const double* gU,
                    const double* gP, const double* gB, const double* gF1, double* gU_in, double* gP_in,
                    double* gB_in, double* g_gamma);

/* Gradient of U = kh_prim_to_cons(P, B) at interior cells: gP (5 planes), gB
 * (3 planes) = (dU/dP)^T gU, and the gamma derivative; ghosts written as 0.
 * FP64 contexts; synchronises the stream. */
int kh_prim_to_cons_adjoint(kh_ctx* ctx, const double* P, const double* B, const double* gU, double* gP, double* gB,
                            double* g_gamma);
/* The fluxes through the lower x^dir faces (dir 1..3; 8 planes, after
 * Flux-CT) of the last stage the context ran -- after kh_step, its second
 * stage. Copied on the context stream (asynchronous). FP64 contexts. */
int kh_get_stage_flux(kh_ctx* ctx, int dir, double* F);

/* ---------------------------------------------------------------------------
 * Static mesh refinement: many blocks at several levels stepped together
 * ("Requirements" section: refinement against the polar time-step limit;
 * "Code Structure" section: SMR through the mesh framework).
 *
 * The domain and scheme come from a kh_coords whose n1, n2, n3 give the
 * level-0 grid; level l is 2^l times finer in every direction (x1 and x2 only
 * when n3 == 1). A block covers the level-l index box [i0, i0+n1) x [j0, j0+n2)
 * x [k0, k0+n3); blocks must tile the domain exactly, blocks above level 0
 * must start and end on even indices, and blocks whose ghost zones meet must
 * be at most one level apart. Boundaries: periodic, outflow, polar.
 *
 * Arrays are arenas of all blocks in order: block b's U occupies
 * U + 8 * off_b with 8 planes of its own padded shape (kh_mesh_block_shape;
 * rows padded to a multiple of 8 elements),
 * its P (5 planes) P + 5 * off_b, its B (3 planes) B + 3 * off_b, where off_b
 * is the block's cell offset. Ghost cells are filled from other blocks: a
 * same-level copy, an MC-limited linear prolongation from a coarser block,
 * or the average of the 2x2(x2) cells of a finer block. A prolongation slope
 * takes the coarse-level values on both sides of the coarse cell (a cell of
 * a block at that level, or the mean of a finer block's cells there) and is
 * zero where one is missing (past a non-periodic domain edge, or inside a
 * still coarser block). Every block takes the same dt (no sub-cycling);
 * fluxes at level interfaces are not corrected (no refluxing) and Flux-CT
 * keeps divB only inside blocks. With face-centred CT (kh_coords.bfield =
 * KH_B_FACE) each block carries its face field in an arena like B's (3 planes
 * per block at fB + 3 * off_b; kh_mesh_set_face_field); after the blocks'
 * edge EMFs are computed, every coarse edge lying on the surface of a block
 * one level finer takes the fine block's EMF there (the mean of the two fine
 * edges along a refined edge direction), so each coarse face on a level
 * interface moves exactly as the mean of the fine faces covering it and the
 * face divergence stays zero in every block (interfaces across a periodic
 * domain edge are not matched).
 *
 * The mesh takes every kh_coords option of a single grid except face-centred
 * CT together with a Runge-Kutta integrator or with the flux correction.
 *
 * kh_mesh_init returns KH_EINVAL for blocks that overlap, leave a hole, are
 * smaller than 4 cells a side (n3 == 1 in 2-D), are misaligned, meet a block
 * more than one level away, or for more than 5 levels or 2^31 cells, and for
 * the option combinations above; it copies the block list, so the caller may
 * free it on return. */
typedef struct {
  int level;
  int i0, j0, k0;  /* first interior cell in level-l indices */
  int n1, n2, n3;  /* interior cells */
} kh_block;

typedef struct kh_mesh kh_mesh;

int kh_mesh_init(double a, const kh_coords* c, double gamma, int nblocks, const kh_block* blocks, kh_mesh** out);
int kh_mesh_block_shape(const kh_mesh* mesh, int b, int* n1s, int* n2s, int* n3s, int64_t* cell_offset);
/* KH_B_FACE meshes: register the face-field arena (device, caller-owned,
 * 3 planes per block as above) that every later kh_mesh_step advances. The
 * zones' B must be the face means over sqrt(-g) when stepping starts. */
int kh_mesh_set_face_field(kh_mesh* mesh, double* fB);
int64_t kh_mesh_cells(const kh_mesh* mesh);       /* sum of the blocks' allocation planes */
int64_t kh_mesh_zones(const kh_mesh* mesh);       /* interior zones of all blocks */
int64_t kh_mesh_ghost_cells(const kh_mesh* mesh); /* entries of the ghost map */
int kh_mesh_set_stream(kh_mesh* mesh, void* cuda_stream);
int kh_mesh_prim_to_cons(kh_mesh* mesh, const double* P, const double* B, double* U);
int kh_mesh_fill_ghosts(kh_mesh* mesh, double* P, double* B);
/* Same contract as kh_cfl_dt / kh_step, over all blocks; one kernel launch
 * per step phase covers every block. */
int kh_mesh_cfl_dt(kh_mesh* mesh, const double* P, const double* B, double* dt_cfl);
int kh_mesh_step(kh_mesh* mesh, double* U, double* P, double* B, double dt, double* dt_cfl);
/* Corner divB of sqrt(-g) B (as kh_divb) at the corners of every block whose
 * adjacent cells are all interior cells of that block: max |divB| and its
 * mean over those corners. Corners on block faces are left out: Flux-CT
 * holds divB only inside blocks (level interfaces are not constrained). */
int kh_mesh_divb(kh_mesh* mesh, const double* B, double* max_abs, double* l1);
int kh_mesh_set_graph(kh_mesh* mesh, int enable);
/* Threads per block of the face kernels and of the update kernel over all
 * blocks (multiples of 32 in [32, 256]; KH_EINVAL otherwise), and the
 * autotuner: times the pairs {64, 128, 256}^2 on scratch copies of (U, P, B)
 * (allocated for the search and freed), keeps the fastest and caches it for
 * the process per (block shapes with their counts, coordinates,
 * reconstruction, precision). Results are bitwise independent of the choice. */
int kh_mesh_set_launch(kh_mesh* mesh, int tpb_flux, int tpb_update);
int kh_mesh_get_launch(const kh_mesh* mesh, int* tpb_flux, int* tpb_update);
/* The mixed mesh's update with its inputs staged in shared memory by TMA
 * tensor copies (as kh_step's on 3-D grids), used when the mesh qualifies:
 * KH_MIXED, 3-D, Flux-CT, Noble-2D, every block 16 or 32 zones wide along x1,
 * and the U passed to kh_mesh_step 16-byte aligned (its tensor maps are
 * rebuilt, and copied to the device on the mesh's stream, whenever the step
 * is handed another U). enable = 0 selects the update that loads its inputs
 * itself; results are bitwise the same. Returns 1 if the staged update is
 * selected and the mesh qualifies (the U condition is checked per step), 0
 * otherwise, KH_EINVAL for a null mesh. Enabled by default. */
int kh_mesh_set_staged_update(kh_mesh* mesh, int enable);
int kh_mesh_autotune(kh_mesh* mesh, const double* U, const double* P, const double* B, double dt, int* tpb_flux,
                     int* tpb_update);
int kh_mesh_get_stats(kh_mesh* mesh, kh_stats* out);
int64_t kh_mesh_launch_count(const kh_mesh* mesh);
int kh_mesh_destroy(kh_mesh* mesh);

/* No-allocation divB (no counterpart in the paper; an interface addition).
 * For callers that cannot call cudaMalloc -- code confined to a pre-sized
 * memory pool or a hard device-memory budget, or frameworks whose allocator
 * forbids raw CUDA allocations -- and therefore cannot create a kh_ctx. It
 * computes the same corner divergence of sqrt(-g) B as kh_divb, without a
 * context, allocating nothing: its only scratch (one partial result per row
 * of corners) is a file-scope static __device__ array of
 * 2 * KH_DIVB_NOALLOC_MAX_ROWS doubles (1 MiB), which every GPU that loads the
 * library holds until the process exits.
 *   B:    device, [3][n3s][n2s][n1s] with n3s = n3 + 6 (n3 > 1) or 1 (n3 == 1),
 *         ng = 3 ghost zones, interior as in kh_shape();
 *   gdet: device, [n2s][n1s], sqrt(-g) at cell centres;
 *   dx1..dx3: native zone widths (dx3 ignored when n3 == 1);
 *   out:  device, 2 doubles: out[0] = max |divB|, out[1] = mean |divB| over the
 *         corners whose adjacent cells are all interior;
 *   cuda_stream: cudaStream_t to launch on (NULL = legacy default stream).
 * B, gdet and out must be memory of the CURRENT device (cudaGetDevice), and
 * cuda_stream a stream of that device: the scratch address used is the
 * current device's. Asynchronous on the stream; returns KH_EINVAL for bad
 * sizes, including a grid with more than KH_DIVB_NOALLOC_MAX_ROWS rows of
 * corners ((n2 - 1) * max(n3 - 1, 1)), or for an array that is not memory of
 * the current device, and KH_ECUDA if a CUDA error was already pending on
 * entry (left untouched for the caller) or a launch fails. The scratch
 * address looked up for a device is kept for the life of the process; it
 * does not survive a cudaDeviceReset of that device.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture. Every call shares the one array and leaves its
 * last contents there; each call writes every slot it later reads, so nothing
 * needs clearing between calls, but calls that overlap on the GPU (concurrent
 * streams, or several host threads) race on it and must be serialised. */
#define KH_DIVB_NOALLOC_MAX_ROWS 65536
int kh_divb_noalloc(const double* B, const double* gdet, int n1, int n2, int n3, int n1s, int n2s, double dx1,
                    double dx2, double dx3, double* out, void* cuda_stream);

/* Free the context and its device buffers (synchronises its stream). */
int kh_destroy(kh_ctx* ctx);

/* Static description of an error code. */
const char* kh_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* KHARMA_GB300_H */
