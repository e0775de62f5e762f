// The context behind kh_ctx* (shared by the step driver and the adjoint).
#pragma once

#include "kh_internal.h"

struct kh_ctx {
  kh_coords c;
  double a, gam;
  kh::Layout L;
  kh::Scheme S;
  kh::CoordParams cp;
  cudaStream_t stream;
  double* geo;
  double* dgm;
  double* flo;     // geometric floors of rho and u per (i, j)
  double* pstar;   // 8 planes: stage-1 output
  double* F[3];    // 8 planes each
  double* ctop[3];
  double* emf[3];
  int8_t* pflag;
  int8_t* fflag;   // first-order flux correction: flags of the current stage (one plane)
  double* fsave;   // ... and the raw field fluxes kept across the trial (3 planes per direction)
  float* fsavef;   // (unused: the mixed path never overwrites its raw field fluxes)
  // face-centred CT (KH_B_FACE): the caller's face field (kh_set_face_field),
  // the stage-1 face field and the cell-centred EMFs (3 planes each)
  double* fB;
  double* fBstar;
  double* ecc;
  float* eccf;     // the cell-centred EMFs of KH_MIXED (FP32)
  double* rk;      // Runge-Kutta integrators: stage states, base, stage-4 increment (8 planes each)
  double* rkf;     // with face-centred CT: the face field's stage states and base (3 planes each)
  // the face field a stage reads and writes (set per Runge-Kutta stage;
  // null: the predictor-corrector's fB -> fBstar, fB -> fB)
  const double* fb_in;
  double* fb_out;
  double* partial;
  int npartial;
  double* dscalar;              // [0] dt_cfl out, [1..2] divb max/sum, [3] dt in
  unsigned long long* counters; // NCNT
  double* dirichlet[2];
  // mixed precision (KH_MIXED): FP32 geometry copy, FP32 flux pass buffers,
  // FP32 stage-1 output and FP32 Dirichlet ghosts
  float* geof;
  float* dgmf;
  float* geodf;    // [NDF] planes of double-float (hi, lo) pairs: the cell-centre geometry and floors
  unsigned* flist; // failed-zone list of the current stage (one entry per zone at most)
  float* pstarf;   // 8 planes
  float* pnf;      // 8 planes: FP32 copy of the ghost-filled stage-1 input
  float* Ff[3];    // 8 planes each
  float* ctopf[3];
  float* emff[3];
  float* dirichletf[2];
  long long launches;
  kh_stats last;
  // launch configuration (threads per block of the stencil and update kernels)
  int tpb_flux, tpb_update;
  unsigned wait_limit;  // polls of a face CTA's wait for its TMA tile (kh_set_wait_limit)
  // CUDA-graph replay of the step, keyed by the (U, P, B) pointers captured
  int graph_on;
  cudaStream_t cap_stream;
  cudaGraphExec_t gexec;
  const void* gkey[3];
  int graph_launches;
  // optional per-kernel-group timing (CUDA events on the context stream)
  int profiling;
  cudaEvent_t ev[KH_NTIMERS][2][2];  // [group][stage][start, stop]
  int ev_used[KH_NTIMERS][2];
  // a step captured while profiling holds its group events as external event
  // record nodes; gev_used is the set it records on every replay
  int capturing, gprof;
  int gev_used[KH_NTIMERS][2];
  double prof_ms[KH_NTIMERS];
  long long prof_n[KH_NTIMERS];
  // adjoint step (kh_step_adjoint): recorded forward states and adjoint
  // scratch, allocated on the first call
  double* adj;      // ADJ_PLANES planes
  int8_t* adj_i8;   // 4 planes: pflag and floor masks of both stages
  double* adj_red;  // reduction slot for d/dgamma
};

// Plane offsets inside kh_ctx::adj.
enum {
  ADJ_PH1 = 0,    // 8: ghost-filled stage-1 input
  ADJ_RAW1 = 8,   // 8: stage-1 inversion result before floors
  ADJ_PN1 = 16,   // 8: P^{n+1}
  ADJ_RAW2 = 24,  // 8: stage-2 inversion result before floors
  ADJ_UN1 = 32,   // 8: U^{n+1}
  ADJ_LP = 40,    // 8: adjoint of the ghost-filled stage input
  ADJ_LU = 48,    // 8: adjoint of U before the inversion
  ADJ_LF = 56,    // 24: adjoint of the face fluxes, 3 directions x 8
  ADJ_LE = 80,    // 3: adjoint of the edge EMFs
  ADJ_PLANES = 83
};
