// Static mesh refinement on one GPU: many uneven blocks at several levels
// stepped by one launch per kernel over all blocks (arXiv 2408.01361,
// "Requirements": refinement of the grid away from where the polar zones
// limit the time step; "Code Structure": SMR/AMR through Parthenon).
//
// Every kernel of the step runs over the concatenation of all blocks' items
// (faces, edges, zones, ghost cells): a thread finds its block by binary
// search over a per-kernel prefix sum of item counts, then runs the same
// per-item device function as the single-grid kernels with that block's
// layout, geometry and arena offsets. Ghost cells of every block are filled
// by one gather (two launches: same-level copies, then the interpolating
// ops) from a map built on the host at set-up: each ghost
// cell's centre is carried through the physical boundary rules (outflow
// clamps to the first interior cell, polar reflection, periodic wrap), the
// leaf block owning that point is found, and the ghost cell copies the
// owner's cell (same level), prolongs from the owner's coarse cell with
// MC-limited slopes (coarser owner), or averages the owner's 2x2(x2) fine
// cells (finer owner). The slopes take the coarse-level values beside the
// coarse cell: a cell of a block at that level, or the mean of a finer
// block's cells there; where neither exists (past a non-periodic domain edge,
// or inside a still coarser block) the slope in that direction is zero.
// Every source is an interior cell, so the fill has no ordering between
// ghost cells.
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kh_update_tile.cuh"
#include "kh_zone.cuh"

using namespace kh;

namespace {

constexpr int MTPB = 128;

struct MBlock {
  Layout L;
  long long off;   // cell offset of the block in cell-concatenated arenas
  long long goff;  // (j, i) offset in the geometry arenas
  FaceBox fb[3];
  int polar_lo, polar_hi;
  int level;
  int i0, j0, k0;
};

enum { G_COPY = 0, G_PROLONG = 1, G_RESTRICT = 2 };
enum { G_FLIP2 = 1, G_CLAMP_IN = 2, G_CLAMP_OUT = 4 };

struct GhostOp {
  int dst_block, dst_cell;
  int src_block, src_cell;
  int nbi;             // prolongation: index of the coarse cell's neighbour record
  signed char off[3];  // prolongation: sign of the fine-cell offset from the coarse centre per direction
  unsigned char mode, flags, pad;
};

// A same-level copy in 16 bytes (one vector load per thread): the source
// cell in the low 28 bits of the last word, the boundary flags above them.
struct __align__(16) GhostCopy {
  int dst_block, dst_cell, src_block;
  unsigned src_cell_flags;
};

// Coarse-level values on either side of a prolonged coarse cell, per
// direction: [d][0] below, [d][1] above. mode G_COPY: a cell of a block at
// the coarse level; G_RESTRICT: the mean of a finer block's 2x2(x2) cells
// starting at that cell; NB_NONE: no value (beyond a non-periodic edge of
// the domain, or inside a still coarser block), the slope is then zero.
enum { NB_NONE = 3 };
struct ProlongNb {
  int block[3][2];
  int cell[3][2];
  unsigned char mode[3][2];
  unsigned char pad[2];
};

// Arena of 8 primitive slots: slots [0, na) at a + na * off + v * plane,
// slots [na, 8) at b + (8 - na) * off + (v - na) * plane.
template <class T> struct Arena {
  T* a;
  T* b;
  int na;
};

template <class T> __device__ __forceinline__ VarsT<T> vars_at(const Arena<T>& A, const MBlock& m) {
  VarsT<T> V;
#pragma unroll
  for (int v = 0; v < NV; ++v)
    V.v[v] = v < A.na ? A.a + A.na * m.off + v * m.L.plane : A.b + (NV - A.na) * m.off + (v - A.na) * m.L.plane;
  return V;
}
template <class T> __device__ __forceinline__ CVarsT<T> cvars_at(const Arena<T>& A, const MBlock& m) {
  const VarsT<T> V = vars_at(A, m);
  CVarsT<T> C;
#pragma unroll
  for (int v = 0; v < NV; ++v) C.v[v] = V.v[v];
  return C;
}

struct GeoArena {
  const double* g;
  const double* dgm;
  const double* flo;
  const float* gf;
  const float* dgmf;
  const float* df;
};
__device__ __forceinline__ DevGeom geo64(const GeoArena& A, const MBlock& m) {
  return DevGeom{A.g + 3LL * NGEO * m.goff, A.dgm + (long long)NDG * m.goff, A.flo + 3 * m.goff};
}
__device__ __forceinline__ GeomT<float> geo32(const GeoArena& A, const MBlock& m) {
  return GeomT<float>{A.gf + 3LL * NGEO * m.goff, A.dgmf + (long long)NDG * m.goff, A.flo + 3 * m.goff,
                      A.df ? A.df + 2LL * NDF * m.goff : nullptr};
}

// Largest b with pre[b] <= t (pre has nb + 1 entries, pre[0] = 0, non-
// decreasing). After the prefix the array holds a granule table: entry g is
// that block for t = g * 2^GRAN_SHIFT; from there a forward scan (over at most
// the few block ends inside one granule -- every block holds far more than
// 2^GRAN_SHIFT items) replaces a binary search's chain of dependent loads.
constexpr int GRAN_SHIFT = 8;
__device__ __forceinline__ int find_block(const unsigned* pre, int nb, unsigned t) {
  int b = (int)__ldg(pre + nb + 1 + (t >> GRAN_SHIFT));
  while (b + 1 < nb && __ldg(pre + b + 1) <= t) ++b;
  return b;
}

// One face per thread. The FP32 faces are held to 64 registers (four
// 256-thread blocks per SM): their stencil loads are latency-bound, and the
// extra warps hide more of it than the few spilled values cost (refined torus
// 870 -> 915 M zone-cycles/s against 80 registers); the FP64 faces would
// spill ~700 bytes a thread under that cap and keep their registers.
template <int D, int RECON, class TIN, class R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1)
    km_flux(const MBlock* blk, const unsigned* pre, int nb, Arena<TIN> Pin, GeoArena GA, Scheme S, R* F, R* ctop) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  int i, j, k;
  const FaceBox& fb = m.fb[D - 1];
  split3(t - __ldg(pre + b), fb.n[0], fb.n[1], i, j, k);
  GeomT<R> G;
  if constexpr (sizeof(R) == sizeof(double)) G = geo64(GA, m); else G = geo32(GA, m);
  flux_face<D, RECON, TIN, R>(cvars_at(Pin, m), m.L, G, S, i + fb.lo[0], j + fb.lo[1], k + fb.lo[2],
                              F + NV * m.off, ctop + m.off, m.polar_lo, m.polar_hi);
}

template <class R>
__global__ void km_ct(const MBlock* blk, const unsigned* pre, int nb, R* F1, R* F2, R* F3, R* e1, R* e2, R* e3,
                      int phase) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  const Layout& L = m.L;
  int i, j, k;
  split3(t - __ldg(pre + b), L.e[0] - L.s[0] + 1, L.e[1] - L.s[1] + 1, i, j, k);
  i += L.s[0];
  j += L.s[1];
  k += (L.ndim == 3 ? L.s[2] : 0);
  const long long o8 = NV * m.off, o1 = m.off;
  R* f3 = L.ndim == 3 ? F3 + o8 : nullptr;
  R* ee1 = L.ndim == 3 ? e1 + o1 : nullptr;
  R* ee2 = L.ndim == 3 ? e2 + o1 : nullptr;
  if (phase == 0)
    emf_at<R>(F1 + o8, F2 + o8, f3, ee1, ee2, e3 + o1, L, i, j, k);
  else
    apply_ct_at<R>(F1 + o8, F2 + o8, f3, ee1, ee2, e3 + o1, L, i, j, k);
}

// The stage's failed-zone list as block b's update appends to it (entries
// b << 20 | cell; the list is off when idx is null).
__device__ __forceinline__ FailList block_list(const FailList& fl, int b) {
  return FailList{fl.idx, fl.n, fl.idx ? (unsigned)b << 20 : 0u};
}

template <int INV>
__global__ void __launch_bounds__(256) km_update(const MBlock* blk, const unsigned* pre, int nb, const double* U0,
                                                Arena<double> Pin, Arena<double> Pout, double* Uout,
                                                const double* F1, const double* F2, const double* F3, GeoArena GA,
                                                Scheme S, const double* dtp, double coef, int8_t* pflag,
                                                unsigned long long* cnt, const double* fBn, double* dUout,
                                                FailList fl) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  int i, j, k;
  zone_ijk(m.L, t - __ldg(pre + b), i, j, k);
  const long long o8 = NV * m.off;
  update_zone<false, INV>(U0 + o8, cvars_at(Pin, m), vars_at(Pout, m), Uout ? Uout + o8 : nullptr, F1 + o8, F2 + o8,
              m.L.ndim == 3 ? F3 + o8 : nullptr, m.L, geo64(GA, m), S, coef * __ldg(dtp), pflag + m.off, cnt, i, j,
              k, nullptr, block_list(fl, b), fBn ? fBn + 3 * m.off : nullptr, dUout ? dUout + o8 : nullptr);
}

template <int INV>
__global__ void __launch_bounds__(256, 2) km_update_mixed(const MBlock* blk, const unsigned* pre, int nb,
                                                      const double* U0, Arena<float> Pin, Arena<double> Pout64,
                                                      Arena<float> Pout32, double* Uout, const float* F1,
                                                      const float* F2, const float* F3, GeoArena GA, Scheme S,
                                                      const double* dtp, double coef, int8_t* pflag,
                                                      unsigned long long* cnt, const double* fBn, const float* e1,
                                                      const float* e2, const float* e3, double* dUout, FailList fl) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  int i, j, k;
  zone_ijk(m.L, t - __ldg(pre + b), i, j, k);
  const long long o8 = NV * m.off;
  Vars P64;
  VarsT<float> P32;
  if (Pout64.a) P64 = vars_at(Pout64, m); else for (int v = 0; v < NV; ++v) P64.v[v] = nullptr;
  if (Pout32.a) P32 = vars_at(Pout32, m); else for (int v = 0; v < NV; ++v) P32.v[v] = nullptr;
  // the FP64 fallback inversion out of line, as in the staged update: both
  // then run the one compiled copy and round alike
  update_mixed_zone<false, INV, true>(U0 + o8, cvars_at(Pin, m), P64, P32, Uout ? Uout + o8 : nullptr, F1 + o8, F2 + o8,
                    m.L.ndim == 3 ? F3 + o8 : nullptr, m.L, geo64(GA, m), geo32(GA, m), S,
                    df_of_f64(coef * __ldg(dtp)), pflag + m.off, cnt, i, j, k, block_list(fl, b),
                    fBn ? fBn + 3 * m.off : nullptr, dUout ? dUout + o8 : nullptr,
                    CtEmf{{e1 ? e1 + m.off : nullptr, e2 ? e2 + m.off : nullptr, e3 ? e3 + m.off : nullptr}});
}

// ---- the mixed update with TMA-staged tiles (3-D Flux-CT stages) ----
// As on the single grid (kh_update_tile.cuh): one CTA of 256 threads per tile
// of TX zones along x1 -- a block's whole interior row, TX = 16 or 32 -- by
// 256 / TX rows along x2 of one x3 plane, its inputs staged by eight tensor
// copies. The tensor maps sit in a device table, two or three sets per block
// over the block's own allocation (set 0: the first stage's input and the
// caller's U^n; set 1: the FP32 shadow of later stages and U^n; set 2, with
// a Runge-Kutta integrator: the shadow and the stage base): built at set-up
// for the internal arrays, and rebuilt for U^n (the caller's array) whenever
// the step is handed another one. Blocks start their rows at cell 0, a 16-byte
// boundary at or below the first interior cell (3) for floats and doubles
// alike; the U^n box starts at cell 2.
struct MTile {
  int b, j0, k;  // block, first row (x2 cell index), plane (x3 cell index)
};
constexpr int TMA_N1[2] = {16, 32};  // block widths the staged update serves (one kernel each)

template <int TX, int INV>
__global__ void __launch_bounds__(256, 3)
    km_update_mixed_tma(const MBlock* blk, const MTile* tiles, const UpdateMaps* maps, int nsets, int set,
                        Arena<double> Pout64, Arena<float> Pout32, double* Uout, GeoArena GA, Scheme S,
                        const double* dtp, double coef, int8_t* pflag, unsigned long long* cnt, unsigned wlim,
                        double* dUout, FailList fl) {
  using T = UpdTile<TX, 256 / TX>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = aligned_smem(smem_raw);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + T::O_BAR);
  const MTile t = tiles[blockIdx.x];
  const MBlock& m = blk[t.b];
  const UpdateMaps& tm = maps[nsets * t.b + set];
  const int lx = threadIdx.x & (TX - 1), ly = threadIdx.x / TX;
  const int i0 = m.L.s[0], x0 = i0 & ~3, xu0 = i0 & ~1;
  if (threadIdx.x == 0) {
    mbar_init(bar);
    // the maps were written through the generic proxy (a host copy)
    tensormap_acquire(&tm.p);
    tensormap_acquire(&tm.f1);
    tensormap_acquire(&tm.f2);
    tensormap_acquire(&tm.f3);
    tensormap_acquire(&tm.e1);
    tensormap_acquire(&tm.e2);
    tensormap_acquire(&tm.e3);
    tensormap_acquire(&tm.u);
  }
  __syncthreads();
  if (threadIdx.x == 0) issue_update_tile<T>(smem, tm, x0, xu0, t.j0, t.k, bar);
  if (!cta_wait_tiles(bar, wlim, cnt)) return;
  const Layout& L = m.L;
  const int i = i0 + lx, j = t.j0 + ly, k = t.k;
  if (i >= L.e[0] || j >= L.e[1]) return;  // ragged tile
  if (KH_OOB(L, kh_in(L, i, j, k, 1))) return;
  Vars P64;
  VarsT<float> P32;
  if (Pout64.a) P64 = vars_at(Pout64, m); else for (int v = 0; v < NV; ++v) P64.v[v] = nullptr;
  if (Pout32.a) P32 = vars_at(Pout32, m); else for (int v = 0; v < NV; ++v) P32.v[v] = nullptr;
  const typename T::In in{smem, (i0 - x0) + lx, (i0 - xu0) + lx, ly};
  update_mixed_zone_in<false, INV, typename T::In, true>(
      in, P64, P32, Uout ? Uout + NV * m.off : nullptr, L, geo64(GA, m), geo32(GA, m), S,
      df_of_f64(coef * __ldg(dtp)), pflag + m.off, cnt, i, j, k, block_list(fl, t.b), nullptr,
      dUout ? dUout + NV * m.off : nullptr);
}

// ---- first-order flux correction over all blocks (as the single grid's
// k_fofc_trial / k_flag_ghosts / k_fofc_faces) ----
// The trial update of every interior zone from the corrected-so-far fluxes:
// flag = 1 where the inversion fails or a floor or ceiling would act.
template <int INV>
__global__ void __launch_bounds__(256) km_fofc_trial(const MBlock* blk, const unsigned* pre, int nb, const double* U0,
                                                    Arena<double> Pin, const double* F1, const double* F2,
                                                    const double* F3, GeoArena GA, Scheme S, const double* dtp,
                                                    double coef, int8_t* flag, unsigned long long* cnt) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  int i, j, k;
  zone_ijk(m.L, t - __ldg(pre + b), i, j, k);
  const long long o8 = NV * m.off;
  update_zone<true, INV>(U0 + o8, cvars_at(Pin, m), Vars{}, nullptr, F1 + o8, F2 + o8,
                         m.L.ndim == 3 ? F3 + o8 : nullptr, m.L, geo64(GA, m), S, coef * __ldg(dtp), flag + m.off,
                         cnt, i, j, k);
}

template <int INV>
__global__ void __launch_bounds__(256, 2) km_fofc_trial_mixed(const MBlock* blk, const unsigned* pre, int nb,
                                                          const double* U0, Arena<float> Pin, const float* F1,
                                                          const float* F2, const float* F3, GeoArena GA, Scheme S,
                                                          const double* dtp, double coef, int8_t* flag,
                                                          unsigned long long* cnt, const float* e1, const float* e2,
                                                          const float* e3) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  int i, j, k;
  zone_ijk(m.L, t - __ldg(pre + b), i, j, k);
  const long long o8 = NV * m.off;
  update_mixed_zone<true, INV>(U0 + o8, cvars_at(Pin, m), Vars{}, VarsT<float>{}, nullptr, F1 + o8, F2 + o8,
                               m.L.ndim == 3 ? F3 + o8 : nullptr, m.L, geo64(GA, m), geo32(GA, m), S,
                               df_of_f64(coef * __ldg(dtp)), flag + m.off, cnt, i, j, k, FailList{nullptr, nullptr, 0u},
                               nullptr, nullptr,
                               CtEmf{{e1 ? e1 + m.off : nullptr, e2 ? e2 + m.off : nullptr, e3 + m.off}});
}

// The flags' ghost cells by the state's ghost map: a copied or prolonged
// ghost takes its source cell's flag, a restricted one the largest flag of
// the 2x2(x2) fine cells whose mean it takes.
__global__ void km_flag_ghost(const MBlock* blk, const GhostOp* ops, long long nops, int8_t* flag) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nops) return;
  const GhostOp op = ops[t];
  const MBlock& ms = blk[op.src_block];
  const int8_t* fs = flag + ms.off;
  int8_t f = fs[op.src_cell];
  if (op.mode == G_RESTRICT) {
    const Layout& L = ms.L;
    const long long sj = L.n1s, sk = (long long)L.n1s * L.n2s;
    for (int dk = 0; dk < (L.ndim == 3 ? 2 : 1); ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) f = max(f, fs[op.src_cell + di + dj * sj + dk * sk]);
  }
  flag[blk[op.dst_block].off + op.dst_cell] = f;
}

// Every face of every block's face box that borders a flagged cell takes the
// LLF flux of its two cells' own (donor-cell) states.
template <int D, class TIN, class R>
__global__ void __launch_bounds__(256) km_fofc_faces(const MBlock* blk, const unsigned* pre, int nb, Arena<TIN> P,
                                                    GeoArena GA, Scheme S, const int8_t* flag, R* F, R* ctop) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  int i, j, k;
  const FaceBox& fb = m.fb[D - 1];
  split3(t - __ldg(pre + b), fb.n[0], fb.n[1], i, j, k);
  i += fb.lo[0];
  j += fb.lo[1];
  k += fb.lo[2];
  const Layout& L = m.L;
  const long long c = L.at(k, j, i);
  const long long st = D == 1 ? 1 : (D == 2 ? (long long)L.n1s : (long long)L.n1s * L.n2s);
  const int8_t* fl = flag + m.off;
  if (!(fl[c] | fl[c - st])) return;
  GeomT<R> G;
  if constexpr (sizeof(R) == sizeof(double)) G = geo64(GA, m); else G = geo32(GA, m);
  flux_face<D, RECON_DONOR, TIN, R>(cvars_at(P, m), L, G, S, i, j, k, F + NV * m.off, ctop + m.off, m.polar_lo,
                                    m.polar_hi);
}

// The fixup over the stage's failed-zone list (its length read on the
// device), one warp per failed zone, as the single grid's k_fixup_list.
template <class T>
__global__ void __launch_bounds__(256) km_fixup_list(const MBlock* blk, Arena<T> P, double* Uout, const int8_t* pflag,
                                                     GeoArena GA, Scheme S, unsigned long long* cnt, FailList fl) {
  const unsigned long long n = *fl.n;
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long q = warp; q < n; q += nwarps) {
    const unsigned e = fl.idx[q];
    const MBlock& m = blk[e >> 20];
    const Layout& L = m.L;
    const long long c = e & 0xFFFFFu;
    const int k = (int)(c / L.gplane), j = (int)((c % L.gplane) / L.n1s), i = (int)(c % L.n1s);
    fixup_warp<T>(vars_at(P, m), Uout ? Uout + NV * m.off : nullptr, pflag + m.off, L, geo64(GA, m), S, cnt, i, j, k,
                  lane);
  }
}

template <class T>
__global__ void km_fixup(const MBlock* blk, const unsigned* pre, int nb, Arena<T> P, double* Uout,
                         const int8_t* pflag, GeoArena GA, Scheme S, unsigned long long* cnt) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  int i, j, k;
  zone_ijk(m.L, t - __ldg(pre + b), i, j, k);
  if (pflag[m.off + m.L.at(k, j, i)] == 0) return;
  fixup_zone<T>(vars_at(P, m), Uout ? Uout + NV * m.off : nullptr, pflag + m.off, m.L, geo64(GA, m), S, cnt, i, j,
                k);
}

__device__ __forceinline__ double wmax(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

template <class T>
__global__ void __launch_bounds__(RED_THREADS) km_cfl(const MBlock* blk, const unsigned* pre, int nb, const T* c1,
                                                     const T* c2, const T* c3, double cfl, double* partial) {
  T mt = T(0);  // per-thread maximum in the speeds' precision
  const unsigned nz = __ldg(pre + nb);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < nz; t += gridDim.x * blockDim.x) {
    const int b = find_block(pre, nb, t);
    const MBlock& m = blk[b];
    int i, j, k;
    zone_ijk(m.L, t - __ldg(pre + b), i, j, k);
    const T v = cfl_inv_zone(c1 + m.off, c2 + m.off, m.L.ndim == 3 ? c3 + m.off : c3, m.L, i, j, k);
    mt = v > mt ? v : mt;
  }
  double mx = (double)mt;
  __shared__ double sm[RED_THREADS / 32];
  mx = wmax(mx);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < RED_THREADS / 32 ? sm[threadIdx.x] : 0.0;
    mx = wmax(mx);
    if (threadIdx.x == 0) partial[blockIdx.x] = mx;
  }
}

__global__ void km_cfl_finish(const double* partial, int n, double cfl, double* out) {
  __shared__ double sm[RED_THREADS / 32];
  double mx = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) mx = fmax(mx, partial[q]);
  mx = wmax(mx);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < RED_THREADS / 32 ? sm[threadIdx.x] : 0.0;
    mx = wmax(mx);
    if (threadIdx.x == 0) out[0] = cfl / mx;
  }
}

// Mean of variable v over the 2x2(x2) cells of block m starting at cell c
// (a restriction to the next coarser level), summed i fastest, then j, k.
template <class T>
__device__ __forceinline__ T restrict_at(const Arena<T>& P, const MBlock& m, int v, long long c) {
  // in the arena's precision (FP32 on the mixed path)
  const Layout& L = m.L;
  const T* q = vars_at(P, m).v[v];
  const long long sj = L.n1s, sk = (long long)L.n1s * L.n2s;
  const int nk = L.ndim == 3 ? 2 : 1;
  T acc = T(0);
  for (int dk = 0; dk < nk; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) acc += q[c + di + dj * sj + dk * sk];
  return T(L.ndim == 3 ? 0.125 : 0.25) * acc;
}

__device__ __forceinline__ double wsum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block-wide max and sum of (a, b); thread 0 holds the result.
__device__ __forceinline__ void block_max_sum2(double& a, double& b) {
  __shared__ double sa[RED_THREADS / 32], sb[RED_THREADS / 32];
  a = wmax(a);
  b = wsum(b);
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = a;
    sb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    a = threadIdx.x < RED_THREADS / 32 ? sa[threadIdx.x] : 0.0;
    b = threadIdx.x < RED_THREADS / 32 ? sb[threadIdx.x] : 0.0;
    a = wmax(a);
    b = wsum(b);
  }
}

// Corner divB at the corners of every block whose adjacent cells are all
// interior cells of that block; per launch block: (max |divB|, sum |divB|).
__global__ void __launch_bounds__(RED_THREADS) km_divb(const MBlock* blk, const unsigned* pre, int nb,
                                                      const double* B, const double* geo, double* partial) {
  double mx = 0.0, sm = 0.0;
  const unsigned tot = __ldg(pre + nb);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
    const int b = find_block(pre, nb, t);
    const MBlock& m = blk[b];
    const Layout& L = m.L;
    int i, j, k;
    split3(t - __ldg(pre + b), L.n1 - 1, L.n2 - 1, i, j, k);
    i += L.s[0] + 1;
    j += L.s[1] + 1;
    k += L.ndim == 3 ? L.s[2] + 1 : 0;
    const double* Bb = B + 3 * m.off;
    const double* gd = geo + 3LL * NGEO * m.goff + (long long)LOC_CENT * NGEO * L.gplane + 20 * L.gplane;
    const double dv = divb_corner(Bb, Bb + L.plane, Bb + 2 * L.plane, L, gd, i, j, k);
    mx = fmax(mx, fabs(dv));
    sm += fabs(dv);
  }
  block_max_sum2(mx, sm);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = mx;
    partial[2 * blockIdx.x + 1] = sm;
  }
}

__global__ void km_max_sum_finish(const double* partial, int n, double* out) {
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    a = fmax(a, partial[2 * q]);
    b += partial[2 * q + 1];
  }
  block_max_sum2(a, b);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

// The physical boundary rules a ghost cell's op carries: polar reflection of
// the x2 components, no inflow through the x1 boundaries.
template <class T> __device__ __forceinline__ void ghost_flags(unsigned char flags, T* val) {
  if (flags & G_FLIP2) {
    val[V_U2] = -val[V_U2];
    val[V_B2] = -val[V_B2];
  }
  if ((flags & G_CLAMP_IN) && val[V_U1] > T(0)) val[V_U1] = T(0);
  if ((flags & G_CLAMP_OUT) && val[V_U1] < T(0)) val[V_U1] = T(0);
}

// The ghost-fill gather, part 1: the ghost cells whose owner is at the same
// level (the op list holds them first), one thread per ghost cell. They are
// most ghost cells (~88% on the refined torus); on their own they run without
// the registers and branches of the interpolating ops below.
template <class T>
__global__ void __launch_bounds__(MTPB) km_ghost_copy(const MBlock* blk, const GhostCopy* ops, long long n,
                                                      Arena<T> P) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int4 q = __ldg(reinterpret_cast<const int4*>(ops) + t);
  const unsigned sc = (unsigned)q.w;
  const VarsT<T> D = vars_at(P, blk[q.x]);
  const VarsT<T> Sv = vars_at(P, blk[q.z]);
  const long long c = sc & 0x0FFFFFFFu;
  T val[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) val[v] = Sv.v[v][c];
  ghost_flags((unsigned char)(sc >> 28), val);
#pragma unroll
  for (int v = 0; v < NV; ++v) D.v[v][q.y] = val[v];
}

// Part 2: the ops from index `first` on, restriction (finer owner) or
// prolongation (coarser owner), one thread per ghost cell.
template <class T>
__global__ void km_ghost(const MBlock* blk, const GhostOp* ops, long long first, long long nops, const ProlongNb* nbs,
                         Arena<T> P) {
  const long long t = first + blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nops) return;
  const GhostOp op = ops[t];
  const MBlock& md = blk[op.dst_block];
  const MBlock& ms = blk[op.src_block];
  const VarsT<T> D = vars_at(P, md);
  const VarsT<T> Sv = vars_at(P, ms);
  const long long c = op.src_cell;
  T val[NV];
  if (op.mode == G_COPY) {
#pragma unroll
    for (int v = 0; v < NV; ++v) val[v] = Sv.v[v][c];
  } else if (op.mode == G_RESTRICT) {
#pragma unroll
    for (int v = 0; v < NV; ++v) val[v] = restrict_at(P, ms, v, c);
  } else {  // prolongation from the coarse cell c with MC slopes over coarse-level neighbours
    // (in the arena's precision: FP64 arithmetic on FP32 data would run on
    // GB300's 1/64-rate FP64 pipe); each neighbour's block is looked up once
    // for all 8 variables
    const ProlongNb& nb = nbs[op.nbi];
    const int nd = ms.L.ndim;
    T q0[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) val[v] = q0[v] = Sv.v[v][c];
    for (int d = 0; d < nd; ++d) {
      if (op.off[d] == 0 || nb.mode[d][0] == NB_NONE || nb.mode[d][1] == NB_NONE) continue;
      T q[2][NV];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const MBlock& mn = blk[nb.block[d][side]];
        const long long cn = nb.cell[d][side];
        if (nb.mode[d][side] == G_COPY) {
          const VarsT<T> V = vars_at(P, mn);
#pragma unroll
          for (int v = 0; v < NV; ++v) q[side][v] = V.v[v][cn];
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) q[side][v] = restrict_at(P, mn, v, cn);
        }
      }
      const T w = T(0.25) * T(op.off[d]);
#pragma unroll
      for (int v = 0; v < NV; ++v) val[v] += w * mc_slope(q[0][v], q0[v], q[1][v]);
    }
  }
  ghost_flags(op.flags, val);
#pragma unroll
  for (int v = 0; v < NV; ++v) D.v[v][op.dst_cell] = val[v];
}

// FP64 -> FP32 copy of the 8 slots of every cell of every block.
__global__ void km_to_f32(const MBlock* blk, const unsigned* pre, int nb, Arena<double> src, Arena<float> dst) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  const long long c = t - __ldg(pre + b);
  const CVars S = cvars_at(src, m);
  const VarsT<float> D = vars_at(dst, m);
  // all eight loads first (in flight together), then the conversions
  // (integer ops, not the FP64 pipe) and stores
  double q[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) q[v] = S.v[v][c];
#pragma unroll
  for (int v = 0; v < NV; ++v) D.v[v][c] = f32_of_f64(q[v]);
}

// FP64 -> FP32 copy of the 8 slots of the interior cells of every block (the
// first mixed stage: its ghost cells are filled in FP32 by the gather right
// after, from interior cells only, so converting them as well is wasted work
// -- 2.4x the interior on a 16x16x32 block).
__global__ void km_to_f32_interior(const MBlock* blk, const unsigned* pre, int nb, Arena<double> src,
                                   Arena<float> dst) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  int i, j, k;
  zone_ijk(m.L, t - __ldg(pre + b), i, j, k);
  const long long c = m.L.at(k, j, i);
  const CVars S = cvars_at(src, m);
  const VarsT<float> D = vars_at(dst, m);
  // all eight loads first (in flight together), then the conversions
  // (integer ops, not the FP64 pipe) and stores
  double q[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) q[v] = S.v[v][c];
#pragma unroll
  for (int v = 0; v < NV; ++v) D.v[v][c] = f32_of_f64(q[v]);
}

__global__ void km_p2c(const MBlock* blk, const unsigned* pre, int nb, Arena<double> P, double* U, GeoArena GA,
                       Scheme S) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  const Layout& L = m.L;
  int i, j, k;
  split3(t - __ldg(pre + b), L.N1, L.N2, i, j, k);
  const long long c = L.at(k, j, i);
  const CVars Pv = cvars_at(P, m);
  double p[NV], u[NV];
  for (int v = 0; v < NV; ++v) p[v] = Pv.v[v][c];
  const DevGeom G = geo64(GA, m);
  const Met<double> met = load_met(G, L.gplane, LOC_CENT, (long long)j * L.n1s + i);
  FState<double> s;
  fluid_state(p, met, s);
  cons_only(p, s, met, S.gam, u);
  for (int v = 0; v < NV; ++v) U[NV * m.off + v * L.plane + c] = u[v];
}

inline int nblk(long long n, int tpb) { return (int)((n + tpb - 1) / tpb); }

}  // namespace

// ---------------------------------------------------------------------------
// The mesh context
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Face-centred CT on the mesh: each block's face field lives in an arena of 3
// planes per block (block b at 3 * off). Cell EMFs over every allocated cell
// of every block (ghosts hold the filled state), edge EMFs over each block's
// [s, e] box, then the interface matching (a coarse edge on the surface of a
// finer block takes the fine EMF, the mean of the two fine edges along a
// refined edge direction), then the face update.
// ---------------------------------------------------------------------------
template <class R>
__global__ void km_cell_emf(const MBlock* blk, const unsigned* pre, int nb, Arena<R> Pin, GeoArena GA, R* ecc) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  const Layout& L = m.L;
  int i, j, k;
  split3(t - __ldg(pre + b), L.N1, L.N2, i, j, k);
  const long long c = L.at(k, j, i);
  const CVarsT<R> P = cvars_at(Pin, m);
  R Pc[NV], E[3];
#pragma unroll
  for (int v = 0; v < NV; ++v) Pc[v] = P.v[v][c];
  Met<R> mt;
  if constexpr (sizeof(R) == sizeof(double)) mt = load_met(geo64(GA, m), L.gplane, LOC_CENT, (long long)j * L.n1s + i);
  else mt = load_met(geo32(GA, m), L.gplane, LOC_CENT, (long long)j * L.n1s + i);
  cell_emfs(Pc, mt, E);
  R* out = ecc + 3 * m.off;
#pragma unroll
  for (int q = 0; q < 3; ++q) out[q * L.plane + c] = E[q];
}

template <class R>
__global__ void km_face_emf(const MBlock* blk, const unsigned* pre, int nb, const R* F1, const R* F2, const R* F3,
                            const R* ecc, R* e1, R* e2, R* e3, int emf) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  const Layout& L = m.L;
  int i, j, k;
  split3(t - __ldg(pre + b), L.e[0] - L.s[0] + 1, L.e[1] - L.s[1] + 1, i, j, k);
  i += L.s[0];
  j += L.s[1];
  k += (L.ndim == 3 ? L.s[2] : 0);
  const long long o8 = NV * m.off, o1 = m.off, c = L.at(k, j, i);
  const R* F[3] = {F1 + o8, F2 + o8, L.ndim == 3 ? F3 + o8 : nullptr};
  const R* C = ecc ? ecc + 3 * m.off : nullptr;
  const bool axis = (m.polar_lo && j == L.s[1]) || (m.polar_hi && j == L.e[1]);
  if (L.ndim == 3) {
    if (k < L.e[2]) e3[o1 + c] = axis ? R(0) : edge_emf<R>(2, F, C, L, emf, i, j, k);
    if (i < L.e[0]) e1[o1 + c] = axis ? R(0) : edge_emf<R>(0, F, C, L, emf, i, j, k);
    if (j < L.e[1]) e2[o1 + c] = edge_emf<R>(1, F, C, L, emf, i, j, k);
  } else {
    e3[o1 + c] = axis ? R(0) : edge_emf<R>(2, F, C, L, emf, i, j, k);
    if (i < L.e[0]) e1[o1 + c] = axis ? R(0) : F[1][V_B3 * L.plane + c];
    if (j < L.e[1]) e2[o1 + c] = -F[0][V_B3 * L.plane + c];
  }
}

// One interface edge: E_c[dst] = mean of E_c[src[0..n)] (arena indices).
struct EmfMatch {
  long long dst, src[2];
  int c, n;
};
template <class R>
__global__ void km_emf_match(const EmfMatch* mt, long long nm, R* e1, R* e2, R* e3) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= nm) return;
  const EmfMatch M = mt[q];
  R* E = M.c == 0 ? e1 : (M.c == 1 ? e2 : e3);
  E[M.dst] = M.n == 2 ? R(0.5) * (E[M.src[0]] + E[M.src[1]]) : E[M.src[0]];
}

template <class R>
__global__ void km_face_update(const MBlock* blk, const unsigned* pre, int nb, const double* fB0, double* fBout,
                               const R* e1, const R* e2, const R* e3, const double* dtp, double coef) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= __ldg(pre + nb)) return;
  const int b = find_block(pre, nb, t);
  const MBlock& m = blk[b];
  const Layout& L = m.L;
  int x[3];
  split3(t - __ldg(pre + b), L.e[0] - L.s[0] + 1, L.e[1] - L.s[1] + 1, x[0], x[1], x[2]);
  x[0] += L.s[0];
  x[1] += L.s[1];
  x[2] += (L.ndim == 3 ? L.s[2] : 0);
  const long long c = L.at(x[2], x[1], x[0]);
  const long long st[3] = {1, (long long)L.n1s, (long long)L.n1s * L.n2s};
  const R* E[3] = {e1 + m.off, e2 + m.off, e3 + m.off};
  const double cdt = coef * __ldg(dtp);
  const double* f0 = fB0 + 3 * m.off;
  double* f1 = fBout + 3 * m.off;
  const int nd = L.ndim;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int bb = (a + 1) % 3, cc = (a + 2) % 3;
    bool in = true;
    for (int q = 0; q < nd; ++q)
      if (q != a && x[q] >= L.e[q]) in = false;
    if (!in) continue;
    auto f64 = [](R v) -> double {
      if constexpr (sizeof(R) == sizeof(double)) return v;
      else return f64_of_f32(v);
    };
    double rhs = 0.0;
    if (bb < nd) rhs += (f64(E[cc][c + st[bb]]) - f64(E[cc][c])) * L.idx[bb];
    if (cc < nd) rhs -= (f64(E[bb][c + st[cc]]) - f64(E[bb][c])) * L.idx[cc];
    f1[a * L.plane + c] = f0[a * L.plane + c] + cdt * rhs;
  }
}

struct kh_mesh {
  kh_coords c;
  Scheme S;
  CoordParams cp;
  int nb, ndim, lmax;
  int N0[3];  // level-0 grid
  std::vector<MBlock> hb;
  std::vector<unsigned> pre_face[3], pre_zone, pre_ct, pre_alloc, pre_all, pre_corner;
  long long corners;   // divB corners (adjacent cells all interior to one block)
  long long cells;     // sum of allocation planes
  long long gcells;    // sum of (j, i) planes
  long long zones;     // interior zones
  cudaStream_t stream;
  MBlock* dblk;
  unsigned* dpre[8];   // face1..3, zone, ct, alloc cells (km_to_f32), all-cells (p2c), divB corners
  GhostOp* dops;
  GhostCopy* dcopy = nullptr;  // ops [0, ncopy) in the compact form km_ghost_copy reads
  long long nops;
  long long ncopy;  // ops [0, ncopy) are same-level copies
  ProlongNb* dnbs;
  long long nnbs;
  double *geo, *dgm, *flo;
  float *geof, *dgmf;
  float* geodf;  // [NDF] planes of double-float (hi, lo) pairs per block (goff-based)
  double* pstar;
  float *pstarf, *pnf;
  double* F[3];
  double* ctop[3];
  double* emf[3];
  float* Ff[3];
  float* ctopf[3];
  float* emff[3];
  int8_t* pflag;
  unsigned* flist = nullptr;  // a stage's failed zones, b << 20 | cell (null: the fixup scans every zone)
  double* partial;
  int npartial;
  double* dscalar;  // [0] dt out, [1..2] divB max and sum, [3] dt in
  unsigned long long* counters;
  long long launches;
  int graph_on;
  int tpb_flux, tpb_update;  // threads per block of the face and update kernels
  cudaStream_t cap_stream;
  cudaGraphExec_t gexec;
  const void* gkey[3];
  int graph_launches;
  // face-centred CT: the caller's face field, the stage-1 face field, cell
  // EMFs (FP64 or FP32) and the interface EMF matches
  double* fB;
  double* fBstar;
  double* ecc;
  float* eccf;
  EmfMatch* dmatch;
  long long nmatch;
  // Runge-Kutta integrators: the stage states after U (SSPRK(5,4): 4, RK2: 1,
  // RK1: 0), the stage base and (SSPRK(5,4)) stage 4's raw increment, each
  // 8 planes of every block's cells
  double* rk;
  // first-order flux correction: the flags (every cell) and, FP64, the raw
  // fluxes saved before Flux-CT (8 planes of every block's cells per direction)
  int8_t* fflag;
  double* fsave;
  // TMA-staged mixed update (3-D Flux-CT, Noble-2D, every block 16 or 32
  // zones wide): tiles of the 16-wide blocks, then of the 32-wide ones; two
  // map sets per block (stage 1 and 2 inputs), host copy and device table
  int tma_upd;        // the mesh qualifies
  int tma_off;        // disabled by the caller (kh_mesh_set_staged_update)
  int tma_now;        // the maps hold the U^n of the current step
  MTile* dtiles;
  long long ntile[2];
  int nsets;          // map sets per block (see km_update_mixed_tma)
  UpdateMaps* dmaps;
  std::vector<UpdateMaps> hmaps;
  const double* umap_key;  // the U^n the maps point at
};

namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? KH_OK : (e == cudaErrorMemoryAllocation ? KH_ENOMEM : KH_ECUDA); }

// Stored stage states of a Runge-Kutta integrator besides U (the stage base follows them).
int rk_states(int integrator) { return integrator == KH_INT_SSPRK54 ? 4 : (integrator == KH_INT_RK2 ? 1 : 0); }

// Doubled finest-level index coordinates of cell centres (exact integers):
// the centre of level-l cell g along a direction refined by ratio r is
// (2 g + 1) * r^(lmax - l).
struct Locator {
  int lmax, ndim;
  long long nf[3];  // finest-level cells per direction
  std::vector<int> owner;
  long long ratio_pow(int d, int l) const {
    long long r = 1;
    const int rr = (d == 2 && ndim == 2) ? 1 : 2;
    for (int q = 0; q < lmax - l; ++q) r *= rr;
    return r;
  }
};

}  // namespace

extern "C" {

int kh_mesh_destroy(kh_mesh* x);

int kh_mesh_init(double a, const kh_coords* c, double gamma, int nblocks, const kh_block* blocks, kh_mesh** out) {
  if (!c || !blocks || !out || nblocks < 1) return KH_EINVAL;
  if (c->kind < KH_MINKOWSKI || c->kind > KH_FMKS || c->n1 < 2 || c->n2 < 2 || c->n3 < 1) return KH_EINVAL;
  if (c->precision != KH_FP64 && c->precision != KH_MIXED) return KH_EINVAL;
  if (c->recon != KH_RECON_MC && c->recon != KH_RECON_WENO5) return KH_EINVAL;
  if (c->fofc != 0 && c->fofc != 1) return KH_EINVAL;
  if (c->fofc && c->bfield == KH_B_FACE) return KH_EINVAL;  // the correction runs with Flux-CT
  if (c->inverter < KH_INV_NOBLE2D || c->inverter > KH_INV_KASTAUN) return KH_EINVAL;
  if (c->integrator < KH_INT_VL2 || c->integrator > KH_INT_SSPRK54) return KH_EINVAL;
  // Runge-Kutta stages carry U (and P) only: with face-centred CT the face field would be stage state too
  if (c->integrator != KH_INT_VL2 && c->bfield == KH_B_FACE) return KH_EINVAL;
  if (c->mixed_inversion != KH_MIXINV_DF && c->mixed_inversion != KH_MIXINV_FP64) return KH_EINVAL;
  if (c->bfield != KH_B_FLUXCT && c->bfield != KH_B_FACE) return KH_EINVAL;
  if (c->emf != KH_EMF_AVERAGE && c->emf != KH_EMF_GS05) return KH_EINVAL;
  if (!(gamma > 1.0) || !(c->cfl > 0.0) || !(fabs(a) < 1.0)) return KH_EINVAL;
  for (int q = 0; q < 6; ++q) {
    const int b = c->bc[q];
    if (b != KH_BC_PERIODIC && b != KH_BC_OUTFLOW && b != KH_BC_POLAR) return KH_EINVAL;
    if (b == KH_BC_POLAR && (q < 2 || q >= 4)) return KH_EINVAL;
  }
  kh_mesh* x = new kh_mesh();
  x->c = *c;
  x->nb = nblocks;
  x->ndim = c->n3 > 1 ? 3 : 2;
  x->N0[0] = c->n1;
  x->N0[1] = c->n2;
  x->N0[2] = c->n3;
  x->stream = 0;
  x->tpb_flux = x->tpb_update = MTPB;
  Scheme& S = x->S;
  S.gam = gamma;
  S.igam = 1.0 / gamma;
  S.gfac = (gamma - 1.0) / gamma;
  S.cfl = c->cfl;
  S.recon = c->recon;
  for (int q = 0; q < 6; ++q) S.bc[q] = c->bc[q];
  S.fl = FloorParams{c->rho_min,       c->u_min,           c->bsq_rho_max,         c->bsq_u_max,
                     c->u_rho_max,      c->gamma_max,       1.0 / c->bsq_rho_max,   1.0 / c->bsq_u_max};
  S.c2p.max_iter = c->newton_max_iter > 0 ? c->newton_max_iter : 30;
  S.c2p.tol = c->newton_tol > 0.0 ? c->newton_tol : 1e-14;
  S.c2p.method = c->inverter;
  S.mixed_fp64 = c->precision == KH_MIXED && c->inverter == KH_INV_NOBLE2D && c->mixed_inversion == KH_MIXINV_FP64;
  S.bfield = c->bfield;
  S.emf = c->emf;
  S.integrator = c->integrator;
  S.fofc = c->fofc;
  set_mixed(S);
  x->cp = CoordParams{c->kind, a, c->x1min, c->hslope, c->poly_xt, c->poly_alpha, c->mks_smooth};

  // ---- validate the blocks and rasterise ownership at the finest level ----
  int lmax = 0;
  for (int b = 0; b < nblocks; ++b) lmax = std::max(lmax, blocks[b].level);
  if (lmax > 4) { delete x; return KH_EINVAL; }
  x->lmax = lmax;
  Locator loc;
  loc.lmax = lmax;
  loc.ndim = x->ndim;
  for (int d = 0; d < 3; ++d) loc.nf[d] = (long long)x->N0[d] * loc.ratio_pow(d, 0);
  const long long nfin = loc.nf[0] * loc.nf[1] * loc.nf[2];
  if (nfin > (1LL << 31)) { delete x; return KH_EINVAL; }
  loc.owner.assign((size_t)nfin, -1);
  const double dx0[3] = {(c->x1max - c->x1min) / c->n1, (c->x2max - c->x2min) / c->n2,
                         (c->x3max - c->x3min) / c->n3};
  long long cells = 0, gcells = 0, zones = 0;
  x->hb.resize(nblocks);
  for (int b = 0; b < nblocks; ++b) {
    const kh_block& B = blocks[b];
    const int n[3] = {B.n1, B.n2, B.n3};
    const int o[3] = {B.i0, B.j0, B.k0};
    if (B.level < 0 || B.n1 < 4 || B.n2 < 4 || B.n3 < 1) { delete x; return KH_EINVAL; }
    if (x->ndim == 2 && (B.n3 != 1 || B.k0 != 0)) { delete x; return KH_EINVAL; }
    if (x->ndim == 3 && B.n3 < 4) { delete x; return KH_EINVAL; }
    for (int d = 0; d < 3; ++d) {
      const long long rl = loc.ratio_pow(d, 0) / loc.ratio_pow(d, B.level);  // level-l cells per level-0 cell
      const long long nl = (long long)x->N0[d] * rl;
      if (o[d] < 0 || o[d] + n[d] > nl) { delete x; return KH_EINVAL; }
      const bool refined_dir = !(d == 2 && x->ndim == 2);
      if (B.level > 0 && refined_dir && ((o[d] & 1) || (n[d] & 1))) { delete x; return KH_EINVAL; }
    }
    MBlock& m = x->hb[b];
    m.level = B.level;
    m.i0 = B.i0;
    m.j0 = B.j0;
    m.k0 = B.k0;
    Layout& L = m.L;
    L.n1 = B.n1; L.n2 = B.n2; L.n3 = B.n3;
    L.ng = NGHOST;
    L.ndim = x->ndim;
    L.ng3 = L.ndim == 3 ? NGHOST : 0;
    L.N1 = L.n1 + 2 * L.ng;
    L.N2 = L.n2 + 2 * L.ng;
    L.N3 = L.n3 + 2 * L.ng3;
    L.n1s = (L.N1 + 7) / 8 * 8;  // small blocks: 8-element rows waste less than 16 (22 -> 24, not 32)
    L.n2s = L.N2;
    L.n3s = L.N3;
    L.gplane = (long long)L.n1s * L.n2s;
    L.plane = L.gplane * L.n3s;
    for (int d = 0; d < 3; ++d) {
      const double rr = (double)(loc.ratio_pow(d, 0) / loc.ratio_pow(d, B.level));
      L.dx[d] = dx0[d] / rr;
      L.idx[d] = 1.0 / L.dx[d];
      L.idxf[d] = (float)L.idx[d];
    }
    L.s[0] = L.ng; L.e[0] = L.ng + L.n1;
    L.s[1] = L.ng; L.e[1] = L.ng + L.n2;
    L.s[2] = L.ng3; L.e[2] = L.ng3 + L.n3;
    for (int d = 1; d <= 3; ++d) m.fb[d - 1] = face_box(L, d);
    const long long nl2 = (long long)x->N0[1] * (loc.ratio_pow(1, 0) / loc.ratio_pow(1, B.level));
    m.polar_lo = c->bc[2] == KH_BC_POLAR && B.j0 == 0;
    m.polar_hi = c->bc[3] == KH_BC_POLAR && B.j0 + B.n2 == nl2;
    m.off = cells;
    m.goff = gcells;
    cells += L.plane;
    gcells += L.gplane;
    zones += (long long)L.n1 * L.n2 * L.n3;
    // ownership raster
    long long sc[3];
    for (int d = 0; d < 3; ++d) sc[d] = loc.ratio_pow(d, B.level);
    for (long long kf = o[2] * sc[2]; kf < (o[2] + n[2]) * sc[2]; ++kf)
      for (long long jf = o[1] * sc[1]; jf < (o[1] + n[1]) * sc[1]; ++jf)
        for (long long ifn = o[0] * sc[0]; ifn < (o[0] + n[0]) * sc[0]; ++ifn) {
          int& w = loc.owner[(size_t)((kf * loc.nf[1] + jf) * loc.nf[0] + ifn)];
          if (w != -1) { delete x; return KH_EINVAL; }  // overlap
          w = b;
        }
  }
  for (long long q = 0; q < nfin; ++q)
    if (loc.owner[(size_t)q] < 0) { delete x; return KH_EINVAL; }  // hole
  if (cells >= (1LL << 31)) { delete x; return KH_EINVAL; }
  x->cells = cells;
  x->gcells = gcells;
  x->zones = zones;

  // ---- ghost map ----
  std::vector<GhostOp> ops;
  std::vector<ProlongNb> nbs;
  std::map<std::pair<int, long long>, int> nb_of;  // (source block, coarse cell) -> its record
  const long long two_nf[3] = {2 * loc.nf[0], 2 * loc.nf[1], 2 * loc.nf[2]};
  for (int b = 0; b < nblocks && true; ++b) {
    const MBlock& m = x->hb[b];
    const Layout& L = m.L;
    const long long rp[3] = {loc.ratio_pow(0, m.level), loc.ratio_pow(1, m.level), loc.ratio_pow(2, m.level)};
    for (int k = 0; k < L.N3; ++k)
      for (int j = 0; j < L.N2; ++j)
        for (int i = 0; i < L.N1; ++i) {
          const bool inside = i >= L.s[0] && i < L.e[0] && j >= L.s[1] && j < L.e[1] && k >= L.s[2] && k < L.e[2];
          if (inside) continue;
          const int gi[3] = {m.i0 + i - L.ng, m.j0 + j - L.ng, m.k0 + k - L.ng3};
          long long X[3];
          for (int d = 0; d < 3; ++d) X[d] = (2LL * gi[d] + 1) * rp[d];
          unsigned char flags = 0;
          // x1: outflow clamps to the first/last interior cell at this level; periodic wraps
          if (X[0] < 0) {
            if (c->bc[0] == KH_BC_PERIODIC) X[0] += two_nf[0];
            else { X[0] = rp[0]; flags |= G_CLAMP_IN; }
          } else if (X[0] > two_nf[0]) {
            if (c->bc[1] == KH_BC_PERIODIC) X[0] -= two_nf[0];
            else { X[0] = two_nf[0] - rp[0]; flags |= G_CLAMP_OUT; }
          }
          // x2: polar reflection, periodic wrap or outflow clamp
          if (X[1] < 0) {
            if (c->bc[2] == KH_BC_POLAR) { X[1] = -X[1]; flags ^= G_FLIP2; }
            else if (c->bc[2] == KH_BC_PERIODIC) X[1] += two_nf[1];
            else X[1] = rp[1];
          } else if (X[1] > two_nf[1]) {
            if (c->bc[3] == KH_BC_POLAR) { X[1] = 2 * two_nf[1] - X[1]; flags ^= G_FLIP2; }
            else if (c->bc[3] == KH_BC_PERIODIC) X[1] -= two_nf[1];
            else X[1] = two_nf[1] - rp[1];
          }
          if (x->ndim == 3) {
            if (X[2] < 0) {
              if (c->bc[4] == KH_BC_PERIODIC) X[2] += two_nf[2]; else X[2] = rp[2];
            } else if (X[2] > two_nf[2]) {
              if (c->bc[5] == KH_BC_PERIODIC) X[2] -= two_nf[2]; else X[2] = two_nf[2] - rp[2];
            }
          } else {
            X[2] = 1;
          }
          const long long fi[3] = {X[0] / 2, X[1] / 2, X[2] / 2};
          const int s = loc.owner[(size_t)((fi[2] * loc.nf[1] + fi[1]) * loc.nf[0] + fi[0])];
          const MBlock& ms = x->hb[s];
          const Layout& Ls = ms.L;
          const int dl = ms.level - m.level;
          GhostOp op;
          op.dst_block = b;
          op.dst_cell = (int)L.at(k, j, i);
          op.src_block = s;
          op.flags = flags;
          op.pad = 0;
          op.off[0] = op.off[1] = op.off[2] = 0;
          const long long rs[3] = {loc.ratio_pow(0, ms.level), loc.ratio_pow(1, ms.level),
                                   loc.ratio_pow(2, ms.level)};
          const int so[3] = {ms.i0, ms.j0, ms.k0};
          const int sg[3] = {Ls.ng, Ls.ng, Ls.ng3};
          int li[3];
          op.nbi = -1;
          if (dl == 0 || dl == -1) {
            // the owner's cell containing the point
            for (int d = 0; d < 3; ++d) li[d] = (int)(X[d] / (2 * rs[d])) - so[d] + sg[d];
            op.mode = dl == 0 ? G_COPY : G_PROLONG;
            if (dl == -1) {
              long long gc[3];
              for (int d = 0; d < 3; ++d) {
                gc[d] = X[d] / (2 * rs[d]);  // the coarse cell's index at its own level
                const long long cc = (2LL * gc[d] + 1) * rs[d];
                op.off[d] = (signed char)(X[d] > cc ? 1 : (X[d] < cc ? -1 : 0));
              }
              ProlongNb nb{};
              for (int d = 0; d < 3; ++d)
                for (int side = 0; side < 2; ++side) {
                  nb.mode[d][side] = NB_NONE;
                  nb.block[d][side] = 0;
                  nb.cell[d][side] = 0;
                  if (d >= x->ndim) continue;
                  long long nc[3] = {gc[0], gc[1], gc[2]};
                  nc[d] += side ? 1 : -1;
                  const long long ncl = loc.nf[d] / rs[d];  // coarse-level cells across the domain
                  if (nc[d] < 0 || nc[d] >= ncl) {
                    if (c->bc[2 * d + (nc[d] < 0 ? 0 : 1)] != KH_BC_PERIODIC) continue;
                    nc[d] = (nc[d] + ncl) % ncl;
                  }
                  long long Y[3];
                  for (int q = 0; q < 3; ++q) Y[q] = x->ndim == 2 && q == 2 ? 1 : (2 * nc[q] + 1) * rs[q];
                  const int w = loc.owner[(size_t)(((Y[2] / 2) * loc.nf[1] + Y[1] / 2) * loc.nf[0] + Y[0] / 2)];
                  const MBlock& mw = x->hb[w];
                  const int wo[3] = {mw.i0, mw.j0, mw.k0};
                  const int wg[3] = {mw.L.ng, mw.L.ng, mw.L.ng3};
                  int lw[3];
                  if (mw.level == ms.level) {
                    for (int q = 0; q < 3; ++q) lw[q] = (int)(nc[q] - wo[q] + wg[q]);
                    nb.mode[d][side] = G_COPY;
                  } else if (mw.level == ms.level + 1) {
                    for (int q = 0; q < 3; ++q) {
                      const bool refined_dir = !(q == 2 && x->ndim == 2);
                      lw[q] = (int)((refined_dir ? 2 * nc[q] : nc[q]) - wo[q] + wg[q]);
                    }
                    nb.mode[d][side] = G_RESTRICT;
                  } else {
                    continue;  // inside a coarser block: no slope in this direction
                  }
                  nb.block[d][side] = w;
                  nb.cell[d][side] = (int)mw.L.at(lw[2], lw[1], lw[0]);
                }
              // one record per coarse cell, shared by the fine ghost cells prolonged from it
              const auto key = std::make_pair(s, (long long)Ls.at(li[2], li[1], li[0]));
              const auto it = nb_of.find(key);
              if (it != nb_of.end()) {
                op.nbi = it->second;
              } else {
                op.nbi = (int)nbs.size();
                nbs.push_back(nb);
                nb_of.emplace(key, op.nbi);
              }
            }
          } else if (dl == 1) {
            // the owner's 2x2(x2) fine cells covering this coarse cell
            for (int d = 0; d < 3; ++d) {
              const bool refined_dir = !(d == 2 && x->ndim == 2);
              const long long gcell = X[d] / (2 * rp[d]);  // this level's cell index
              li[d] = (int)((refined_dir ? 2 * gcell : gcell) - so[d] + sg[d]);
            }
            op.mode = G_RESTRICT;
          } else {
            kh_mesh_destroy(x);
            return KH_EINVAL;  // neighbours more than one level apart
          }
          op.src_cell = (int)Ls.at(li[2], li[1], li[0]);
          ops.push_back(op);
        }
  }
  // same-level copies first (km_ghost_copy), the interpolating ops after
  // (km_ghost); the fill has no ordering, every source being an interior cell
  std::stable_partition(ops.begin(), ops.end(), [](const GhostOp& o) { return o.mode == G_COPY; });
  x->nops = (long long)ops.size();
  x->ncopy = (long long)std::count_if(ops.begin(), ops.end(), [](const GhostOp& o) { return o.mode == G_COPY; });
  // the interpolating ops grouped by source cell: the fine ghost cells
  // prolonged from one coarse cell (up to 8) sit in neighbouring lanes and
  // their identical loads of the coarse cell and its neighbours merge
  std::stable_sort(ops.begin() + x->ncopy, ops.end(), [](const GhostOp& a, const GhostOp& b) {
    return a.src_block != b.src_block ? a.src_block < b.src_block : a.src_cell < b.src_cell;
  });
  x->nnbs = (long long)nbs.size();

  // ---- prefix sums per kernel ----
  for (int d = 0; d < 3; ++d) x->pre_face[d].assign(1, 0u);
  x->pre_zone.assign(1, 0u);
  x->pre_ct.assign(1, 0u);
  x->pre_alloc.assign(1, 0u);
  x->pre_all.assign(1, 0u);
  x->pre_corner.assign(1, 0u);
  for (int b = 0; b < nblocks; ++b) {
    const MBlock& m = x->hb[b];
    const Layout& L = m.L;
    for (int d = 0; d < 3; ++d) {
      const FaceBox& f = m.fb[d];
      x->pre_face[d].push_back(x->pre_face[d].back() + (unsigned)(f.n[0] * f.n[1] * f.n[2]));
    }
    x->pre_zone.push_back(x->pre_zone.back() + (unsigned)(L.n1 * L.n2 * L.n3));
    x->pre_ct.push_back(x->pre_ct.back() +
                        (unsigned)((L.e[0] - L.s[0] + 1) * (L.e[1] - L.s[1] + 1) * (L.ndim == 3 ? L.e[2] - L.s[2] + 1 : 1)));
    x->pre_alloc.push_back(x->pre_alloc.back() + (unsigned)L.plane);
    x->pre_all.push_back(x->pre_all.back() + (unsigned)(L.N1 * L.N2 * L.N3));
    x->pre_corner.push_back(x->pre_corner.back() +
                            (unsigned)((L.n1 - 1) * (L.n2 - 1) * (L.ndim == 3 ? L.n3 - 1 : 1)));
  }
  x->corners = x->pre_corner.back();

  // ---- face-centred CT: coarse edges on the surface of a finer block ----
  std::vector<EmfMatch> matches;
  if (c->bfield == KH_B_FACE) {
    const int nd = x->ndim;
    auto act = [&](int q) { return q < 2 || nd == 3; };
    for (int b = 0; b < nblocks; ++b)
      for (int f = 0; f < nblocks; ++f) {
        const MBlock& mb = x->hb[b];
        const MBlock& mf = x->hb[f];
        if (mf.level != mb.level + 1) continue;
        const int ob[3] = {mb.i0, mb.j0, mb.k0}, nb3[3] = {mb.L.n1, mb.L.n2, mb.L.n3};
        const int of[3] = {mf.i0, mf.j0, mf.k0}, nf3[3] = {mf.L.n1, mf.L.n2, mf.L.n3};
        bool touch = true;  // closed boxes in level-(l+1) indices
        for (int q = 0; q < 3; ++q)
          if (act(q) && (2 * (ob[q] + nb3[q]) < of[q] || of[q] + nf3[q] < 2 * ob[q])) touch = false;
        if (!touch) continue;
        for (int cdir = 0; cdir < 3; ++cdir) {
          int lo[3], hi[3];
          for (int q = 0; q < 3; ++q) {
            lo[q] = act(q) ? mb.L.s[q] : 0;
            hi[q] = act(q) ? (q == cdir ? mb.L.e[q] - 1 : mb.L.e[q]) : 0;
          }
          for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
              for (int i = lo[0]; i <= hi[0]; ++i) {
                const int l[3] = {i, j, k};
                bool edge_of_box = false;
                for (int q = 0; q < 3; ++q)
                  if (q != cdir && act(q) && (l[q] == mb.L.s[q] || l[q] == mb.L.e[q])) edge_of_box = true;
                if (!edge_of_box) continue;
                int fl[3][2], nfl[3];
                bool ok = true;
                for (int q = 0; q < 3; ++q) {
                  if (!act(q)) {
                    fl[q][0] = 0;
                    nfl[q] = 1;
                    continue;
                  }
                  const int G = ob[q] + (l[q] - mb.L.s[q]);
                  const int flo = mf.L.s[q], fhi = q == cdir ? mf.L.e[q] - 1 : mf.L.e[q];
                  nfl[q] = q == cdir ? 2 : 1;
                  for (int r = 0; r < nfl[q]; ++r) {
                    fl[q][r] = 2 * G + r - of[q] + mf.L.s[q];
                    if (fl[q][r] < flo || fl[q][r] > fhi) ok = false;
                  }
                }
                if (!ok) continue;
                EmfMatch M{};
                M.c = cdir;
                M.dst = mb.off + mb.L.at(k, j, i);
                M.n = 0;
                for (int r2 = 0; r2 < nfl[2]; ++r2)
                  for (int r1 = 0; r1 < nfl[1]; ++r1)
                    for (int r0 = 0; r0 < nfl[0]; ++r0)
                      M.src[M.n++] = mf.off + mf.L.at(fl[2][r2], fl[1][r1], fl[0][r0]);
                matches.push_back(M);
              }
        }
      }
  }
  x->nmatch = (long long)matches.size();

  // ---- device buffers ----
  int rc = KH_OK;
#define KM_ALLOC(ptr, bytes) \
  if (rc == KH_OK) rc = cuda_rc(cudaMalloc((void**)&(ptr), (bytes)));
  const bool mixed = c->precision == KH_MIXED;
  const size_t pl = (size_t)cells * sizeof(double), plf = (size_t)cells * sizeof(float);
  const size_t gp = (size_t)gcells * sizeof(double), gpf = (size_t)gcells * sizeof(float);
  KM_ALLOC(x->dblk, sizeof(MBlock) * nblocks);
  // prefix sums, each followed by its granule table (see find_block)
  const std::vector<unsigned>* pres[8] = {&x->pre_face[0], &x->pre_face[1], &x->pre_face[2], &x->pre_zone,
                                          &x->pre_ct,      &x->pre_alloc,   &x->pre_all,     &x->pre_corner};
  std::vector<unsigned> pretab[8];
  for (int q = 0; q < 8; ++q) {
    const std::vector<unsigned>& pr = *pres[q];
    const unsigned tot = pr.back();
    const size_t ngran = ((size_t)tot >> GRAN_SHIFT) + 1;
    pretab[q] = pr;
    int b = 0;
    for (size_t g = 0; g < ngran; ++g) {
      const unsigned t = (unsigned)(g << GRAN_SHIFT);
      while (b + 1 < nblocks && pr[b + 1] <= t) ++b;
      pretab[q].push_back((unsigned)b);
    }
    KM_ALLOC(x->dpre[q], sizeof(unsigned) * pretab[q].size());
  }
  KM_ALLOC(x->dops, sizeof(GhostOp) * std::max<long long>(x->nops, 1));
  KM_ALLOC(x->dcopy, sizeof(GhostCopy) * std::max<long long>(x->ncopy, 1));
  KM_ALLOC(x->dnbs, sizeof(ProlongNb) * std::max<long long>(x->nnbs, 1));
  KM_ALLOC(x->geo, 3 * NGEO * gp);
  KM_ALLOC(x->dgm, NDG * gp);
  KM_ALLOC(x->flo, 3 * gp);
  KM_ALLOC(x->pstar, NV * pl);
  KM_ALLOC(x->pflag, (size_t)cells);
  {
    bool list_ok = nblocks <= 4096;
    for (int b = 0; b < nblocks; ++b) list_ok = list_ok && x->hb[b].L.plane < (1LL << 20);
    if (list_ok) KM_ALLOC(x->flist, sizeof(unsigned) * (size_t)std::max<long long>(zones, 1));
  }
  if (!mixed) {
    for (int d = 0; d < x->ndim; ++d) {
      KM_ALLOC(x->F[d], NV * pl);
      KM_ALLOC(x->ctop[d], pl);
    }
    KM_ALLOC(x->emf[2], pl);
    if (x->ndim == 3 || c->bfield == KH_B_FACE) {
      KM_ALLOC(x->emf[0], pl);
      KM_ALLOC(x->emf[1], pl);
    }
    if (c->bfield == KH_B_FACE && c->emf == KH_EMF_GS05) KM_ALLOC(x->ecc, 3 * pl);
  } else {
    KM_ALLOC(x->geof, 3 * NGEO * gpf);
    KM_ALLOC(x->dgmf, NDG * gpf);
    KM_ALLOC(x->geodf, 2 * NDF * gpf);
    KM_ALLOC(x->pstarf, NV * plf);
    KM_ALLOC(x->pnf, NV * plf);
    for (int d = 0; d < x->ndim; ++d) {
      KM_ALLOC(x->Ff[d], NV * plf);
      KM_ALLOC(x->ctopf[d], plf);
    }
    KM_ALLOC(x->emff[2], plf);
    if (x->ndim == 3 || c->bfield == KH_B_FACE) {
      KM_ALLOC(x->emff[0], plf);
      KM_ALLOC(x->emff[1], plf);
    }
    if (c->bfield == KH_B_FACE && c->emf == KH_EMF_GS05) KM_ALLOC(x->eccf, 3 * plf);
  }
  if (c->bfield == KH_B_FACE) {
    KM_ALLOC(x->fBstar, 3 * pl);
    KM_ALLOC(x->dmatch, sizeof(EmfMatch) * std::max<long long>(x->nmatch, 1));
  }
  if (c->fofc) {
    KM_ALLOC(x->fflag, (size_t)cells);
    if (!mixed) KM_ALLOC(x->fsave, (size_t)x->ndim * NV * pl);
  }
  if (c->integrator != KH_INT_VL2)
    KM_ALLOC(x->rk, (size_t)(rk_states(c->integrator) + (c->integrator == KH_INT_SSPRK54 ? 2 : 1)) * NV * pl);
  x->npartial = 152 * 4;
  KM_ALLOC(x->partial, sizeof(double) * 2 * x->npartial);  // (max, sum) pairs for divB
  KM_ALLOC(x->dscalar, 4 * sizeof(double));
  KM_ALLOC(x->counters, NCNT * sizeof(unsigned long long));
#undef KM_ALLOC
  if (rc == KH_OK) rc = cuda_rc(cudaMemcpy(x->dblk, x->hb.data(), sizeof(MBlock) * nblocks, cudaMemcpyHostToDevice));
  for (int q = 0; q < 8 && rc == KH_OK; ++q)
    rc = cuda_rc(
        cudaMemcpy(x->dpre[q], pretab[q].data(), sizeof(unsigned) * pretab[q].size(), cudaMemcpyHostToDevice));
  if (rc == KH_OK && x->nops)
    rc = cuda_rc(cudaMemcpy(x->dops, ops.data(), sizeof(GhostOp) * x->nops, cudaMemcpyHostToDevice));
  if (rc == KH_OK && x->ncopy) {
    std::vector<GhostCopy> cops((size_t)x->ncopy);
    for (long long q = 0; q < x->ncopy && rc == KH_OK; ++q) {
      const GhostOp& o = ops[(size_t)q];
      if ((unsigned)o.src_cell >= (1u << 28) || o.flags >= 16) rc = KH_EINVAL;  // beyond the compact form
      cops[(size_t)q] = GhostCopy{o.dst_block, o.dst_cell, o.src_block, (unsigned)o.src_cell | ((unsigned)o.flags << 28)};
    }
    if (rc == KH_OK)
      rc = cuda_rc(cudaMemcpy(x->dcopy, cops.data(), sizeof(GhostCopy) * x->ncopy, cudaMemcpyHostToDevice));
  }
  if (rc == KH_OK && x->nnbs)
    rc = cuda_rc(cudaMemcpy(x->dnbs, nbs.data(), sizeof(ProlongNb) * x->nnbs, cudaMemcpyHostToDevice));
  if (rc == KH_OK && x->nmatch)
    rc = cuda_rc(cudaMemcpy(x->dmatch, matches.data(), sizeof(EmfMatch) * x->nmatch, cudaMemcpyHostToDevice));
  if (rc == KH_OK && x->fBstar) rc = cuda_rc(cudaMemset(x->fBstar, 0, 3 * pl));
  // the TMA-staged update: its tiles and the maps of the internal arrays (U^n's are made per step)
  x->tma_upd = mixed && x->ndim == 3 && c->bfield == KH_B_FLUXCT && c->inverter == KH_INV_NOBLE2D &&
               tensor_map_encoder() != nullptr;
  for (int b = 0; b < nblocks && x->tma_upd; ++b)
    if (x->hb[b].L.n1 != TMA_N1[0] && x->hb[b].L.n1 != TMA_N1[1]) x->tma_upd = 0;
  if (rc == KH_OK && x->tma_upd) {
    std::vector<MTile> tl;
    for (int cls = 0; cls < 2; ++cls) {
      const size_t t0 = tl.size();
      for (int b = 0; b < nblocks; ++b) {
        const Layout& L = x->hb[b].L;
        if (L.n1 != TMA_N1[cls]) continue;
        const int ty = 256 / L.n1;
        for (int k = L.s[2]; k < L.e[2]; ++k)
          for (int j0 = L.s[1]; j0 < L.e[1]; j0 += ty) tl.push_back(MTile{b, j0, k});
      }
      x->ntile[cls] = (long long)(tl.size() - t0);
    }
    x->nsets = c->integrator == KH_INT_VL2 ? 2 : 3;
    x->hmaps.resize((size_t)x->nsets * nblocks);
    const double* rkbase = x->rk ? x->rk + (size_t)rk_states(c->integrator) * NV * cells : nullptr;
    for (int b = 0; b < nblocks && x->tma_upd; ++b) {
      const MBlock& m = x->hb[b];
      const float* F[3] = {x->Ff[0] + NV * m.off, x->Ff[1] + NV * m.off, x->Ff[2] + NV * m.off};
      const float* E[3] = {x->emff[0] + m.off, x->emff[1] + m.off, x->emff[2] + m.off};
      const float* Pst[3] = {x->pnf + NV * m.off, x->pstarf + NV * m.off, x->pstarf + NV * m.off};
      for (int st = 0; st < x->nsets && x->tma_upd; ++st) {
        UpdateMaps& tm = x->hmaps[(size_t)x->nsets * b + st];
        // the caller's U^n (sets 0, 1) is encoded per step (refresh_umaps); set 2 reads the stage base
        const double* Ub = st == 2 ? rkbase + NV * m.off : nullptr;
        const bool ok = m.L.n1 == 16 ? encode_update_maps<UpdTile<16, 16>>(&tm, Pst[st], Ub, F, E, m.L.n1s,
                                                                             m.L.n2s, m.L.n3s)
                                     : encode_update_maps<UpdTile<32, 8>>(&tm, Pst[st], Ub, F, E, m.L.n1s,
                                                                            m.L.n2s, m.L.n3s);
        if (!ok) x->tma_upd = 0;
      }
    }
    if (x->tma_upd) {
      rc = cuda_rc(cudaMalloc((void**)&x->dtiles, sizeof(MTile) * std::max<size_t>(tl.size(), 1)));
      if (rc == KH_OK) rc = cuda_rc(cudaMalloc((void**)&x->dmaps, sizeof(UpdateMaps) * x->hmaps.size()));
      if (rc == KH_OK)
        rc = cuda_rc(cudaMemcpy(x->dtiles, tl.data(), sizeof(MTile) * tl.size(), cudaMemcpyHostToDevice));
    }
  }
  // zero scratch so never-written entries stay finite
  for (int d = 0; d < 3 && rc == KH_OK; ++d) {
    if (x->F[d]) rc = cuda_rc(cudaMemset(x->F[d], 0, NV * pl));
    if (rc == KH_OK && x->ctop[d]) rc = cuda_rc(cudaMemset(x->ctop[d], 0, pl));
    if (rc == KH_OK && x->emf[d]) rc = cuda_rc(cudaMemset(x->emf[d], 0, pl));
    if (rc == KH_OK && x->Ff[d]) rc = cuda_rc(cudaMemset(x->Ff[d], 0, NV * plf));
    if (rc == KH_OK && x->ctopf[d]) rc = cuda_rc(cudaMemset(x->ctopf[d], 0, plf));
    if (rc == KH_OK && x->emff[d]) rc = cuda_rc(cudaMemset(x->emff[d], 0, plf));
  }
  if (rc == KH_OK) rc = cuda_rc(cudaMemset(x->pstar, 0, NV * pl));
  if (rc == KH_OK && x->fflag) rc = cuda_rc(cudaMemset(x->fflag, 0, (size_t)cells));
  if (rc == KH_OK && x->pstarf) rc = cuda_rc(cudaMemset(x->pstarf, 0, NV * plf));
  if (rc == KH_OK && x->pnf) rc = cuda_rc(cudaMemset(x->pnf, 0, NV * plf));
  // geometry of every block
  for (int b = 0; b < nblocks && rc == KH_OK; ++b) {
    const MBlock& m = x->hb[b];
    const double x1o = c->x1min + m.i0 * m.L.dx[0];
    const double x2o = c->x2min + m.j0 * m.L.dx[1];
    x->launches += launch_geometry(x->cp, x1o, x2o, S.fl, m.L, x->geo + 3LL * NGEO * m.goff,
                                   x->dgm + (long long)NDG * m.goff, x->flo + 3 * m.goff, 0);
    rc = cuda_rc(cudaGetLastError());
  }
  if (rc == KH_OK && mixed) {
    x->launches += launch_to_f32(x->geo, x->geof, 3LL * NGEO * gcells, 0);
    x->launches += launch_to_f32(x->dgm, x->dgmf, (long long)NDG * gcells, 0);
    for (int b = 0; b < nblocks; ++b) {
      const MBlock& m = x->hb[b];
      x->launches += launch_df_planes(x->geo + 3LL * NGEO * m.goff, x->flo + 3 * m.goff, x->geodf + 2LL * NDF * m.goff,
                                      m.L.gplane, 0);
    }
    rc = cuda_rc(cudaGetLastError());
  }
  if (rc == KH_OK) rc = cuda_rc(cudaDeviceSynchronize());
  if (rc != KH_OK) {
    kh_mesh_destroy(x);
    return rc;
  }
  *out = x;
  return KH_OK;
}

}  // extern "C"

namespace {

GeoArena garena(const kh_mesh* x) { return GeoArena{x->geo, x->dgm, x->flo, x->geof, x->dgmf, x->geodf}; }

template <class T> Arena<T> arena8(T* p) { return Arena<T>{p, nullptr, NV}; }
Arena<double> arena_pb(double* P, double* B) { return Arena<double>{P, B, 5}; }

template <class T> int fill_ghosts(kh_mesh* x, const Arena<T>& P) {
  if (!x->nops) return 0;
  int n = 0;
  if (x->ncopy) {
    km_ghost_copy<T><<<nblk(x->ncopy, MTPB), MTPB, 0, x->stream>>>(x->dblk, x->dcopy, x->ncopy, P);
    ++n;
  }
  if (x->nops > x->ncopy) {
    km_ghost<T><<<nblk(x->nops - x->ncopy, MTPB), MTPB, 0, x->stream>>>(x->dblk, x->dops, x->ncopy, x->nops,
                                                                         x->dnbs, P);
    ++n;
  }
  return n;
}

// fluxct: Flux-CT after the face fluxes (its EMF phase; the field-flux phase
// too unless emf_only, for an update that forms the field fluxes from the
// EMFs).
// Flux-CT over all blocks: the edge EMFs, then (unless emf_only) the field
// fluxes rewritten from them.
template <class R> int ct_pass(kh_mesh* x, R* const F[3], R* const emf[3], bool emf_only) {
  const unsigned tot = x->pre_ct.back();
  int n = 0;
  for (int phase = 0; phase < (emf_only ? 1 : 2); ++phase) {
    km_ct<R><<<nblk(tot, MTPB), MTPB, 0, x->stream>>>(x->dblk, x->dpre[4], x->nb, F[0], F[1], F[2], emf[0], emf[1],
                                                      emf[2], phase);
    ++n;
  }
  return n;
}

template <class TIN, class R>
int flux_pass(kh_mesh* x, const Arena<TIN>& P, R* const F[3], R* const ct[3], R* const emf[3], bool fluxct = true,
              bool emf_only = false) {
  int n = 0;
  const GeoArena GA = garena(x);
  for (int d = 1; d <= x->ndim; ++d) {
    const unsigned tot = x->pre_face[d - 1].back();
    const int tpb = x->tpb_flux;
    const int g = nblk(tot, tpb);
#define KM_FLUX(DD)                                                                                             \
  if (x->S.recon == KH_RECON_MC)                                                                                \
    km_flux<DD, KH_RECON_MC, TIN, R><<<g, tpb, 0, x->stream>>>(x->dblk, x->dpre[DD - 1], x->nb, P, GA, x->S,    \
                                                               F[DD - 1], ct[DD - 1]);                          \
  else                                                                                                          \
    km_flux<DD, KH_RECON_WENO5, TIN, R><<<g, tpb, 0, x->stream>>>(x->dblk, x->dpre[DD - 1], x->nb, P, GA, x->S, \
                                                                  F[DD - 1], ct[DD - 1]);
    if (d == 1) { KM_FLUX(1) } else if (d == 2) { KM_FLUX(2) } else { KM_FLUX(3) }
#undef KM_FLUX
    ++n;
  }
  if (fluxct) n += ct_pass(x, F, emf, emf_only);
  return n;
}

// The first-order flux correction of one stage over all blocks (Flux-CT),
// after the flux pass: the trial update of every zone from U0 with the
// fluxes so far, the flags' ghost cells, donor-cell fluxes on the faces of
// the flagged zones (FP64: on the raw fluxes saved before Flux-CT, restored
// first), Flux-CT again (mixed: the EMFs only; its raw field fluxes were
// never overwritten).
template <class TIN, class R>
int fofc_pass(kh_mesh* x, const double* U0, const Arena<TIN>& P, R* const F[3], R* const ct[3], R* const emf[3],
              double coef) {
  cudaStream_t s = x->stream;
  const GeoArena GA = garena(x);
  const unsigned nz = x->pre_zone.back();
  const int g = nblk(nz, 256);
  constexpr bool mixed = sizeof(R) == sizeof(float);
  auto go = [&](auto kern) {
    if constexpr (mixed)
      kern<<<g, 256, 0, s>>>(x->dblk, x->dpre[3], x->nb, U0, P, F[0], F[1], F[2], GA, x->S, x->dscalar + 3, coef,
                             x->fflag, x->counters, x->ndim == 3 ? emf[0] : nullptr,
                             x->ndim == 3 ? emf[1] : nullptr, emf[2]);
    else
      kern<<<g, 256, 0, s>>>(x->dblk, x->dpre[3], x->nb, U0, P, F[0], F[1], F[2], GA, x->S, x->dscalar + 3, coef,
                             x->fflag, x->counters);
  };
  if constexpr (mixed) {
    if (x->S.c2p.method == C2P_KASTAUN) go(km_fofc_trial_mixed<C2P_KASTAUN>);
    else if (x->S.c2p.method == C2P_1DW) go(km_fofc_trial_mixed<C2P_1DW>);
    else if (x->S.mixed_fp64) go(km_fofc_trial_mixed<C2P_NOBLE2D_FP64>);
    else go(km_fofc_trial_mixed<C2P_NOBLE2D>);
  } else {
    if (x->S.c2p.method == C2P_KASTAUN) go(km_fofc_trial<C2P_KASTAUN>);
    else if (x->S.c2p.method == C2P_1DW) go(km_fofc_trial<C2P_1DW>);
    else go(km_fofc_trial<C2P_NOBLE2D>);
  }
  int n = 1;
  if (x->nops) {
    km_flag_ghost<<<nblk(x->nops, MTPB), MTPB, 0, s>>>(x->dblk, x->dops, x->nops, x->fflag);
    ++n;
  }
  if constexpr (!mixed) {
    const size_t bytes = (size_t)NV * x->cells * sizeof(double);
    for (int d = 0; d < x->ndim; ++d)
      cudaMemcpyAsync(F[d], x->fsave + (size_t)d * NV * x->cells, bytes, cudaMemcpyDeviceToDevice, s);
  }
  for (int d = 1; d <= x->ndim; ++d) {
    const unsigned tot = x->pre_face[d - 1].back();
    auto faces = [&](auto kern) {
      kern<<<nblk(tot, 256), 256, 0, s>>>(x->dblk, x->dpre[d - 1], x->nb, P, GA, x->S, x->fflag, F[d - 1],
                                          ct[d - 1]);
    };
    if (d == 1) faces(km_fofc_faces<1, TIN, R>);
    else if (d == 2) faces(km_fofc_faces<2, TIN, R>);
    else faces(km_fofc_faces<3, TIN, R>);
    ++n;
  }
  return n + ct_pass(x, F, emf, mixed);
}

// Face-centred CT of one stage over all blocks (after the flux pass without
// Flux-CT): cell EMFs (upwinded EMFs only), edge EMFs, interface matching,
// face update fBout = fB0 + coef dt curl E.
template <class R>
int face_ct_pass(kh_mesh* x, const Arena<R>& P, R* const F[3], R* ecc, R* const emf[3], double* fBout, double coef) {
  int n = 0;
  cudaStream_t s = x->stream;
  if (x->S.emf == KH_EMF_GS05) {
    km_cell_emf<R><<<nblk(x->pre_all.back(), MTPB), MTPB, 0, s>>>(x->dblk, x->dpre[6], x->nb, P, garena(x), ecc);
    ++n;
  }
  const unsigned tot = x->pre_ct.back();
  km_face_emf<R><<<nblk(tot, MTPB), MTPB, 0, s>>>(x->dblk, x->dpre[4], x->nb, F[0], F[1], F[2],
                                                  x->S.emf == KH_EMF_GS05 ? ecc : nullptr, emf[0], emf[1], emf[2],
                                                  x->S.emf);
  ++n;
  if (x->nmatch) {
    km_emf_match<R><<<nblk(x->nmatch, MTPB), MTPB, 0, s>>>(x->dmatch, x->nmatch, emf[0], emf[1], emf[2]);
    ++n;
  }
  km_face_update<R><<<nblk(tot, MTPB), MTPB, 0, s>>>(x->dblk, x->dpre[4], x->nb, x->fB, fBout, emf[0], emf[1],
                                                     emf[2], x->dscalar + 3, coef);
  return n + 1;
}

template <class T> int cfl_pass(kh_mesh* x, T* const ct[3]) {
  km_cfl<T><<<x->npartial, RED_THREADS, 0, x->stream>>>(x->dblk, x->dpre[3], x->nb, ct[0], ct[1], ct[2], x->S.cfl,
                                                        x->partial);
  km_cfl_finish<<<1, RED_THREADS, 0, x->stream>>>(x->partial, x->npartial, x->S.cfl, x->dscalar);
  return 2;
}

// The stage's failed-zone list (off when the mesh has none: more than 4096
// blocks, or a block allocation of 2^20 cells or more).
FailList mesh_list(const kh_mesh* x) {
  return x->flist ? FailList{x->flist, x->counters + CNT_LIST0, 0u} : FailList{nullptr, nullptr, 0u};
}
// Before a stage's update: its failed-zone list starts empty.
void start_list(kh_mesh* x) {
  if (x->flist) cudaMemsetAsync(x->counters + CNT_LIST0, 0, sizeof(unsigned long long), x->stream);
}
// The stage's fixup: over the failed-zone list (one warp per zone; the list
// is short in practice and its length known only on the device), else over
// every zone.
template <class T> void mesh_fixup(kh_mesh* x, const Arena<T>& P, double* Uout) {
  const unsigned nz = x->pre_zone.back();
  if (x->flist) {
    const long long b = std::min<long long>(nblk(nz, 256), 152);
    km_fixup_list<T><<<(unsigned)b, 256, 0, x->stream>>>(x->dblk, P, Uout, x->pflag, garena(x), x->S, x->counters,
                                                         mesh_list(x));
  } else {
    km_fixup<T><<<nblk(nz, MTPB), MTPB, 0, x->stream>>>(x->dblk, x->dpre[3], x->nb, P, Uout, x->pflag, garena(x), x->S,
                                                       x->counters);
  }
}

// The update kernels over all blocks, instantiated for the context's solver
// (the mixed path: double-float Noble-2D, or FP64 for every zone).
void km_update_any(const kh_mesh* x, int g, int t, const double* U0, const Arena<double>& Pin,
                   const Arena<double>& Pout, double* Uout, double coef, const double* fBn, double* dUout) {
  const GeoArena GA = garena(x);
  auto go = [&](auto kern) {
    kern<<<g, t, 0, x->stream>>>(x->dblk, x->dpre[3], x->nb, U0, Pin, Pout, Uout, x->F[0], x->F[1], x->F[2], GA,
                                 x->S, x->dscalar + 3, coef, x->pflag, x->counters, fBn, dUout, mesh_list(x));
  };
  if (x->S.c2p.method == C2P_KASTAUN) go(km_update<C2P_KASTAUN>);
  else if (x->S.c2p.method == C2P_1DW) go(km_update<C2P_1DW>);
  else go(km_update<C2P_NOBLE2D>);
}
void km_update_mixed_any(const kh_mesh* x, int g, int t, const double* U0, const Arena<float>& Pin,
                         const Arena<double>& Pout64, const Arena<float>& Pout32, double* Uout, double coef,
                         const double* fBn, const float* const* ce, double* dUout) {
  const GeoArena GA = garena(x);
  auto go = [&](auto kern) {
    kern<<<g, t, 0, x->stream>>>(x->dblk, x->dpre[3], x->nb, U0, Pin, Pout64, Pout32, Uout, x->Ff[0], x->Ff[1],
                                 x->Ff[2], GA, x->S, x->dscalar + 3, coef, x->pflag, x->counters, fBn, ce[0], ce[1],
                                 ce[2], dUout, mesh_list(x));
  };
  if (x->S.c2p.method == C2P_KASTAUN) go(km_update_mixed<C2P_KASTAUN>);
  else if (x->S.c2p.method == C2P_1DW) go(km_update_mixed<C2P_1DW>);
  else if (x->S.mixed_fp64) go(km_update_mixed<C2P_NOBLE2D_FP64>);
  else go(km_update_mixed<C2P_NOBLE2D>);
}

// Points the U^n maps of the staged update at U (the caller's conserved
// array) and copies the table to the device, ordered on the mesh's stream.
// Leaves the staged update off for this U if a map cannot be encoded (U not
// 16-byte aligned).
int refresh_umaps(kh_mesh* x, const double* U) {
  x->tma_now = 0;
  x->umap_key = U;
  for (int b = 0; b < x->nb; ++b) {
    const MBlock& m = x->hb[b];
    const double* Ub = U + NV * m.off;
    for (int st = 0; st < 2; ++st) {
      CUtensorMap* tm = &x->hmaps[(size_t)x->nsets * b + st].u;
      const bool ok = m.L.n1 == 16 ? encode_update_umap<UpdTile<16, 16>>(tm, Ub, m.L.n1s, m.L.n2s, m.L.n3s)
                                   : encode_update_umap<UpdTile<32, 8>>(tm, Ub, m.L.n1s, m.L.n2s, m.L.n3s);
      if (!ok) return KH_OK;
    }
  }
  const int rc = cuda_rc(cudaMemcpyAsync(x->dmaps, x->hmaps.data(), sizeof(UpdateMaps) * x->hmaps.size(),
                                         cudaMemcpyHostToDevice, x->stream));
  x->tma_now = rc == KH_OK;
  return rc;
}

template <int TX, int INV> bool mesh_tma_smem_once() {
  static bool done = false;
  if (!done)
    done = cudaFuncSetAttribute(km_update_mixed_tma<TX, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                UpdTile<TX, 256 / TX>::SMEM) == cudaSuccess;
  return done;
}

// The staged update of one stage over all blocks (one launch per block
// width); the number of launches, or -1.
int km_update_mixed_tma_all(const kh_mesh* x, int set, const Arena<double>& Pout64, const Arena<float>& Pout32,
                            double* Uout, double coef, double* dUout) {
  int n = 0;
  long long t0 = 0;
  for (int cls = 0; cls < 2; ++cls) {
    const long long nt = x->ntile[cls];
    if (!nt) continue;
    auto go = [&](auto kern, bool ok, int smem) {
      if (!ok) return false;
      kern<<<(unsigned)nt, 256, smem, x->stream>>>(x->dblk, x->dtiles + t0, x->dmaps, x->nsets, set, Pout64,
                                                   Pout32, Uout, garena(x), x->S, x->dscalar + 3, coef, x->pflag,
                                                   x->counters, (unsigned)KH_WAIT_POLLS, dUout, mesh_list(x));
      return true;
    };
    bool ok;
    if (cls == 0) {
      ok = x->S.mixed_fp64
               ? go(km_update_mixed_tma<16, C2P_NOBLE2D_FP64>, mesh_tma_smem_once<16, C2P_NOBLE2D_FP64>(),
                    UpdTile<16, 16>::SMEM)
               : go(km_update_mixed_tma<16, C2P_NOBLE2D>, mesh_tma_smem_once<16, C2P_NOBLE2D>(), UpdTile<16, 16>::SMEM);
    } else {
      ok = x->S.mixed_fp64
               ? go(km_update_mixed_tma<32, C2P_NOBLE2D_FP64>, mesh_tma_smem_once<32, C2P_NOBLE2D_FP64>(),
                    UpdTile<32, 8>::SMEM)
               : go(km_update_mixed_tma<32, C2P_NOBLE2D>, mesh_tma_smem_once<32, C2P_NOBLE2D>(), UpdTile<32, 8>::SMEM);
    }
    if (!ok) return -1;
    ++n;
    t0 += nt;
  }
  return n;
}

// One FP64 stage over all blocks: Pin's ghost cells, the fluxes (with
// Flux-CT, or face-centred CT moving the face field into fBst), the update
// U0 + coef dt (S - div F) -> Pout (Uout and dUout when given; Pin = Pout is
// allowed: every zone reads only its own input), the fixup.
int mesh_stage64(kh_mesh* x, const double* U0, const Arena<double>& Pin, const Arena<double>& Pout, double* Uout,
                 double coef, double* dUout, double* fBst) {
  const bool face = x->S.bfield == KH_B_FACE;
  const unsigned nz = x->pre_zone.back();
  int n = fill_ghosts(x, Pin);
  if (x->S.fofc) {
    // Flux-CT overwrites the raw field fluxes; the correction needs them again
    n += flux_pass<double, double>(x, Pin, x->F, x->ctop, x->emf, false);
    const size_t bytes = (size_t)NV * x->cells * sizeof(double);
    for (int d = 0; d < x->ndim; ++d)
      cudaMemcpyAsync(x->fsave + (size_t)d * NV * x->cells, x->F[d], bytes, cudaMemcpyDeviceToDevice, x->stream);
    n += ct_pass<double>(x, x->F, x->emf, false);
    n += fofc_pass<double, double>(x, U0, Pin, x->F, x->ctop, x->emf, coef);
  } else {
    n += flux_pass<double, double>(x, Pin, x->F, x->ctop, x->emf, !face);
  }
  if (face) n += face_ct_pass<double>(x, Pin, x->F, x->ecc, x->emf, fBst, coef);
  start_list(x);
  km_update_any(x, nblk(nz, x->tpb_update), x->tpb_update, U0, Pin, Pout, Uout, coef, face ? fBst : nullptr, dUout);
  mesh_fixup(x, Pout, Uout);
  return n + 2;
}

// One mixed stage over all blocks. first: the caller's FP64 P^n (Pn64)
// converted to FP32 (pnf) and ghost-filled there; otherwise the FP32 shadow
// (pstarf) ghost-filled in place. Outputs: the FP64 primitives (Pout64, the
// last stage) or the FP32 shadow (Pout32), Uout and dUout when given; set:
// the staged update's map set for this stage's input and U0 (-1: U0 has
// none).
int mesh_stage_mixed(kh_mesh* x, bool first, const double* U, const double* U0, const Arena<double>& Pn64,
                     const Arena<double>& Pout64, const Arena<float>& Pout32, double* Uout, double coef,
                     double* dUout, double* fBst, int set) {
  cudaStream_t s = x->stream;
  const bool face = x->S.bfield == KH_B_FACE;
  const unsigned nz = x->pre_zone.back();
  const Arena<float> Pin = first ? arena8(x->pnf) : arena8(x->pstarf);
  int n = 0;
  if (first) {
    km_to_f32_interior<<<nblk(nz, 256), 256, 0, s>>>(x->dblk, x->dpre[3], x->nb, Pn64, Pin);
    ++n;
  }
  n += fill_ghosts(x, Pin);
  // Flux-CT: EMFs only, the update forms the field fluxes from them
  const float* ce[3] = {face ? nullptr : x->emff[0], face ? nullptr : x->emff[1], face ? nullptr : x->emff[2]};
  n += flux_pass<float, float>(x, Pin, x->Ff, x->ctopf, x->emff, !face, true);
  if (x->S.fofc) n += fofc_pass<float, float>(x, U0, Pin, x->Ff, x->ctopf, x->emff, coef);
  if (face) n += face_ct_pass<float>(x, Pin, x->Ff, x->eccf, x->emff, fBst, coef);
  const bool staged = set >= 0 && x->tma_upd && !x->tma_off && x->tma_now && x->umap_key == U && !face;
  start_list(x);
  if (staged) {
    const int r = km_update_mixed_tma_all(x, set, Pout64, Pout32, Uout, coef, dUout);
    if (r < 0) return -1;
    n += r;
  } else {
    km_update_mixed_any(x, nblk(nz, x->tpb_update), x->tpb_update, U0, Pin, Pout64, Pout32, Uout, coef,
                        face ? fBst : nullptr, ce, dUout);
    ++n;
  }
  if (Pout64.a) mesh_fixup(x, Pout64, Uout);
  else mesh_fixup(x, Pout32, Uout);
  return n + 1;
}

// A Runge-Kutta step (RK1, RK2, SSPRK(5,4); Flux-CT) over all blocks: the
// stages of the single grid's Runge-Kutta step, each stage's input
// ghost-filled across blocks; stage bases formed over the whole arena. The
// FP64 path updates P in place; the mixed path enters with the caller's FP64
// P^n, carries the FP32 shadow between stages and writes the FP64 P^{n+1} at
// the last stage.
int issue_mesh_rk(kh_mesh* x, double* U, const Arena<double>& Pn) {
  cudaStream_t s = x->stream;
  const long long n8 = (long long)NV * x->cells;
  const int nst = rk_states(x->S.integrator);
  double* st[5] = {U, x->rk, x->rk + n8, x->rk + 2 * n8, x->rk + 3 * n8};
  double* base = x->rk + nst * n8;
  double* dU4 = base + n8;
  const int nstage = x->S.integrator == KH_INT_SSPRK54 ? 5 : (x->S.integrator == KH_INT_RK2 ? 2 : 1);
  const Arena<double> none64{nullptr, nullptr, NV};
  const Arena<float> none32{nullptr, nullptr, NV};
  int n = 0;
  bool ok = true;
  auto stage = [&](int q, const double* U0, double* Uout, double c, double* dUout) {
    if (x->c.precision == KH_FP64) {
      n += mesh_stage64(x, U0, Pn, Pn, Uout, c, dUout, nullptr);
      return;
    }
    const bool last = q == nstage - 1;
    // map sets: the first stage reads P^n and the caller's U, later ones the shadow and the base
    const int set = q == 0 ? 0 : (U0 == base ? 2 : -1);
    const int r = mesh_stage_mixed(x, q == 0, U, U0, Pn, last ? Pn : none64, last ? none32 : arena8(x->pstarf), Uout,
                                   c, dUout, nullptr, set);
    if (r < 0) ok = false;
    n += r;
  };
  auto comb = [&](int nt, const double* const* in, const double* a) { n += launch_lincomb(base, nt, in, a, n8, s); };
  if (x->S.integrator == KH_INT_RK1) {
    stage(0, U, U, 1.0, nullptr);
  } else if (x->S.integrator == KH_INT_RK2) {
    stage(0, U, st[1], 1.0, nullptr);
    const double* in[2] = {U, st[1]};
    const double a[2] = {0.5, 0.5};
    comb(2, in, a);
    stage(1, base, U, 0.5, nullptr);
  } else {
    using T = Ssprk54;
    stage(0, U, st[1], T::c1, nullptr);
    for (int q = 1; q <= 3; ++q) {
      const double* in[2] = {U, st[q]};
      comb(2, in, T::a[q - 1]);
      stage(q, base, st[q + 1], T::c[q - 1], q == 3 ? dU4 : nullptr);
    }
    const double a[4] = {T::a5[0], T::a5[1], T::a5[2], T::c53 / T::c[2]};
    const double* in[4] = {st[2], st[3], st[4], dU4};
    comb(4, in, a);
    stage(4, base, U, T::c5, nullptr);
  }
  return ok ? n : -1;
}

int issue_mesh_step(kh_mesh* x, double* U, double* P, double* B) {
  if (cudaMemsetAsync(x->counters, 0, NCNT * sizeof(unsigned long long), x->stream) != cudaSuccess) return -1;
  const Arena<double> Pn = arena_pb(P, B);
  const bool face = x->S.bfield == KH_B_FACE;
  const bool fp64 = x->c.precision == KH_FP64;
  int n = 0;
  if (x->S.integrator != KH_INT_VL2) {
    const int r = issue_mesh_rk(x, U, Pn);
    if (r < 0) return -1;
    n += r;
  } else if (fp64) {
    // stage 1: P^n -> P* (U* is not stored); stage 2: P* -> P^{n+1}, U^{n+1}
    const Arena<double> Ps = arena8(x->pstar);
    n += mesh_stage64(x, U, Pn, Ps, nullptr, 0.5, nullptr, face ? x->fBstar : nullptr);
    n += mesh_stage64(x, U, Ps, Pn, U, 1.0, nullptr, face ? x->fB : nullptr);
  } else {
    // stage 1: FP64 P^n (converted once, then ghost-filled in FP32) -> FP32 P*; stage 2: FP32 P* -> FP64 P^{n+1}, U^{n+1}
    const Arena<double> none64{nullptr, nullptr, NV};
    const Arena<float> none32{nullptr, nullptr, NV};
    int r = mesh_stage_mixed(x, true, U, U, Pn, none64, arena8(x->pstarf), nullptr, 0.5, nullptr,
                             face ? x->fBstar : nullptr, 0);
    if (r < 0) return -1;
    n += r;
    r = mesh_stage_mixed(x, false, U, U, Pn, Pn, none32, U, 1.0, nullptr, face ? x->fB : nullptr, 1);
    if (r < 0) return -1;
    n += r;
  }
  n += fp64 ? cfl_pass<double>(x, x->ctop) : cfl_pass<float>(x, x->ctopf);
  return n;
}

void drop_mesh_graph(kh_mesh* x) {
  if (x->gexec) cudaGraphExecDestroy(x->gexec);
  x->gexec = nullptr;
  x->gkey[0] = x->gkey[1] = x->gkey[2] = nullptr;
}

}  // namespace

extern "C" {

int kh_mesh_block_shape(const kh_mesh* x, int b, int* n1s, int* n2s, int* n3s, int64_t* cell_offset) {
  if (!x || b < 0 || b >= x->nb) return KH_EINVAL;
  const Layout& L = x->hb[b].L;
  if (n1s) *n1s = L.n1s;
  if (n2s) *n2s = L.n2s;
  if (n3s) *n3s = L.n3s;
  if (cell_offset) *cell_offset = x->hb[b].off;
  return KH_OK;
}

int64_t kh_mesh_cells(const kh_mesh* x) { return x ? (int64_t)x->cells : 0; }
int64_t kh_mesh_zones(const kh_mesh* x) { return x ? (int64_t)x->zones : 0; }
int64_t kh_mesh_ghost_cells(const kh_mesh* x) { return x ? (int64_t)x->nops : 0; }
int64_t kh_mesh_launch_count(const kh_mesh* x) { return x ? (int64_t)x->launches : 0; }

int kh_mesh_set_stream(kh_mesh* x, void* s) {
  if (!x) return KH_EINVAL;
  x->stream = (cudaStream_t)s;
  drop_mesh_graph(x);
  return KH_OK;
}

int kh_mesh_prim_to_cons(kh_mesh* x, const double* P, const double* B, double* U) {
  if (!x || !P || !B || !U) return KH_EINVAL;
  const unsigned tot = x->pre_all.back();
  km_p2c<<<nblk(tot, MTPB), MTPB, 0, x->stream>>>(x->dblk, x->dpre[6], x->nb,
                                                  arena_pb(const_cast<double*>(P), const_cast<double*>(B)), U,
                                                  garena(x), x->S);
  x->launches += 1;
  return cuda_rc(cudaGetLastError());
}

int kh_mesh_fill_ghosts(kh_mesh* x, double* P, double* B) {
  if (!x || !P || !B) return KH_EINVAL;
  x->launches += fill_ghosts(x, arena_pb(P, B));
  return cuda_rc(cudaGetLastError());
}

int kh_mesh_cfl_dt(kh_mesh* x, const double* P, const double* B, double* dt_cfl) {
  if (!x || !P || !B || !dt_cfl) return KH_EINVAL;
  cudaStream_t s = x->stream;
  // ghost-fill a scratch copy (block by block: P is a [block][5][plane], B a [block][3][plane] arena)
  for (int b = 0; b < x->nb; ++b) {
    const MBlock& m = x->hb[b];
    const size_t pl = (size_t)m.L.plane * sizeof(double);
    int rc = cuda_rc(cudaMemcpyAsync(x->pstar + NV * m.off, P + 5 * m.off, 5 * pl, cudaMemcpyDeviceToDevice, s));
    if (rc == KH_OK)
      rc = cuda_rc(cudaMemcpyAsync(x->pstar + NV * m.off + 5 * m.L.plane, B + 3 * m.off, 3 * pl,
                                   cudaMemcpyDeviceToDevice, s));
    if (rc != KH_OK) return rc;
  }
  const Arena<double> Ps = arena8(x->pstar);
  int n = fill_ghosts(x, Ps);
  if (x->c.precision == KH_FP64) {
    n += flux_pass<double, double>(x, Ps, x->F, x->ctop, x->emf);
    n += cfl_pass<double>(x, x->ctop);
  } else {
    km_to_f32<<<nblk(x->pre_alloc.back(), 256), 256, 0, s>>>(x->dblk, x->dpre[5], x->nb, Ps, arena8(x->pnf));
    n += 1;
    n += flux_pass<float, float>(x, arena8(x->pnf), x->Ff, x->ctopf, x->emff);
    n += cfl_pass<float>(x, x->ctopf);
  }
  x->launches += n;
  int rc = cuda_rc(cudaGetLastError());
  if (rc != KH_OK) return rc;
  rc = cuda_rc(cudaMemcpyAsync(dt_cfl, x->dscalar, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (rc == KH_OK) rc = cuda_rc(cudaStreamSynchronize(s));
  if (rc != KH_OK) return rc;
  return isfinite(*dt_cfl) ? KH_OK : KH_ENAN;
}

int kh_mesh_divb(kh_mesh* x, const double* B, double* max_abs, double* l1) {
  if (!x || !B) return KH_EINVAL;
  cudaStream_t s = x->stream;
  km_divb<<<x->npartial, RED_THREADS, 0, s>>>(x->dblk, x->dpre[7], x->nb, B, x->geo, x->partial);
  km_max_sum_finish<<<1, RED_THREADS, 0, s>>>(x->partial, x->npartial, x->dscalar + 1);
  x->launches += 2;
  int rc = cuda_rc(cudaGetLastError());
  double h[2];
  if (rc == KH_OK) rc = cuda_rc(cudaMemcpyAsync(h, x->dscalar + 1, sizeof(h), cudaMemcpyDeviceToHost, s));
  if (rc == KH_OK) rc = cuda_rc(cudaStreamSynchronize(s));
  if (rc != KH_OK) return rc;
  if (max_abs) *max_abs = h[0];
  if (l1) *l1 = x->corners > 0 ? h[1] / (double)x->corners : 0.0;
  return KH_OK;
}

int kh_mesh_get_stats(kh_mesh* x, kh_stats* out) {
  if (!x || !out) return KH_EINVAL;
  unsigned long long h[NCNT];
  double dt;
  int rc = cuda_rc(cudaMemcpyAsync(h, x->counters, sizeof(h), cudaMemcpyDeviceToHost, x->stream));
  if (rc == KH_OK) rc = cuda_rc(cudaMemcpyAsync(&dt, x->dscalar, sizeof(double), cudaMemcpyDeviceToHost, x->stream));
  if (rc == KH_OK) rc = cuda_rc(cudaStreamSynchronize(x->stream));
  if (rc != KH_OK) return rc;
  out->nfail = (int64_t)h[CNT_FAIL];
  out->nfloor = (int64_t)h[CNT_FLOOR];
  out->nunfixed = (int64_t)h[CNT_UNFIXED];
  out->nfp64 = (int64_t)h[CNT_FP64];
  out->nfofc = (int64_t)h[CNT_FOFC];
  out->nbounds = 0;
  out->dt_cfl = dt;
  return KH_OK;
}

int kh_mesh_set_face_field(kh_mesh* x, double* fB) {
  if (!x || !fB || x->S.bfield != KH_B_FACE) return KH_EINVAL;
  if (x->fB != fB) drop_mesh_graph(x);
  x->fB = fB;
  return KH_OK;
}

int kh_mesh_step(kh_mesh* x, double* U, double* P, double* B, double dt, double* dt_cfl) {
  if (!x || !U || !P || !B || !(dt > 0.0) || !isfinite(dt)) return KH_EINVAL;
  if (x->S.bfield == KH_B_FACE && !x->fB) return KH_EINVAL;
  int rc = cuda_rc(cudaMemcpyAsync(x->dscalar + 3, &dt, sizeof(double), cudaMemcpyHostToDevice, x->stream));
  if (rc != KH_OK) return rc;
  if (x->tma_upd && x->umap_key != U) {
    rc = refresh_umaps(x, U);
    if (rc != KH_OK) return rc;
  }
  if (x->graph_on) {
    if (!(x->gexec && x->gkey[0] == U && x->gkey[1] == P && x->gkey[2] == B)) {
      drop_mesh_graph(x);
      if (!x->cap_stream && cudaStreamCreateWithFlags(&x->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return KH_ECUDA;
      cudaStream_t user = x->stream;
      x->stream = x->cap_stream;
      if (cudaStreamBeginCapture(x->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        x->stream = user;
        return KH_ECUDA;
      }
      const int n = issue_mesh_step(x, U, P, B);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(x->cap_stream, &g);
      x->stream = user;
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
      x->graph_launches = n;
    }
    if (cudaGraphLaunch(x->gexec, x->stream) != cudaSuccess) return KH_ECUDA;
    x->launches += x->graph_launches;
  } else {
    const int n = issue_mesh_step(x, U, P, B);
    if (n < 0) return KH_ECUDA;
    x->launches += n;
  }
  rc = cuda_rc(cudaGetLastError());
  if (rc != KH_OK || !dt_cfl) return rc;
  kh_stats st;
  rc = kh_mesh_get_stats(x, &st);
  if (rc != KH_OK) return rc;
  *dt_cfl = st.dt_cfl;
  if (!isfinite(st.dt_cfl)) return KH_ENAN;
  return (int)(st.nfail > 0x7fffffffLL ? 0x7fffffff : st.nfail);
}

int kh_mesh_set_launch(kh_mesh* x, int tpb_flux, int tpb_update) {
  if (!x) return KH_EINVAL;
  auto ok = [](int t) { return t >= 32 && t <= 256 && t % 32 == 0; };
  if (!ok(tpb_flux) || !ok(tpb_update)) return KH_EINVAL;
  x->tpb_flux = tpb_flux;
  x->tpb_update = tpb_update;
  drop_mesh_graph(x);
  return KH_OK;
}

int kh_mesh_get_launch(const kh_mesh* x, int* tpb_flux, int* tpb_update) {
  if (!x) return KH_EINVAL;
  if (tpb_flux) *tpb_flux = x->tpb_flux;
  if (tpb_update) *tpb_update = x->tpb_update;
  return KH_OK;
}

int kh_mesh_autotune(kh_mesh* x, const double* U, const double* P, const double* B, double dt, int* tpb_flux,
                     int* tpb_update) {
  if (!x || !U || !P || !B || !(dt > 0.0)) return KH_EINVAL;
  // process-wide cache keyed by the block shapes (with counts), coordinates,
  // reconstruction and precision
  static std::mutex lock;
  static std::map<std::string, std::pair<int, int>> cache;
  std::map<std::tuple<int, int, int, int>, int> shapes;
  for (const MBlock& m : x->hb) ++shapes[std::make_tuple(m.level, m.L.n1, m.L.n2, m.L.n3)];
  std::string key = std::to_string(x->c.kind) + "/" + std::to_string(x->c.recon) + "/" +
                    std::to_string(x->c.precision);
  for (const auto& kv : shapes)
    key += "/" + std::to_string(std::get<1>(kv.first)) + "x" + std::to_string(std::get<2>(kv.first)) + "x" +
           std::to_string(std::get<3>(kv.first)) + "L" + std::to_string(std::get<0>(kv.first)) + ":" +
           std::to_string(kv.second);
  {
    std::lock_guard<std::mutex> g(lock);
    auto it = cache.find(key);
    if (it != cache.end()) {
      const int rc = kh_mesh_set_launch(x, it->second.first, it->second.second);
      if (tpb_flux) *tpb_flux = x->tpb_flux;
      if (tpb_update) *tpb_update = x->tpb_update;
      return rc;
    }
  }
  const size_t pl = (size_t)x->cells * sizeof(double);
  double *Us = nullptr, *Ps = nullptr, *Bs = nullptr;
  int rc = cuda_rc(cudaMalloc((void**)&Us, 8 * pl));
  if (rc == KH_OK) rc = cuda_rc(cudaMalloc((void**)&Ps, 5 * pl));
  if (rc == KH_OK) rc = cuda_rc(cudaMalloc((void**)&Bs, 3 * pl));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == KH_OK) rc = cuda_rc(cudaEventCreate(&e0));
  if (rc == KH_OK) rc = cuda_rc(cudaEventCreate(&e1));
  const int graph = x->graph_on;
  x->graph_on = 0;
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
        rc = cuda_rc(cudaMemcpyAsync(Us, U, 8 * pl, cudaMemcpyDeviceToDevice, x->stream));
        if (rc == KH_OK) rc = cuda_rc(cudaMemcpyAsync(Ps, P, 5 * pl, cudaMemcpyDeviceToDevice, x->stream));
        if (rc == KH_OK) rc = cuda_rc(cudaMemcpyAsync(Bs, B, 3 * pl, cudaMemcpyDeviceToDevice, x->stream));
        if (rc == KH_OK) rc = cuda_rc(cudaEventRecord(e0, x->stream));
        if (rc == KH_OK) {
          const int r = kh_mesh_step(x, Us, Ps, Bs, dt, nullptr);
          rc = r < 0 ? r : KH_OK;
        }
        if (rc == KH_OK) rc = cuda_rc(cudaEventRecord(e1, x->stream));
        if (rc == KH_OK) rc = cuda_rc(cudaEventSynchronize(e1));
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
  drop_mesh_graph(x);
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

int kh_mesh_set_staged_update(kh_mesh* x, int enable) {
  if (!x) return KH_EINVAL;
  if (x->tma_off != !enable) drop_mesh_graph(x);
  x->tma_off = !enable;
  return x->tma_upd && !x->tma_off ? 1 : 0;
}

int kh_mesh_set_graph(kh_mesh* x, int enable) {
  if (!x) return KH_EINVAL;
  if (!enable) drop_mesh_graph(x);
  x->graph_on = enable ? 1 : 0;
  return KH_OK;
}

int kh_mesh_destroy(kh_mesh* x) {
  if (!x) return KH_EINVAL;
  cudaStreamSynchronize(x->stream);
  drop_mesh_graph(x);
  if (x->cap_stream) cudaStreamDestroy(x->cap_stream);
  void* ptrs[] = {x->dblk, x->dops, x->dcopy, x->dnbs, x->geo, x->dgm, x->flo, x->geof, x->dgmf, x->geodf, x->pstar, x->pstarf, x->pnf,
                  x->pflag, x->flist, x->partial, x->dscalar, x->counters, x->F[0], x->F[1], x->F[2], x->ctop[0],
                  x->ctop[1], x->ctop[2], x->emf[0], x->emf[1], x->emf[2], x->Ff[0], x->Ff[1], x->Ff[2],
                  x->ctopf[0], x->ctopf[1], x->ctopf[2], x->emff[0], x->emff[1], x->emff[2],
                  x->fBstar, x->ecc, x->eccf, x->dmatch, x->dtiles, x->dmaps, x->rk, x->fflag, x->fsave};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int q = 0; q < 8; ++q)
    if (x->dpre[q]) cudaFree(x->dpre[q]);
  delete x;
  return KH_OK;
}

}  // extern "C"
