// The mixed path's update with its inputs staged in shared memory by TMA.
//
// The update of a zone reads the stage input P (8 FP32), U^n (8 FP64), the
// fluid variables' face fluxes in three directions (both faces of the zone)
// and Flux-CT's edge EMFs around it -- ~60 values from six arrays, the
// fluxes and EMFs just written by the face and EMF kernels and mostly no
// longer in L2. Read by the threads themselves, those loads hold the
// registers of a kernel whose arithmetic (the double-float inversion) wants
// ~220 of them, and their DRAM latency is exposed at the ~35% occupancy the
// register budget leaves. Here one CTA updates a tile of 32 (x1) x 8 (x2)
// zones of one x3 plane: thread 0 issues eight tensor copies (P, U^n, the
// three flux arrays, the three EMF arrays; boxes covering the tile plus the
// upper faces and edges it needs) on one mbarrier, the copy engine moves
// them while the SM runs other CTAs, and every thread then runs the same
// per-zone update (update_mixed_zone_in) reading its values from the tiles.
//
// Tile boxes start at a 16-byte boundary at or below the tile's first zone
// along x1 (the innermost coordinate: a multiple of 4 floats, 2 doubles);
// cells past the array's end are zero-filled by the copy and belong only to
// zones past the interior, which are skipped.
#include "kh_tma.cuh"
#include "kh_zone.cuh"

namespace kh {
namespace {

constexpr int TX = 32, TY = 8;  // zones per tile along x1, x2
constexpr int PX = 36;          // floats per staged row (32 + alignment slack + the upper face)
constexpr int UX = 34;          // doubles per staged row of U^n
constexpr int NFL = 5;          // fluid variables whose face fluxes are staged (the field's come from the EMFs)

constexpr int round128(int b) { return (b + 127) / 128 * 128; }
// box bytes per staged array, and their shared-memory offsets (128-byte aligned)
constexpr int B_P = 4 * PX * TY * NV;
constexpr int B_F1 = 4 * PX * TY * NFL;
constexpr int B_F2 = 4 * PX * (TY + 1) * NFL;
constexpr int B_F3 = 4 * PX * TY * 2 * NFL;
constexpr int B_E1 = 4 * PX * (TY + 1) * 2;
constexpr int B_E2 = 4 * PX * TY * 2;
constexpr int B_E3 = 4 * PX * (TY + 1);
constexpr int B_U = 8 * UX * TY * NV;
constexpr int O_P = 0;
constexpr int O_F1 = O_P + round128(B_P);
constexpr int O_F2 = O_F1 + round128(B_F1);
constexpr int O_F3 = O_F2 + round128(B_F2);
constexpr int O_E1 = O_F3 + round128(B_F3);
constexpr int O_E2 = O_E1 + round128(B_E1);
constexpr int O_E3 = O_E2 + round128(B_E2);
constexpr int O_U = O_E3 + round128(B_E3);
constexpr int O_BAR = O_U + round128(B_U);
constexpr int SMEM = O_BAR + 128 + 128;  // + slack to align the dynamic base to 128 bytes
constexpr unsigned TX_BYTES = B_P + B_F1 + B_F2 + B_F3 + B_E1 + B_E2 + B_E3 + B_U;

// The mixed update's inputs from the staged tiles (see MixedInGlobal): x is
// the zone's column in the float tiles, xu in the FP64 tile, y its row.
struct MixedInTile {
  const float *p, *f1, *f2, *f3, *e1, *e2, *e3;
  const double* u;
  int x, xu, y;
  __device__ __forceinline__ float pin(int v) const { return p[(v * TY + y) * PX + x]; }
  __device__ __forceinline__ double u0(int v) const { return u[(v * TY + y) * UX + xu]; }
  __device__ __forceinline__ float f(int d, int v, int up) const {
    if (d == 0) return f1[(v * TY + y) * PX + x + up];
    if (d == 1) return f2[(v * (TY + 1) + y + up) * PX + x];
    return f3[((v * 2 + up) * TY + y) * PX + x];
  }
  __device__ __forceinline__ float e(int a, int di, int dj, int dk) const {
    if (a == 0) return e1[(dk * (TY + 1) + y + dj) * PX + x + di];
    if (a == 1) return e2[(dk * TY + y + dj) * PX + x + di];
    return e3[(y + dj) * PX + x + di];
  }
  __device__ __forceinline__ bool has_emf() const { return true; }
};

struct UpdateMaps {
  CUtensorMap p, f1, f2, f3, e1, e2, e3, u;
};

template <int INV>
__global__ void __launch_bounds__(TX * TY, 3)
    k_update_mixed_tma(const __grid_constant__ UpdateMaps tm, Vars Pout64, VarsT<float> Pout32, double* Uout,
                       Layout L, DevGeom G, GeomT<float> Gf, Scheme S, const double* dtp, double coef, int8_t* pflag,
                       unsigned long long* cnt, FailList fl, double* dUout, unsigned wlim) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + O_BAR);
  const int lx = threadIdx.x & (TX - 1), ly = threadIdx.x / TX;
  const int i0 = L.s[0] + TX * (int)blockIdx.x, j0 = L.s[1] + TY * (int)blockIdx.y, k = L.s[2] + (int)blockIdx.z;
  const int x0 = i0 & ~3, xu0 = i0 & ~1;  // 16-byte boundaries at or below i0
  if (threadIdx.x == 0) mbar_init(bar);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, TX_BYTES);
    tma_load_4d(smem + O_P, &tm.p, x0, j0, k, 0, bar);
    tma_load_4d(smem + O_F1, &tm.f1, x0, j0, k, 0, bar);
    tma_load_4d(smem + O_F2, &tm.f2, x0, j0, k, 0, bar);
    tma_load_4d(smem + O_F3, &tm.f3, x0, j0, k, 0, bar);
    tma_load_3d(smem + O_E1, &tm.e1, x0, j0, k, bar);
    tma_load_3d(smem + O_E2, &tm.e2, x0, j0, k, bar);
    tma_load_3d(smem + O_E3, &tm.e3, x0, j0, k, bar);
    tma_load_4d(smem + O_U, &tm.u, xu0, j0, k, 0, bar);
  }
  if (!cta_wait_tiles(bar, wlim, cnt)) return;
  const int i = i0 + lx, j = j0 + ly;
  if (i >= L.e[0] || j >= L.e[1]) return;  // ragged tile
  if (KH_OOB(L, kh_in(L, i, j, k, 1))) return;
  const MixedInTile in{reinterpret_cast<const float*>(smem + O_P),  reinterpret_cast<const float*>(smem + O_F1),
                       reinterpret_cast<const float*>(smem + O_F2), reinterpret_cast<const float*>(smem + O_F3),
                       reinterpret_cast<const float*>(smem + O_E1), reinterpret_cast<const float*>(smem + O_E2),
                       reinterpret_cast<const float*>(smem + O_E3), reinterpret_cast<const double*>(smem + O_U),
                       (i0 - x0) + lx, (i0 - xu0) + lx, ly};
  update_mixed_zone_in<false, INV, MixedInTile, true>(in, Pout64, Pout32, Uout, L, G, Gf, S,
                                                      df_of_f64(coef * __ldg(dtp)), pflag, cnt, i, j, k, fl, nullptr,
                                                      dUout);
}

template <int INV> bool set_smem_once() {
  static bool done = false;
  if (!done)
    done = cudaFuncSetAttribute(k_update_mixed_tma<INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM) ==
           cudaSuccess;
  return done;
}

}  // namespace

int launch_update_mixed_tma(const double* U0, const float* P8, const Vars& Pout64, const VarsT<float>& Pout32,
                            double* Uout, float* const F[3], float* const emf[3], const Layout& L, const DevGeom& G,
                            const GeomT<float>& Gf, const Scheme& S, const double* dtp, double coef, int8_t* pflag,
                            unsigned long long* cnt, FailList fl, double* dUout, unsigned wlim, cudaStream_t s) {
  if (L.ndim != 3 || !P8 || !U0 || !F[0] || !F[1] || !F[2] || !emf[0] || !emf[1] || !emf[2]) return -1;
  const cuuint64_t d4[4] = {(cuuint64_t)L.n1s, (cuuint64_t)L.n2s, (cuuint64_t)L.n3s, (cuuint64_t)NV};
  const cuuint64_t s4f[3] = {(cuuint64_t)L.n1s * 4, (cuuint64_t)L.gplane * 4, (cuuint64_t)L.plane * 4};
  const cuuint64_t s4d[3] = {(cuuint64_t)L.n1s * 8, (cuuint64_t)L.gplane * 8, (cuuint64_t)L.plane * 8};
  const cuuint64_t s3f[2] = {(cuuint64_t)L.n1s * 4, (cuuint64_t)L.gplane * 4};
  const cuuint32_t bP[4] = {PX, TY, 1, NV}, bF1[4] = {PX, TY, 1, NFL}, bF2[4] = {PX, TY + 1, 1, NFL},
                   bF3[4] = {PX, TY, 2, NFL}, bE1[3] = {PX, TY + 1, 2}, bE2[3] = {PX, TY, 2}, bE3[3] = {PX, TY + 1, 1},
                   bU[4] = {UX, TY, 1, NV};
  const auto F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  UpdateMaps tm;
  if (!encode_tiled(&tm.p, F32, 4, P8, d4, s4f, bP) || !encode_tiled(&tm.f1, F32, 4, F[0], d4, s4f, bF1) ||
      !encode_tiled(&tm.f2, F32, 4, F[1], d4, s4f, bF2) || !encode_tiled(&tm.f3, F32, 4, F[2], d4, s4f, bF3) ||
      !encode_tiled(&tm.e1, F32, 3, emf[0], d4, s3f, bE1) || !encode_tiled(&tm.e2, F32, 3, emf[1], d4, s3f, bE2) ||
      !encode_tiled(&tm.e3, F32, 3, emf[2], d4, s3f, bE3) ||
      !encode_tiled(&tm.u, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, U0, d4, s4d, bU))
    return -1;
  const dim3 grid((L.n1 + TX - 1) / TX, (L.n2 + TY - 1) / TY, L.n3);
  auto go = [&](auto kern, bool ok) {
    if (!ok) return false;
    kern<<<grid, TX * TY, SMEM, s>>>(tm, Pout64, Pout32, Uout, L, G, Gf, S, dtp, coef, pflag, cnt, fl, dUout, wlim);
    return true;
  };
  bool ok;
  if (S.c2p.method == C2P_KASTAUN) ok = go(k_update_mixed_tma<C2P_KASTAUN>, set_smem_once<C2P_KASTAUN>());
  else if (S.c2p.method == C2P_1DW) ok = go(k_update_mixed_tma<C2P_1DW>, set_smem_once<C2P_1DW>());
  else if (S.mixed_fp64) ok = go(k_update_mixed_tma<C2P_NOBLE2D_FP64>, set_smem_once<C2P_NOBLE2D_FP64>());
  else ok = go(k_update_mixed_tma<C2P_NOBLE2D>, set_smem_once<C2P_NOBLE2D>());
  return ok ? 1 : -1;
}

}  // namespace kh
