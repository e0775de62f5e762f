// Shared-memory tiles of the mixed path's update, staged by TMA: the tile
// geometry, the tensor maps, the eight copies and the per-zone update that
// reads them. Used by the single grid's update (kh_update_tma.cu) and by the
// refined mesh's (kh_mesh.cu).
//
// A tile is TX (x1) x TY (x2) zones of one x3 plane, one zone per thread.
// Its inputs are the stage input P (8 FP32 planes), U^n (8 FP64 planes), the
// fluid variables' face fluxes in three directions (both faces of every
// zone) and Flux-CT's three edge-EMF arrays (the edges around every zone):
// eight boxes covering the tile plus the upper faces and edges it needs,
// copied by thread 0 on one mbarrier. Boxes start at a 16-byte boundary at
// or below the tile's first zone along x1 (the innermost coordinate: a
// multiple of 4 floats, 2 doubles); cells past the array's end are
// zero-filled by the copy and belong only to zones past the interior, which
// are skipped.
#pragma once

#include "kh_tma.cuh"
#include "kh_zone.cuh"

namespace kh {

template <int TX_, int TY_> struct UpdTile {
  static constexpr int TX = TX_, TY = TY_;  // zones per tile along x1, x2
  static constexpr int NT = TX * TY;        // threads per CTA
  static constexpr int PX = TX + 4;         // floats per staged row (the tile + alignment slack + the upper face)
  static constexpr int UX = TX + 2;         // doubles per staged row of U^n
  static constexpr int NFL = 5;             // fluid variables whose face fluxes are staged (the field's come from the EMFs)
  static constexpr int round128(int b) { return (b + 127) / 128 * 128; }
  // box bytes per staged array, and their shared-memory offsets (128-byte aligned)
  static constexpr int B_P = 4 * PX * TY * NV;
  static constexpr int B_F1 = 4 * PX * TY * NFL;
  static constexpr int B_F2 = 4 * PX * (TY + 1) * NFL;
  static constexpr int B_F3 = 4 * PX * TY * 2 * NFL;
  static constexpr int B_E1 = 4 * PX * (TY + 1) * 2;
  static constexpr int B_E2 = 4 * PX * TY * 2;
  static constexpr int B_E3 = 4 * PX * (TY + 1);
  static constexpr int B_U = 8 * UX * TY * NV;
  static constexpr int O_P = 0;
  static constexpr int O_F1 = O_P + round128(B_P);
  static constexpr int O_F2 = O_F1 + round128(B_F1);
  static constexpr int O_F3 = O_F2 + round128(B_F2);
  static constexpr int O_E1 = O_F3 + round128(B_F3);
  static constexpr int O_E2 = O_E1 + round128(B_E1);
  static constexpr int O_E3 = O_E2 + round128(B_E2);
  static constexpr int O_U = O_E3 + round128(B_E3);
  static constexpr int O_BAR = O_U + round128(B_U);
  static constexpr int SMEM = O_BAR + 128 + 128;  // + slack to align the dynamic base to 128 bytes
  static constexpr unsigned TX_BYTES = B_P + B_F1 + B_F2 + B_F3 + B_E1 + B_E2 + B_E3 + B_U;

  // The mixed update's inputs from the staged tiles (see MixedInGlobal): x is
  // the zone's column in the float tiles, xu in the FP64 tile, y its row.
  struct In {
    const unsigned char* s;
    int x, xu, y;
    __device__ __forceinline__ const float* fl(int o) const { return reinterpret_cast<const float*>(s + o); }
    __device__ __forceinline__ float pin(int v) const { return fl(O_P)[(v * TY + y) * PX + x]; }
    __device__ __forceinline__ double u0(int v) const {
      return reinterpret_cast<const double*>(s + O_U)[(v * TY + y) * UX + xu];
    }
    __device__ __forceinline__ float f(int d, int v, int up) const {
      if (d == 0) return fl(O_F1)[(v * TY + y) * PX + x + up];
      if (d == 1) return fl(O_F2)[(v * (TY + 1) + y + up) * PX + x];
      return fl(O_F3)[((v * 2 + up) * TY + y) * PX + x];
    }
    __device__ __forceinline__ float e(int a, int di, int dj, int dk) const {
      if (a == 0) return fl(O_E1)[(dk * (TY + 1) + y + dj) * PX + x + di];
      if (a == 1) return fl(O_E2)[(dk * TY + y + dj) * PX + x + di];
      return fl(O_E3)[(y + dj) * PX + x + di];
    }
    __device__ __forceinline__ bool has_emf() const { return true; }
  };
};

// The tensor maps of one update: P, the three flux arrays, the three EMF
// arrays (FP32) and U^n (FP64), each over one allocation [v][k][j][i].
struct UpdateMaps {
  CUtensorMap p, f1, f2, f3, e1, e2, e3, u;
};

// Host: the maps of a tile shape over arrays of extents (n1s, n2s, n3s) with
// plane = n1s n2s n3s cells per variable (U^n's map left as it is when U0 is
// null); encode_update_umap alone encodes the map of U^n. False if the encoder is unavailable or refuses a
// description (an unaligned base or stride).
template <class T> bool encode_update_umap(CUtensorMap* tm, const double* U0, int n1s, int n2s, int n3s) {
  const long long gplane = (long long)n1s * n2s, plane = gplane * n3s;
  const cuuint64_t d4[4] = {(cuuint64_t)n1s, (cuuint64_t)n2s, (cuuint64_t)n3s, (cuuint64_t)NV};
  const cuuint64_t s4d[3] = {(cuuint64_t)n1s * 8, (cuuint64_t)gplane * 8, (cuuint64_t)plane * 8};
  const cuuint32_t bU[4] = {(cuuint32_t)T::UX, (cuuint32_t)T::TY, 1, NV};
  return encode_tiled(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, U0, d4, s4d, bU);
}

template <class T>
bool encode_update_maps(UpdateMaps* tm, const float* P8, const double* U0, const float* const F[3],
                        const float* const emf[3], int n1s, int n2s, int n3s) {
  const long long gplane = (long long)n1s * n2s, plane = gplane * n3s;
  const cuuint64_t d4[4] = {(cuuint64_t)n1s, (cuuint64_t)n2s, (cuuint64_t)n3s, (cuuint64_t)NV};
  const cuuint64_t s4f[3] = {(cuuint64_t)n1s * 4, (cuuint64_t)gplane * 4, (cuuint64_t)plane * 4};
  const cuuint64_t s3f[2] = {(cuuint64_t)n1s * 4, (cuuint64_t)gplane * 4};
  const cuuint32_t PX = T::PX, TY = T::TY, NFL = T::NFL;
  const cuuint32_t bP[4] = {PX, TY, 1, NV}, bF1[4] = {PX, TY, 1, NFL}, bF2[4] = {PX, TY + 1, 1, NFL},
                   bF3[4] = {PX, TY, 2, NFL}, bE1[3] = {PX, TY + 1, 2}, bE2[3] = {PX, TY, 2}, bE3[3] = {PX, TY + 1, 1};
  const auto F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return encode_tiled(&tm->p, F32, 4, P8, d4, s4f, bP) && encode_tiled(&tm->f1, F32, 4, F[0], d4, s4f, bF1) &&
         encode_tiled(&tm->f2, F32, 4, F[1], d4, s4f, bF2) && encode_tiled(&tm->f3, F32, 4, F[2], d4, s4f, bF3) &&
         encode_tiled(&tm->e1, F32, 3, emf[0], d4, s3f, bE1) && encode_tiled(&tm->e2, F32, 3, emf[1], d4, s3f, bE2) &&
         encode_tiled(&tm->e3, F32, 3, emf[2], d4, s3f, bE3) && (!U0 || encode_update_umap<T>(&tm->u, U0, n1s, n2s, n3s));
}

#ifdef __CUDACC__
// Thread 0: the tile's eight tensor copies on bar (initialised, one arrival):
// float boxes from x1 cell x0, the FP64 box from xu0, rows from j0, plane k.
template <class T>
__device__ __forceinline__ void issue_update_tile(unsigned char* smem, const UpdateMaps& tm, int x0, int xu0, int j0,
                                                  int k, unsigned long long* bar) {
  mbar_expect_tx(bar, T::TX_BYTES);
  tma_load_4d(smem + T::O_P, &tm.p, x0, j0, k, 0, bar);
  tma_load_4d(smem + T::O_F1, &tm.f1, x0, j0, k, 0, bar);
  tma_load_4d(smem + T::O_F2, &tm.f2, x0, j0, k, 0, bar);
  tma_load_4d(smem + T::O_F3, &tm.f3, x0, j0, k, 0, bar);
  tma_load_3d(smem + T::O_E1, &tm.e1, x0, j0, k, bar);
  tma_load_3d(smem + T::O_E2, &tm.e2, x0, j0, k, bar);
  tma_load_3d(smem + T::O_E3, &tm.e3, x0, j0, k, bar);
  tma_load_4d(smem + T::O_U, &tm.u, xu0, j0, k, 0, bar);
}

// The CTA's 128-byte aligned base of the dynamic shared memory.
__device__ __forceinline__ unsigned char* aligned_smem(unsigned char* raw) {
  return raw + ((128u - (smem_u32(raw) & 127u)) & 127u);
}
#endif

}  // namespace kh
