// The mixed path's update with its inputs staged in shared memory by TMA.
//
// The update of a zone reads the stage input P (8 FP32), U^n (8 FP64), the
// fluid variables' face fluxes in three directions (both faces of the zone)
// and Flux-CT's edge EMFs around it -- ~60 values from six arrays, the
// fluxes and EMFs just written by the face and EMF kernels and mostly no
// longer in L2. Read by the threads themselves, those loads hold the
// registers of a kernel whose arithmetic (the double-float inversion) wants
// ~220 of them, and their DRAM latency is exposed at the ~35% occupancy the
// register budget leaves. Here one CTA updates a tile of 32 (x1) x 4 (x2)
// zones of one x3 plane: thread 0 issues eight tensor copies (kh_update_tile.cuh)
// on one mbarrier, the copy engine moves them while the SM runs other CTAs,
// and every thread then runs the same per-zone update (update_mixed_zone_in)
// reading its values from the tiles. Seven 128-thread CTAs per SM (72
// registers, 29 KB of tiles each): 2% faster than three 256-thread CTAs at 80
// registers; 32 x 8, 32 x 2 and 32 x 1 x 8 tiles (the last sharing the
// geometry columns of a CTA's warps through L1) measured within 3% of these.
#include "kh_update_tile.cuh"

namespace kh {
namespace {

using Tile = UpdTile<32, 4>;

template <int INV>
__global__ void __launch_bounds__(Tile::NT, 7)
    k_update_mixed_tma(const __grid_constant__ UpdateMaps tm, Vars Pout64, VarsT<float> Pout32, double* Uout,
                       Layout L, DevGeom G, GeomT<float> Gf, Scheme S, const double* dtp, double coef, int8_t* pflag,
                       unsigned long long* cnt, FailList fl, double* dUout, unsigned wlim) {
  pdl_wait();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = aligned_smem(smem_raw);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + Tile::O_BAR);
  const int lx = threadIdx.x & (Tile::TX - 1), ly = threadIdx.x / Tile::TX;
  const int i0 = L.s[0] + Tile::TX * (int)blockIdx.x, j0 = L.s[1] + Tile::TY * (int)blockIdx.y;
  const int k = L.s[2] + (int)blockIdx.z;
  const int x0 = i0 & ~3, xu0 = i0 & ~1;  // 16-byte boundaries at or below i0
  if (threadIdx.x == 0) mbar_init(bar);
  __syncthreads();
  if (threadIdx.x == 0) issue_update_tile<Tile>(smem, tm, x0, xu0, j0, k, bar);
  if (!cta_wait_tiles(bar, wlim, cnt)) return;
  const int i = i0 + lx, j = j0 + ly;
  if (i >= L.e[0] || j >= L.e[1]) return;  // ragged tile
  if (KH_OOB(L, kh_in(L, i, j, k, 1))) return;
  const Tile::In in{smem, (i0 - x0) + lx, (i0 - xu0) + lx, ly};
  update_mixed_zone_in<false, INV, Tile::In, true>(in, Pout64, Pout32, Uout, L, G, Gf, S,
                                                   df_of_f64(coef * __ldg(dtp)), pflag, cnt, i, j, k, fl, nullptr,
                                                   dUout);
}

template <int INV> bool set_smem_once() {
  static bool done = false;
  if (!done)
    done = cudaFuncSetAttribute(k_update_mixed_tma<INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, Tile::SMEM) ==
           cudaSuccess;
  return done;
}

}  // namespace

int launch_update_mixed_tma(const double* U0, const float* P8, const Vars& Pout64, const VarsT<float>& Pout32,
                            double* Uout, float* const F[3], float* const emf[3], const Layout& L, const DevGeom& G,
                            const GeomT<float>& Gf, const Scheme& S, const double* dtp, double coef, int8_t* pflag,
                            unsigned long long* cnt, FailList fl, double* dUout, unsigned wlim, cudaStream_t s) {
  if (L.ndim != 3 || !P8 || !U0 || !F[0] || !F[1] || !F[2] || !emf[0] || !emf[1] || !emf[2]) return -1;
  UpdateMaps tm;
  const float* const Fc[3] = {F[0], F[1], F[2]};
  const float* const Ec[3] = {emf[0], emf[1], emf[2]};
  if (!encode_update_maps<Tile>(&tm, P8, U0, Fc, Ec, L.n1s, L.n2s, L.n3s)) return -1;
  const dim3 grid((L.n1 + Tile::TX - 1) / Tile::TX, (L.n2 + Tile::TY - 1) / Tile::TY, L.n3);
  auto go = [&](auto kern, bool ok) {
    if (!ok) return false;
    launch_pdl(kern, grid, dim3(Tile::NT), Tile::SMEM, s, tm, Pout64, Pout32, Uout, L, G, Gf, S, dtp, coef, pflag, cnt,
               fl, dUout, wlim);
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
