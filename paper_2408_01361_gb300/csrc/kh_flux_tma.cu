// FP32 face fluxes of the mixed path from TMA-staged shared-memory tiles.
//
// One CTA of 256 threads (one per reconstructed cell) computes the LLF fluxes
// of a tile of x^D faces: 31 x 8 faces for x1 (32 cells along x1 per row), 32
// x 7 for x2 and x3 (8 cell rows along the direction). Its 8 primitive planes
// arrive in shared memory by one 4-D tensor
// copy (cp.async.bulk.tensor, completion on an mbarrier): the faces' cells
// plus the 3-cell stencil halo along D. Each cell of the tile is then
// reconstructed ONCE for both of its x^D faces (MC: one slope; WENO5: the
// three smoothness indicators and their weight ratios shared by the upper and
// lower face values), the face states go to shared memory, and each thread
// evaluates the fluid states, fluxes, signal speeds and LLF of its face.
// Tiles are aligned so that the innermost tensor coordinate is a multiple of
// 4 floats (16 bytes); reads past the array edge are zero-filled by the copy
// and only feed faces outside the face box, which are skipped.
#include "kh_pair.cuh"
#include "kh_tma.cuh"
#include "kh_zone.cuh"

namespace kh {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool encode_tiled(CUtensorMap* tm, CUtensorMapDataType type, int rank, const void* base, const cuuint64_t* dims,
                  const cuuint64_t* strides, const cuuint32_t* box) {
  auto fn = tensor_map_encoder();
  if (!fn) return false;
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return fn(tm, type, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

constexpr int NT = 256;    // threads = cells reconstructed per tile
constexpr int CW = 32;     // cells per tile row along x1

// Both face values of one cell from its 5-point stencil (a, b, c, d, e):
// hi at x = +1/2 (as weno5_plus(a, b, c, d, e)), lo at x = -1/2 (as
// weno5_plus(e, d, c, b, a)); the smoothness indicators, their scale-free
// normalisation and the weight ratios are those of weno5_plus, computed once.
__device__ __forceinline__ void weno5_lohi(float a, float b, float c, float d, float e, float& lo, float& hi) {
  const float k = 13.0f / 12.0f;
  const float t0 = a - 2.0f * b + c, u0 = a - 4.0f * b + 3.0f * c;
  const float t1 = b - 2.0f * c + d, u1 = b - d;
  const float t2 = c - 2.0f * d + e, u2 = 3.0f * c - 4.0f * d + e;
  const float b0 = k * t0 * t0 + 0.25f * u0 * u0;
  const float b1 = k * t1 * t1 + 0.25f * u1 * u1;
  const float b2 = k * t2 * t2 + 0.25f * u2 * u2;
  const float in = __frcp_rn(b0 + b1 + b2 + 1e-37f);
  const float s0 = b0 * in + 1e-12f, s1 = b1 * in + 1e-12f, s2 = b2 * in + 1e-12f;
  const float sm = fminf(s0, fminf(s1, s2));
  const float r0 = __fdividef(sm, s0), r1 = __fdividef(sm, s1), r2 = __fdividef(sm, s2);
  const float q0 = r0 * r0, q1 = r1 * r1, q2 = r2 * r2;
  {  // upper face: stencils (a b c), (b c d), (c d e), linear weights 1/16, 5/8, 5/16
    const float p0 = 0.375f * a - 1.25f * b + 1.875f * c;
    const float p1 = -0.125f * b + 0.75f * c + 0.375f * d;
    const float p2 = 0.375f * c + 0.75f * d - 0.125f * e;
    const float w0 = 0.0625f * q0, w1 = 0.625f * q1, w2 = 0.3125f * q2;
    hi = __fdividef(w0 * p0 + w1 * p1 + w2 * p2, w0 + w1 + w2);
  }
  {  // lower face: the mirrored stencils, the indicators' roles swapped (0 <-> 2)
    const float p0 = 0.375f * e - 1.25f * d + 1.875f * c;
    const float p1 = -0.125f * d + 0.75f * c + 0.375f * b;
    const float p2 = 0.375f * c + 0.75f * b - 0.125f * a;
    const float w0 = 0.0625f * q2, w1 = 0.625f * q1, w2 = 0.3125f * q0;
    lo = __fdividef(w0 * p0 + w1 * p1 + w2 * p2, w0 + w1 + w2);
  }
}

// The same for two variables at once (paired FP32 instructions).
__device__ __forceinline__ void weno5_lohi(P2 a, P2 b, P2 c, P2 d, P2 e, P2& lo, P2& hi) {
  const P2 k(13.0f / 12.0f), q4(0.25f);
  const P2 t0 = P2(-2.0f) * b + (a + c), u0 = P2(3.0f) * c + (a - P2(4.0f) * b);
  const P2 t1 = P2(-2.0f) * c + (b + d), u1 = b - d;
  const P2 t2 = P2(-2.0f) * d + (c + e), u2 = P2(3.0f) * c + (e - P2(4.0f) * d);
  const P2 b0 = (k * t0) * t0 + (q4 * u0) * u0;
  const P2 b1 = (k * t1) * t1 + (q4 * u1) * u1;
  const P2 b2 = (k * t2) * t2 + (q4 * u2) * u2;
  const P2 sum = b0 + b1 + b2 + 1e-37f;
  const P2 in(__frcp_rn(sum.v.x), __frcp_rn(sum.v.y));
  const P2 eps(1e-12f);
  const P2 s0 = b0 * in + eps, s1 = b1 * in + eps, s2 = b2 * in + eps;
  const P2 sm(fminf(s0.v.x, fminf(s1.v.x, s2.v.x)), fminf(s0.v.y, fminf(s1.v.y, s2.v.y)));
  const P2 r0 = kdiv(sm, s0), r1 = kdiv(sm, s1), r2 = kdiv(sm, s2);
  const P2 q0 = r0 * r0, q1 = r1 * r1, q2 = r2 * r2;
  {  // upper face
    const P2 p0 = P2(0.375f) * a + (P2(-1.25f) * b + P2(1.875f) * c);
    const P2 p1 = P2(-0.125f) * b + (P2(0.75f) * c + P2(0.375f) * d);
    const P2 p2 = P2(0.375f) * c + (P2(0.75f) * d + P2(-0.125f) * e);
    const P2 w0 = P2(0.0625f) * q0, w1 = P2(0.625f) * q1, w2 = P2(0.3125f) * q2;
    hi = kdiv(w0 * p0 + (w1 * p1 + w2 * p2), w0 + w1 + w2);
  }
  {  // lower face: mirrored stencils, indicators' roles swapped
    const P2 p0 = P2(0.375f) * e + (P2(-1.25f) * d + P2(1.875f) * c);
    const P2 p1 = P2(-0.125f) * d + (P2(0.75f) * c + P2(0.375f) * b);
    const P2 p2 = P2(0.375f) * c + (P2(0.75f) * b + P2(-0.125f) * a);
    const P2 w0 = P2(0.0625f) * q2, w1 = P2(0.625f) * q1, w2 = P2(0.3125f) * q0;
    lo = kdiv(w0 * p0 + (w1 * p1 + w2 * p2), w0 + w1 + w2);
  }
}

template <int D> struct TileShape {
  static constexpr int FX = D == 1 ? CW - 1 : CW;  // faces per tile along x1
  static constexpr int FY = D == 1 ? 8 : 7;        // faces per tile along the second tile direction
  // tensor box: x (with the x1 halo and alignment slack when D = 1), y, z, 8 slots
  static constexpr int BX = D == 1 ? CW + 8 : CW;
  static constexpr int BY = D == 1 ? 8 : (D == 2 ? 12 : 1);
  static constexpr int BZ = D == 3 ? 12 : 1;
};

template <int D, int RECON>
__global__ void __launch_bounds__(NT) k_flux_tma(const __grid_constant__ CUtensorMap tm, Layout L, GeomT<float> G,
                                                 Scheme S, FaceBox box, float* F, float* ctop, int polar_lo,
                                                 int polar_hi, unsigned long long* cnt, unsigned wlim) {
  pdl_wait();
  using Sh = TileShape<D>;
  __shared__ alignas(128) float tile[NV * Sh::BZ * Sh::BY * Sh::BX];
  __shared__ float sL[NV][NT], sR[NV][NT];
  __shared__ alignas(8) unsigned long long bar;
  const int tid = threadIdx.x;
  const int lx = tid % CW, ly = tid / CW;
  // tile origin (cell coordinates) and the tensor coordinates of the box; for
  // x1 the box starts at the 16-byte boundary at or below the stencil's first
  // cell, dx cells earlier
  int i, j, k, c0, c1, c2, dx = 0;
  if (D == 1) {
    const int f0 = L.s[0] + Sh::FX * blockIdx.x;  // first face of the tile
    const int j0 = (L.s[1] - 1) + Sh::FY * blockIdx.y;
    k = L.ndim == 3 ? (L.s[2] - 1) + (int)blockIdx.z : 0;
    c0 = (f0 - 3) & ~3;
    dx = (f0 - 3) - c0;
    i = f0 + lx;
    j = j0 + ly;
    c1 = j0, c2 = k;
  } else if (D == 2) {
    const int x0 = CW * blockIdx.x;
    const int j0 = L.s[1] + Sh::FY * blockIdx.y;
    k = L.ndim == 3 ? (L.s[2] - 1) + (int)blockIdx.z : 0;
    i = x0 + lx;
    j = j0 + ly;
    c0 = x0, c1 = j0 - 3, c2 = k;
  } else {
    const int x0 = CW * blockIdx.x;
    const int k0 = L.s[2] + Sh::FY * blockIdx.y;
    j = (L.s[1] - 1) + (int)blockIdx.z;
    i = x0 + lx;
    k = k0 + ly;
    c0 = x0, c1 = j, c2 = k0 - 3;
  }
  if (tid == 0) mbar_init(&bar);
  __syncthreads();
  if (tid == 0) {
    mbar_expect_tx(&bar, sizeof(float) * NV * Sh::BZ * Sh::BY * Sh::BX);
    tma_load_4d(tile, &tm, c0, c1, c2, 0, &bar);
  }
  // bounded wait; on a timeout the CTA leaves (after its copy has landed)
  // without writing its faces
  if (!cta_wait_tiles(&bar, wlim, cnt)) return;
  // ---- reconstruct this thread's cell once, for both of its x^D faces ----
  // cell cl along D (0 = the cell below the tile's first face), row across
  auto at = [&](int v, int x, int y, int z) { return tile[((v * Sh::BZ + z) * Sh::BY + y) * Sh::BX + x]; };
  {
    const int cl = D == 1 ? lx : ly, row = D == 1 ? ly : lx;
    // stencil of the cell: D = 1 at box x dx + cl .. dx + cl + 4 (the box
    // holds the tile's cells from f0 - 3 on); D = 2, 3 at cl .. cl + 4 along
    // the direction (the box starts 3 below the first face)
    auto sten = [&](int v, int o) {
      if (D == 1) return at(v, dx + cl + o, row, 0);
      else if (D == 2) return at(v, row, cl + o, 0);
      else return at(v, row, 0, cl + o);
    };
    // hi is the left state of the face above the cell, lo the right state of the face at its bottom
    auto put = [&](int v, float lo, float hi) {
      if (D == 1) {
        if (cl < Sh::FX) sL[v][row * CW + cl] = hi;
        if (cl >= 1) sR[v][row * CW + cl - 1] = lo;
      } else {
        if (cl < Sh::FY) sL[v][cl * CW + row] = hi;
        if (cl >= 1) sR[v][(cl - 1) * CW + row] = lo;
      }
    };
    if (RECON == KH_RECON_MC) {
      for (int v = 0; v < NV; ++v) {
        float lo, hi;
        recon_mc(sten(v, 1), sten(v, 2), sten(v, 3), lo, hi);
        put(v, lo, hi);
      }
    } else {
      for (int v = 0; v < NV; v += 2) {  // two variables per pass
        P2 q[5];
#pragma unroll
        for (int o = 0; o < 5; ++o) q[o] = P2(sten(v, o), sten(v + 1, o));
        P2 lo, hi;
        weno5_lohi(q[0], q[1], q[2], q[3], q[4], lo, hi);
        put(v, lo.v.x, hi.v.x);
        put(v + 1, lo.v.y, hi.v.y);
      }
    }
  }
  __syncthreads();
  if ((D == 1 && lx >= Sh::FX) || (D != 1 && ly >= Sh::FY)) return;  // cells without a face of their own
  // ---- the LLF flux of this thread's face ----
  const bool in_box = i >= box.lo[0] && i < box.lo[0] + box.n[0] && j >= box.lo[1] && j < box.lo[1] + box.n[1] &&
                      k >= box.lo[2] && k < box.lo[2] + box.n[2];
  if (!in_box) return;
  if (KH_OOB(L, kh_in(L, i, j, k, 0))) return;
  float PL[NV], PR[NV];
  const int slot = ly * CW + lx;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    PL[v] = sL[v][slot];
    PR[v] = sR[v][slot];
  }
  const long long c = L.at(k, j, i);
  const Met<float> m = load_met(G, L.gplane, D == 3 ? LOC_CENT : D, (long long)j * L.n1s + i);
  // both states at once: (left, right) pairs through paired FP32 instructions
  const P2 gam((float)S.mx.gam);
  P2 Pp[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Pp[v] = P2(PL[v], PR[v]);
  FState<P2> st;
  fluid_state(Pp, m, st);
  P2 Fp[NV], Up[NV];
  flux_cons(Pp, st, m, gam, D, Fp, Up);
  P2 cmax, cmin;
  signal_speeds(Pp, st, m, gam, D, cmax, cmin);
  const float cm = fmaxf(0.0f, fmaxf(cmax.v.x, cmax.v.y));
  const float cn = fmaxf(0.0f, fmaxf(-cmin.v.x, -cmin.v.y));
  const float ct = fmaxf(cm, cn);
  const bool axis = (D == 2) && ((polar_lo && j == L.s[1]) || (polar_hi && j == L.e[1]));
#pragma unroll
  for (int v = 0; v < NV; ++v)
    F[v * L.plane + c] = axis ? 0.0f : 0.5f * (Fp[v].v.x + Fp[v].v.y) - 0.5f * ct * (Up[v].v.y - Up[v].v.x);
  ctop[c] = ct;
}

// The 8 FP32 planes [v][k][j][i] as a 4-D tensor (i, j, k, v) with the box of
// direction D.
template <int D> bool encode(CUtensorMap* tm, const float* base, const Layout& L) {
  using Sh = TileShape<D>;
  const cuuint64_t dims[4] = {(cuuint64_t)L.n1s, (cuuint64_t)L.n2s, (cuuint64_t)L.n3s, (cuuint64_t)NV};
  const cuuint64_t strides[3] = {(cuuint64_t)L.n1s * 4, (cuuint64_t)L.n1s * L.n2s * 4, (cuuint64_t)L.plane * 4};
  const cuuint32_t boxd[4] = {(cuuint32_t)Sh::BX, (cuuint32_t)Sh::BY, (cuuint32_t)Sh::BZ, (cuuint32_t)NV};
  return encode_tiled(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, boxd);
}

template <int D>
int launch_d(const float* P8, const Layout& L, const GeomT<float>& G, const Scheme& S, float* F, float* ctop,
             unsigned long long* cnt, unsigned wlim, cudaStream_t s) {
  alignas(64) CUtensorMap tm;
  if (!encode<D>(&tm, P8, L)) return -1;
  const FaceBox b = face_box(L, D);
  const int plo = S.bc[2] == KH_BC_POLAR, phi = S.bc[3] == KH_BC_POLAR;
  using Sh = TileShape<D>;
  dim3 grid;
  if (D == 1)
    grid = dim3((L.n1 + 1 + Sh::FX - 1) / Sh::FX, (L.n2 + 2 + Sh::FY - 1) / Sh::FY, L.ndim == 3 ? L.n3 + 2 : 1);
  else if (D == 2)
    grid = dim3((L.e[0] + 1 + CW - 1) / CW, (L.n2 + 1 + Sh::FY - 1) / Sh::FY, L.ndim == 3 ? L.n3 + 2 : 1);
  else
    grid = dim3((L.e[0] + 1 + CW - 1) / CW, (L.n3 + 1 + Sh::FY - 1) / Sh::FY, L.n2 + 2);
  if (S.recon == KH_RECON_MC)
    launch_pdl(k_flux_tma<D, KH_RECON_MC>, grid, dim3(NT), 0, s, tm, L, G, S, b, F, ctop, plo, phi, cnt, wlim);
  else
    launch_pdl(k_flux_tma<D, KH_RECON_WENO5>, grid, dim3(NT), 0, s, tm, L, G, S, b, F, ctop, plo, phi, cnt, wlim);
  return 1;
}

}  // namespace

int launch_flux_dir_tma(int D, const float* P8, const Layout& L, const GeomT<float>& G, const Scheme& S, float* F,
                        float* ctop, unsigned long long* cnt, unsigned wlim, cudaStream_t s) {
  if (D == 1) return launch_d<1>(P8, L, G, S, F, ctop, cnt, wlim, s);
  if (D == 2) return launch_d<2>(P8, L, G, S, F, ctop, cnt, wlim, s);
  return launch_d<3>(P8, L, G, S, F, ctop, cnt, wlim, s);
}

}  // namespace kh
