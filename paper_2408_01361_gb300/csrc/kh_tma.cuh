// TMA (cp.async.bulk.tensor) staging shared by the mixed path's face and
// update kernels: tensor-map encoding on the host, mbarrier completion and the
// bounded wait on the device.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "kh_internal.h"

namespace kh {

#ifdef __CUDACC__
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// One arrival expected (the issuing thread's), made visible to the async proxy.
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// Makes a tensor map in global memory, written through the generic proxy (a
// host-to-device copy), visible to the tensor copies that read it.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* tm) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<unsigned long long>(tm))
               : "memory");
}

// Thread 0 of a CTA waits for the phase of parity `phase` of bar (its staged
// tiles) with at most wlim polls. On a timeout it counts it (CNT_TIMEOUT) and
// keeps polling -- up to KH_WAIT_POLLS more times -- until the copies it
// issued have landed: the one on bar and, if `other` is given, the one on
// other (phase other_phase), so that none outlives the CTA's shared memory
// (a drain that also runs out is counted as CNT_DRAIN). Returns, to every
// thread of the CTA, whether the tiles arrived in time; all threads then
// observe the completed phase.
__device__ __forceinline__ bool cta_wait_tiles2(unsigned long long* bar, unsigned phase, unsigned wlim,
                                                unsigned long long* cnt, unsigned long long* other,
                                                unsigned other_phase) {
  __shared__ int ready;
  if (threadIdx.x == 0) {
    bool ok = false;
    for (unsigned spins = 0; spins < wlim && !ok; ++spins) ok = mbar_try_wait(bar, phase);
    if (!ok) {
      atomicAdd(cnt + CNT_TIMEOUT, 1ULL);
      bool landed = false;
      for (unsigned r = 0; r < KH_WAIT_POLLS && !landed; ++r) landed = mbar_try_wait(bar, phase);
      if (other) {
        bool landed2 = false;
        for (unsigned r = 0; r < KH_WAIT_POLLS && !landed2; ++r) landed2 = mbar_try_wait(other, other_phase);
        landed = landed && landed2;
      }
      if (!landed) atomicAdd(cnt + CNT_DRAIN, 1ULL);
    }
    ready = ok ? 1 : 0;
  }
  __syncthreads();
  if (!ready) return false;
  for (unsigned r = 0; r < KH_WAIT_POLLS && !mbar_try_wait(bar, phase); ++r) {  // completed: returns at once
  }
  return true;
}

// The same for a CTA with one copy in flight, on the first phase of bar.
__device__ __forceinline__ bool cta_wait_tiles(unsigned long long* bar, unsigned wlim, unsigned long long* cnt) {
  return cta_wait_tiles2(bar, 0, wlim, cnt, nullptr, 0);
}
#endif

// Host: the driver's cuTensorMapEncodeTiled (null if unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// Host: a tiled tensor map of `rank` dims (innermost first) over base, with
// byte strides of dims 1.. and the box extents; no swizzle, zero fill out of
// bounds. False if the encoder is unavailable or refuses the description.
bool encode_tiled(CUtensorMap* tm, CUtensorMapDataType type, int rank, const void* base, const cuuint64_t* dims,
                  const cuuint64_t* strides, const cuuint32_t* box);

}  // namespace kh
