// kh_divb_noalloc: a variant of the corner-divB reduction that allocates no
// memory at all. It exists for callers that cannot call cudaMalloc: code
// running inside a pre-sized memory pool or under a hard device-memory
// budget, host frameworks whose allocator forbids raw CUDA allocations, and
// embedding runtimes that hand the library only the arrays they already own.
// Such a caller cannot create a kh_ctx (which allocates its geometry cache and
// scratch), so this entry point takes everything it reads as arguments and
// keeps its only scratch -- one partial result per row of corners -- in a
// file-scope device array of fixed size.
//
// The scratch array is a static __device__ symbol: every GPU that loads this
// library holds it (2 * KH_DIVB_NOALLOC_MAX_ROWS doubles = 1 MiB) until the
// process exits. Its host-side name is only a stand-in for the symbol, so the
// host looks up the device address once per device with cudaGetSymbolAddress
// and passes that pointer to the kernels.
#include <mutex>

#include "kh_internal.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kRowThreads = 128;

static __device__ __align__(256) double kh_divb_noalloc_scratch[2 * KH_DIVB_NOALLOC_MAX_ROWS];

std::mutex g_scratch_lock;
double* g_scratch[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up on the
// first call per device, with that device current, and cached for the life of
// the process: a cudaDeviceReset makes the cached address stale).
int scratch_on_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KH_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return KH_EINVAL;
  std::lock_guard<std::mutex> guard(g_scratch_lock);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, kh_divb_noalloc_scratch) != cudaSuccess || !p) return KH_ECUDA;
    g_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_scratch[dev];
  return KH_OK;
}

struct NoAllocGrid {
  int n1, n2, n3, ndim, ng, ng3, n1s, n2s;
  double dx[3];
  __device__ long long at(int k, int j, int i) const { return ((long long)k * n2s + j) * n1s + i; }
};

__device__ __forceinline__ void row_max_sum(double& a, double& b) {
  __shared__ double sa[kRowThreads / 32], sb[kRowThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = (l < kRowThreads / 32) ? sa[l] : 0.0;
    b = (l < kRowThreads / 32) ? sb[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
  }
}

// One block per row of interior corners (fixed j, k); threads stride along i.
// Writes the row's max |divB| and sum |divB| to scratch[2 row], scratch[2 row + 1].
__global__ void __launch_bounds__(kRowThreads) k_divb_rows(const double* B, const double* gdet, NoAllocGrid g,
                                                          long long plane, double* scratch) {
  const int row = blockIdx.x;
  const int nj = g.n2 - 1;
  const int j = g.ng + 1 + row % nj;
  const int k = g.ndim == 3 ? g.ng3 + 1 + row / nj : 0;
  const double* B1 = B;
  const double* B2 = B + plane;
  const double* B3 = B + 2 * plane;
  auto gB = [&](const double* Bd, int kk, int jj, int ii) { return gdet[(long long)jj * g.n1s + ii] * Bd[g.at(kk, jj, ii)]; };
  double mx = 0.0, sm = 0.0;
  for (int i = g.ng + 1 + threadIdx.x; i <= g.ng + g.n1 - 1; i += blockDim.x) {
    double dv;
    if (g.ndim == 2) {
      dv = (gB(B1, k, j, i) + gB(B1, k, j - 1, i) - gB(B1, k, j, i - 1) - gB(B1, k, j - 1, i - 1)) / (2.0 * g.dx[0]) +
           (gB(B2, k, j, i) + gB(B2, k, j, i - 1) - gB(B2, k, j - 1, i) - gB(B2, k, j - 1, i - 1)) / (2.0 * g.dx[1]);
    } else {
      const double p1 = gB(B1, k, j, i) + gB(B1, k, j - 1, i) + gB(B1, k - 1, j, i) + gB(B1, k - 1, j - 1, i);
      const double m1 = gB(B1, k, j, i - 1) + gB(B1, k, j - 1, i - 1) + gB(B1, k - 1, j, i - 1) + gB(B1, k - 1, j - 1, i - 1);
      const double p2 = gB(B2, k, j, i) + gB(B2, k, j, i - 1) + gB(B2, k - 1, j, i) + gB(B2, k - 1, j, i - 1);
      const double m2 = gB(B2, k, j - 1, i) + gB(B2, k, j - 1, i - 1) + gB(B2, k - 1, j - 1, i) + gB(B2, k - 1, j - 1, i - 1);
      const double p3 = gB(B3, k, j, i) + gB(B3, k, j, i - 1) + gB(B3, k, j - 1, i) + gB(B3, k, j - 1, i - 1);
      const double m3 = gB(B3, k - 1, j, i) + gB(B3, k - 1, j, i - 1) + gB(B3, k - 1, j - 1, i) + gB(B3, k - 1, j - 1, i - 1);
      dv = (p1 - m1) / (4.0 * g.dx[0]) + (p2 - m2) / (4.0 * g.dx[1]) + (p3 - m3) / (4.0 * g.dx[2]);
    }
    mx = fmax(mx, fabs(dv));
    sm += fabs(dv);
  }
  row_max_sum(mx, sm);
  if (threadIdx.x == 0) {
    scratch[2 * row] = mx;
    scratch[2 * row + 1] = sm;
  }
}

// Single block: combine the nrows row results into out[0] = max, out[1] = mean.
__global__ void __launch_bounds__(kRowThreads) k_divb_rows_final(const double* scratch, int nrows, double ncorners,
                                                                double* out) {
  double mx = 0.0, sm = 0.0;
  for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
    mx = fmax(mx, scratch[2 * r]);
    sm += scratch[2 * r + 1];
  }
  row_max_sum(mx, sm);
  if (threadIdx.x == 0) {
    out[0] = mx;
    out[1] = sm / ncorners;
  }
}

// True when p is device memory of the device dev (or managed memory).
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // an unregistered host pointer: clear the lookup's error
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" int kh_divb_noalloc(const double* B, const double* gdet, int n1, int n2, int n3, int n1s, int n2s,
                               double dx1, double dx2, double dx3, double* out, void* cuda_stream) {
  if (!B || !gdet || !out) return KH_EINVAL;
  // an error left by an earlier, unrelated call is not this call's: report it
  // without clearing it, so that the caller still sees the original error
  if (cudaPeekAtLastError() != cudaSuccess) return KH_ECUDA;
  if (n1 < 2 || n2 < 2 || n3 < 1) return KH_EINVAL;
  if (n1s < n1 + 2 * kh::NGHOST || n2s < n2 + 2 * kh::NGHOST) return KH_EINVAL;
  if (!(dx1 > 0.0) || !(dx2 > 0.0) || (n3 > 1 && !(dx3 > 0.0))) return KH_EINVAL;
  const long long nrows = (long long)(n2 - 1) * (n3 > 1 ? (n3 - 1) : 1);
  if (nrows > KH_DIVB_NOALLOC_MAX_ROWS) return KH_EINVAL;  // larger than the static scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KH_ECUDA;
  // the scratch address is the current device's: the arrays must live there
  if (!on_device(B, dev) || !on_device(gdet, dev) || !on_device(out, dev)) return KH_EINVAL;
  double* scratch = nullptr;
  const int rc = scratch_on_current_device(&scratch);
  if (rc != KH_OK) return rc;
  NoAllocGrid g;
  g.n1 = n1;
  g.n2 = n2;
  g.n3 = n3;
  g.ndim = n3 > 1 ? 3 : 2;
  g.ng = kh::NGHOST;
  g.ng3 = g.ndim == 3 ? kh::NGHOST : 0;
  g.n1s = n1s;
  g.n2s = n2s;
  g.dx[0] = dx1;
  g.dx[1] = dx2;
  g.dx[2] = dx3;
  const long long n3s = n3 + 2LL * g.ng3;
  const long long plane = (long long)n1s * n2s * n3s;
  const double ncorners = (double)(n1 - 1) * nrows;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  k_divb_rows<<<(unsigned)nrows, kRowThreads, 0, s>>>(B, gdet, g, plane, scratch);
  k_divb_rows_final<<<1, kRowThreads, 0, s>>>(scratch, (int)nrows, ncorners, out);
  return cudaGetLastError() == cudaSuccess ? KH_OK : KH_ECUDA;
}
