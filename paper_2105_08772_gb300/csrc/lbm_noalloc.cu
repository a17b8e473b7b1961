// Mass and centre of mass of a device density field, computed without
// allocating any device memory (lbm_density_moments_noalloc in include/lbm.h).
//
// The reduction is the mass / centre-of-mass part of the field-observable
// pass, applied to a plain density field the caller owns.  Its per-CTA
// partial sums live in a file-scope __device__ array instead of a workspace,
// so the entry point needs no allocation from its caller or from itself.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm.h"

namespace lbm {
void set_global_error(const char* msg);
}

namespace {

constexpr int kNoallocCtas = 4096;          // partial records the scratch holds
constexpr int kNoallocNodesPerCta = 8192;   // nodes one CTA reduces
constexpr int kNoallocRecord = 5;           // mass, sum w, sum w dx, sum w dy, sum w dz
constexpr int kNoallocThreads = 256;
constexpr long long kNoallocMaxNodes = (long long)kNoallocCtas * kNoallocNodesPerCta;

// 4096 x 5 doubles = 160 KiB per device, resident until the process exits
static __device__ __align__(256) double g_noalloc_scratch[kNoallocCtas * kNoallocRecord];

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kNoallocThreads / 32; ++k) s += red[k];
  return s;
}

// minimum-image displacement of coordinate x from the centre node n/2, in
// [-n/2, n/2); the plane at exactly n/2 (even n) is both images and counts 0
__device__ __forceinline__ int centred(int x, int n) {
  int d = x - n / 2;
  if (2 * d == -n) d = 0;
  return d;
}

__global__ void __launch_bounds__(kNoallocThreads)
noalloc_partials(const double* __restrict__ rho, int nx, int ny, int nz, double n_ref,
                 double* __restrict__ scratch) {
  __shared__ double red[kNoallocThreads / 32];
  const long long N = (long long)nx * ny * nz;
  const long long begin = (long long)blockIdx.x * kNoallocNodesPerCta;
  const long long end = begin + kNoallocNodesPerCta < N ? begin + kNoallocNodesPerCta : N;
  double s[kNoallocRecord] = {0, 0, 0, 0, 0};
  for (long long node = begin + threadIdx.x; node < end; node += kNoallocThreads) {
    const int x = (int)(node % nx);
    const long long r = node / nx;
    const int y = (int)(r % ny), z = (int)(r / ny);
    const double n = rho[node];
    const double w = n - n_ref;
    s[0] += n;
    s[1] += w;
    s[2] += w * centred(x, nx);
    s[3] += w * centred(y, ny);
    s[4] += w * centred(z, nz);
  }
  for (int k = 0; k < kNoallocRecord; ++k) {
    const double t = block_sum(s[k], red);
    if (threadIdx.x == 0) scratch[blockIdx.x * kNoallocRecord + k] = t;
  }
}

__global__ void __launch_bounds__(kNoallocThreads)
noalloc_finalize(const double* __restrict__ scratch, int nblocks, int nx, int ny, int nz,
                 double* __restrict__ out) {
  __shared__ double red[kNoallocThreads / 32];
  double s[kNoallocRecord] = {0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += kNoallocThreads)
    for (int k = 0; k < kNoallocRecord; ++k) s[k] += scratch[b * kNoallocRecord + k];
  double t[kNoallocRecord];
  for (int k = 0; k < kNoallocRecord; ++k) t[k] = block_sum(s[k], red);
  if (threadIdx.x == 0) {
    // a field with no excess over n_ref (uniform at n_ref, or excess that
    // cancels exactly) has no centre of mass: NaN, not a division by zero
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    out[0] = t[0];
    out[1] = t[1] != 0.0 ? (double)(nx / 2) + t[2] / t[1] : nan;
    out[2] = t[1] != 0.0 ? (double)(ny / 2) + t[3] / t[1] : nan;
    out[3] = t[1] != 0.0 ? (double)(nz / 2) + t[4] / t[1] : nan;
  }
}

// device address of the scratch array, looked up once per device with that
// device current (the host-side symbol is only a stand-in, not an address)
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_density_moments_noalloc(const double* dev_rho, int nx, int ny, int nz,
                                                  double n_ref, double* dev_out, void* cuda_stream) {
  // sizes first, then pointers: a null pointer at an accepted size reports the
  // pointer, so the size limit can be checked without a device
  if (nx < 1 || ny < 1 || nz < 1) {
    lbm::set_global_error("lbm_density_moments_noalloc: box sides must be >= 1");
    return LBM_EINVAL;
  }
  const long long N = (long long)nx * ny * nz;
  if (N > kNoallocMaxNodes) {
    lbm::set_global_error(
        "lbm_density_moments_noalloc: field has more than 33554432 nodes (the fixed scratch "
        "holds 4096 partial sums of 8192 nodes each)");
    return LBM_EINVAL;
  }
  if (!dev_rho || !dev_out) {
    lbm::set_global_error("lbm_density_moments_noalloc: null device pointer");
    return LBM_EINVAL;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    lbm::set_global_error(cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int nblocks = (int)((N + kNoallocNodesPerCta - 1) / kNoallocNodesPerCta);
  noalloc_partials<<<nblocks, kNoallocThreads, 0, s>>>(dev_rho, nx, ny, nz, n_ref, scratch);
  noalloc_finalize<<<1, kNoallocThreads, 0, s>>>(scratch, nblocks, nx, ny, nz, dev_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    lbm::set_global_error(cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  return LBM_OK;
}
