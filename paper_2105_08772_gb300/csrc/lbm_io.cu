// Initialisation and population transfer kernels.
//
// The stored state is post-collision, pre-streaming: slot i of node y holds
// f*_i(y, t-1) and the pre-collision population of Eq. (3) is
// f_i(x, t) = slot_i(x - xi_i).  Writing a given f_i(x, t) therefore stores
// f_i(y + xi_i, t) into slot i of node y ("un-streaming"), and reading it back
// pulls slot i from x - xi_i.
//
// Initial state (Sec. IV): fluid at rest, f_i = f_i^eq(n, u = 0) = w_i n
// (Eq. (6) at u = 0), n from the radial tanh profile of Eq. (23) or from a
// given field.  Shifted storage keeps w_i (n - n0) times the storage scale.
#include "lbm_launch.h"

namespace lbm {

namespace {

template <int P>
__device__ __forceinline__ void put(const LatticeDesc& d, int i, long long node, double f) {
  using S = typename Storage<P>::S;
  using T = typename Storage<P>::T;
  S* dst = static_cast<S*>(d.dst);
  Storage<P>::store(dst + (long long)i * d.plane + node, (T)(f - wq(i) * d.n0), (T)d.scale);
}

__device__ __forceinline__ void node_xyz(long long node, const LatticeDesc& d, int& x, int& y,
                                         int& z) {
  x = (int)(node % d.nx);
  const long long r = node / d.nx;
  y = (int)(r % d.ny);
  z = (int)(r / d.ny);
}

__device__ __forceinline__ double min_image(double c, double ctr, int n) {
  // displacement c - ctr folded into [-n/2, n/2)
  double dd = c - ctr + 0.5 * n;
  dd = dd - n * floor(dd / n);
  return dd - 0.5 * n;
}

template <int P>
__global__ void init_drop_kernel(LatticeDesc d, DropInit di) {
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < d.plane;
       node += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(node, d, x, y, z);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int xx = wrap(x + cx(i), d.nx), yy = wrap(y + cy(i), d.ny), zz = wrap(z + cz(i), d.nz);
      const double dx = min_image(xx, di.cx, d.nx), dy = min_image(yy, di.cy, d.ny),
                   dz = min_image(zz, di.cz, d.nz);
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      const double n = 0.5 * (di.rho_in + di.rho_out) -
                       0.5 * (di.rho_in - di.rho_out) * tanh((r - di.R) / di.width);
      put<P>(d, i, node, wq(i) * n);
    }
  }
}

template <int P>
__global__ void init_rho_kernel(LatticeDesc d, const double* __restrict__ rho) {
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < d.plane;
       node += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(node, d, x, y, z);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int xx = wrap(x + cx(i), d.nx), yy = wrap(y + cy(i), d.ny), zz = wrap(z + cz(i), d.nz);
      const double n = rho[((long long)zz * d.ny + yy) * d.nx + xx];
      put<P>(d, i, node, wq(i) * n);
    }
  }
}

template <int P>
__global__ void set_plane_kernel(LatticeDesc d, int i, const double* __restrict__ f) {
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < d.plane;
       node += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(node, d, x, y, z);
    const int xx = wrap(x + cx(i), d.nx), yy = wrap(y + cy(i), d.ny), zz = wrap(z + cz(i), d.nz);
    put<P>(d, i, node, f[((long long)zz * d.ny + yy) * d.nx + xx]);
  }
}

template <int P>
__global__ void get_plane_kernel(LatticeDesc d, int i, double* __restrict__ f) {
  using S = typename Storage<P>::S;
  using T = typename Storage<P>::T;
  const S* src = static_cast<const S*>(d.src);
  const T inv_scale = (T)(1.0 / d.scale);
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < d.plane;
       node += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(node, d, x, y, z);
    const int xx = wrap(x - cx(i), d.nx), yy = wrap(y - cy(i), d.ny), zz = wrap(z - cz(i), d.nz);
    const T g = Storage<P>::load(src + (long long)i * d.plane + ((long long)zz * d.ny + yy) * d.nx + xx,
                                 inv_scale);
    f[node] = (double)g + wq(i) * d.n0;
  }
}

inline dim3 grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return dim3((unsigned)b);
}

}  // namespace

#define LBM_DISPATCH_PREC(prec, KERNEL, GRID, ...)                  \
  do {                                                              \
    switch (prec) {                                                 \
      case kF64: KERNEL<kF64><<<GRID, 256, 0, s>>>(__VA_ARGS__); break; \
      case kF32: KERNEL<kF32><<<GRID, 256, 0, s>>>(__VA_ARGS__); break; \
      case kF16: KERNEL<kF16><<<GRID, 256, 0, s>>>(__VA_ARGS__); break; \
      default: return cudaErrorInvalidValue;                        \
    }                                                               \
  } while (0)

cudaError_t launch_init_drop(int prec, const LatticeDesc& d, const DropInit& di, cudaStream_t s) {
  LBM_DISPATCH_PREC(prec, init_drop_kernel, grid_for(d.plane), d, di);
  return cudaGetLastError();
}

cudaError_t launch_init_rho(int prec, const LatticeDesc& d, const double* rho_dev, cudaStream_t s) {
  LBM_DISPATCH_PREC(prec, init_rho_kernel, grid_for(d.plane), d, rho_dev);
  return cudaGetLastError();
}

cudaError_t launch_set_plane(int prec, const LatticeDesc& d, int i, const double* f_dev,
                             cudaStream_t s) {
  LBM_DISPATCH_PREC(prec, set_plane_kernel, grid_for(d.plane), d, i, f_dev);
  return cudaGetLastError();
}

cudaError_t launch_get_plane(int prec, const LatticeDesc& d, int i, double* f_dev, cudaStream_t s) {
  LBM_DISPATCH_PREC(prec, get_plane_kernel, grid_for(d.plane), d, i, f_dev);
  return cudaGetLastError();
}

}  // namespace lbm
