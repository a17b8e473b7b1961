// Launch helpers that instantiate the lattice kernels; each
// lbm_lattice_<prec>.cu includes this file for its own storage precision.
#pragma once

#include "lbm_launch.h"

namespace lbm {

// zchunk == 0 only sets the kernel's shared-memory attribute (done before
// any stream capture, since it is not a stream operation)
template <int P, int ST, int BX, int BY, int MODE>
static cudaError_t launch_one(const LatticeDesc& d, int zchunk, const ObsArgs& oa,
                              cudaStream_t s) {
  using Sh = StepShape<P, ST, BX, BY>;
  auto kern = lattice_kernel<P, ST, BX, BY, MODE>;
  if (zchunk == 0)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Sh::smem_bytes);
  const int tiles = ((d.nx + BX - 1) / BX) * ((d.ny + BY - 1) / BY);
  const int chunks = (d.nz + zchunk - 1) / zchunk;
  dim3 grid(tiles, chunks);
  kern<<<grid, Sh::NT, Sh::smem_bytes, s>>>(d, zchunk, oa);
  return cudaGetLastError();
}

template <int P, int ST, int MODE>
static cudaError_t dispatch_shape(const LatticeDesc& d, TileCfg c, const ObsArgs& oa,
                                  cudaStream_t s) {
  if (c.bx == 32 && c.by == 4) return launch_one<P, ST, 32, 4, MODE>(d, c.zchunk, oa, s);
  if (c.bx == 32 && c.by == 8) return launch_one<P, ST, 32, 8, MODE>(d, c.zchunk, oa, s);
  if (ST == 4 && c.bx == 64 && c.by == 4) return launch_one<P, 4, 64, 4, MODE>(d, c.zchunk, oa, s);
  return cudaErrorInvalidValue;
}

template <int P>
static cudaError_t dispatch_lattice(int stencil, int mode, const LatticeDesc& d, TileCfg c,
                                    const ObsArgs& oa, cudaStream_t s) {
  if (c.zchunk < 0) return cudaErrorInvalidValue;
  if (mode == kModeStep) {
    if (stencil == 4) return dispatch_shape<P, 4, kModeStep>(d, c, oa, s);
    if (stencil == 6) return dispatch_shape<P, 6, kModeStep>(d, c, oa, s);
    if (stencil == 8) return dispatch_shape<P, 8, kModeStep>(d, c, oa, s);
  } else {
    // one shape for the field-observable pass
    TileCfg o{32, 4, c.zchunk};
    if (stencil == 4) return dispatch_shape<P, 4, kModeObs>(d, o, oa, s);
    if (stencil == 6) return dispatch_shape<P, 6, kModeObs>(d, o, oa, s);
    if (stencil == 8) return dispatch_shape<P, 8, kModeObs>(d, o, oa, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
