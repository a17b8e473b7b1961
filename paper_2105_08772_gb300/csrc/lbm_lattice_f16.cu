// Lattice kernels (fused step + field observables) with f16 population storage.
#include "lbm_lattice_inst.cuh"

namespace lbm {
cudaError_t launch_lattice_f16(int stencil, int mode, const LatticeDesc& d, TileCfg cfg,
                               const ObsArgs& oa, cudaStream_t s) {
  return dispatch_lattice<kF16>(stencil, mode, d, cfg, oa, s);
}
}  // namespace lbm
