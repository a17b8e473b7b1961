// Lattice kernels (fused step + field observables) with f16 population storage.
#include "lbm_lattice_inst.cuh"

namespace lbm {
cudaError_t launch_lattice_f16(int stencil, int mode, const LatticeDesc& d, TileCfg cfg,
                               const ObsArgs& oa, cudaStream_t s) {
  return dispatch_lattice<kF16>(stencil, mode, d, cfg, oa, s);
}
cudaError_t launch_batch_f16(int stencil, int mode, const BatchEntry* table,
                              const BatchHeader* hdr, int step, bool prepare, int* grid,
                              cudaStream_t s) {
  if (stencil != 4) return cudaErrorInvalidValue;
  return dispatch_batch<kF16, 4>(mode, table, hdr, step, prepare, grid, s);
}
}  // namespace lbm
