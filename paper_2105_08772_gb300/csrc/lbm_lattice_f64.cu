// Lattice kernels (fused step + field observables) with f64 population storage.
#include "lbm_lattice_inst.cuh"

namespace lbm {
cudaError_t launch_lattice_f64(int stencil, int mode, const LatticeDesc& d, TileCfg cfg,
                               const ObsArgs& oa, cudaStream_t s) {
  return dispatch_lattice<kF64>(stencil, mode, d, cfg, oa, s);
}
cudaError_t launch_batch_f64(int stencil, int mode, const BatchEntry* table,
                              const BatchHeader* hdr, int step, bool prepare, int* grid,
                              cudaStream_t s) {
  return dispatch_batch_stencil<kF64>(stencil, mode, table, hdr, step, prepare, grid, s);
}
}  // namespace lbm
