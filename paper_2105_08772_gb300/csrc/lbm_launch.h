// Host-side launch interface between the C-ABI (lbm_api.cu) and the kernel
// translation units (one per storage precision).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_common.cuh"
#include "lbm_kernels.cuh"

namespace lbm {

// Step-kernel configuration.  kind 0: lattice_kernel (register loads), one CTA
// per (column, chunk of zchunk planes).  kind 1: lattice_async_kernel
// (cp.async stages, prefetch depth `depth`) on a persistent grid; zchunk 0
// lets the launcher choose the chunk, > 0 fixes it.  kind 4: lattice_chunk_kernel
// (16-byte row chunks), kind 5: the unit-tau moment kernel with row chunks, kind 6:
// the moment kernel with element copies; same grid rules.
// prepare = true launches nothing: it sets the kernel's shared-memory limit
// (and caches the occupancy), which must happen outside any stream capture.
struct TileCfg {
  int bx, by, zchunk;
  int kind = 0;
  int depth = 1;
  bool prepare = false;
};

// TMA tensor maps of both population buffers of one lattice (host side; kind 7):
// map[b][0] boxes XW x PY, map[b][k] XW x k wrapped rows (k = 1 .. R + 1),
// map[b][R + 2] 4 x PY (a 16-byte x apron), over the 4-D view (x, y, z,
// population) of buffer b
struct TmaMaps {
  int ok = 0;
  int bx = 0, by = 0;               // tile shape the boxes were encoded for
  const void* base[2] = {nullptr, nullptr};
  CUtensorMap map[2][kMaxTmaMaps];
};
// Encode the maps of one FP32 lattice for bx x by tiles of a stencil of radius R.
// Returns false (t->ok = 0) when the box or the lattice does not meet the TMA
// kernel's requirements or the driver's encoder is unavailable or refuses.
bool build_tma_maps(TmaMaps* t, const void* pop0, const void* pop1, int nx, int ny, int nz, int R, int bx,
                    int by);
// the TMA kernel's requirements on the box (kind 7)
inline bool tma_box_ok(int nx, int ny, int nz, int by) {
  return nx % 4 == 0 && nx >= 64 && ny % by == 0 && ny >= 2 * by && nz >= 3;
}
// tile shapes compiled for the register-load step kernel (E4 / wider stencils)
constexpr int kNumShapesE4 = 3;
constexpr int kShapesE4[kNumShapesE4][2] = {{32, 4}, {32, 8}, {64, 4}};
constexpr int kNumShapesWide = 2;
constexpr int kShapesWide[kNumShapesWide][2] = {{32, 4}, {32, 8}};
// (bx, by, depth) compiled for the pipelined step kernel (F32 / F64 storage)
constexpr int kNumAsyncE4 = 5;
constexpr int kAsyncE4[kNumAsyncE4][3] = {{32, 8, 1}, {32, 8, 2}, {32, 4, 1}, {32, 4, 2}, {64, 4, 1}};
constexpr int kNumAsyncWide = 2;
constexpr int kAsyncWide[kNumAsyncWide][3] = {{32, 4, 1}, {32, 8, 1}};

// Launch one step (mode kModeStep) or the field-observable pass (kModeObs)
// for a lattice of the given precision and stencil.  Returns
// cudaErrorInvalidValue for a configuration that is not compiled.
cudaError_t launch_lattice_f64(int stencil, int mode, const LatticeDesc& d, TileCfg cfg,
                               const ObsArgs& oa, cudaStream_t s);
cudaError_t launch_lattice_f32(int stencil, int mode, const LatticeDesc& d, TileCfg cfg,
                               const ObsArgs& oa, cudaStream_t s);
cudaError_t launch_lattice_f16(int stencil, int mode, const LatticeDesc& d, TileCfg cfg,
                               const ObsArgs& oa, cudaStream_t s);

inline cudaError_t launch_lattice(int prec, int stencil, int mode, const LatticeDesc& d,
                                  TileCfg cfg, const ObsArgs& oa, cudaStream_t s) {
  switch (prec) {
    case kF64: return launch_lattice_f64(stencil, mode, d, cfg, oa, s);
    case kF32: return launch_lattice_f32(stencil, mode, d, cfg, oa, s);
    case kF16: return launch_lattice_f16(stencil, mode, d, cfg, oa, s);
  }
  return cudaErrorInvalidValue;
}

// dynamic shared memory of the pipelined kernel: (R + 1 + depth) population
// stages and 2R + 1 psi planes of the padded (bx + 2R) x (by + 2R) tile
constexpr size_t async_smem_bytes(size_t elem, int R, int bx, int by, int depth) {
  return elem * (size_t)(bx + 2 * R) * (by + 2 * R) * ((R + 1 + depth) * Q + 2 * R + 1);
}
// dynamic shared memory of the chunked kernel: (R + 1 + depth) stages of
// 19 x (by + 2R) rows of bx + 8 elements, psi ring of 2R + 1 padded planes
constexpr size_t chunk_smem_bytes(size_t elem, int R, int bx, int by, int depth) {
  return elem * ((size_t)(R + 1 + depth) * Q * (by + 2 * R) * (bx + 8) +
                 (size_t)(2 * R + 1) * (bx + 2 * R) * (by + 2 * R));
}
// (bx, by, depth) compiled for the chunked step kernel (kind 4)
constexpr int kNumChunkE4 = 5;
constexpr int kChunkE4[kNumChunkE4][3] = {{32, 8, 1}, {32, 8, 2}, {32, 4, 1}, {32, 4, 2}, {64, 4, 1}};
constexpr int kNumChunkWide = 1;
constexpr int kChunkWide[kNumChunkWide][3] = {{32, 4, 1}};

// staged left of a tile by the chunked copies: one 16-byte chunk, at least 4
constexpr int chunk_apron(size_t stored) { return 16 / (int)stored > 4 ? 16 / (int)stored : 4; }
// dynamic shared memory of the unit-tau moment kernel: 1 + depth stages of the
// stored type (rows of bx + 2 apron), psi ring of 2R + 2 padded planes in the
// arithmetic type
// (FP32 32 x 8 E4 tiles pad each staged row by 4 floats: see MomentShape::XWS)
constexpr size_t moment_smem_bytes(size_t stored, size_t arith, int R, int bx, int by, int depth) {
  return stored * (size_t)(1 + depth) * Q * (by + 2 * R) *
             (bx + 2 * chunk_apron(stored) + ((stored == 4 && bx == 32 && by == 8 && R == 1) ? 4 : 0)) +
         arith * (size_t)(2 * R + 2) * (bx + 2 * R) * (by + 2 * R);
}
// (bx, by, depth) compiled for the moment kernel (kind 5; tau = 1, else the
// chunked kernel of the same shape runs)
constexpr int kNumMomentE4 = 5;
constexpr int kMomentE4[kNumMomentE4][3] = {{32, 8, 1}, {32, 8, 2}, {32, 4, 1}, {32, 4, 2}, {64, 4, 1}};
constexpr int kNumMomentWide = 1;
constexpr int kMomentWide[kNumMomentWide][3] = {{32, 4, 1}};

// the moment kernel with element copies (kind 6): 1 + depth stages of 19 padded
// planes of the stored type, psi ring of 2R + 2 padded planes
constexpr size_t moment_elem_smem_bytes(size_t stored, size_t arith, int R, int bx, int by, int depth) {
  return ((size_t)(1 + depth) * Q * stored + (size_t)(2 * R + 2) * arith) * (bx + 2 * R) * (by + 2 * R);
}

// kind 6 runs 2 CTAs per SM (228 KB of shared memory, 1 KB reserved per CTA)
constexpr bool moment_elem_two_per_sm(size_t elem, int R, int bx, int by, int depth) {
  return 2 * (moment_elem_smem_bytes(elem, elem, R, bx, by, depth) + 1024) <= 228 * 1024;
}

constexpr size_t kMaxSmemPerCta = 227 * 1024;   // opt-in limit of one CTA on sm_103

// number of CTAs (= FieldPartial records) a kind-0 lattice launch uses
inline long long lattice_grid_ctas(const LatticeDesc& d, TileCfg cfg) {
  const long long tiles = (long long)((d.nx + cfg.bx - 1) / cfg.bx) * ((d.ny + cfg.by - 1) / cfg.by);
  return tiles * ((d.nz + cfg.zchunk - 1) / cfg.zchunk);
}

// ---------------------------------------------------------------- batches
struct BatchEntry;
struct BatchHeader;
// the tile every batch of this precision / stencil uses, and its launch;
// prepare readies the kernel outside capture and reports the grid it uses
// batch kernel modes: lattices with mixed tau, all tau = 1, or all tau = 1 with
// boxes the moment kernel takes (nx % 4 == 0, nx >= tile width + 8)
// (kBatchMomentElem: all tau = 1, some box not split into 16-byte row chunks: the
// moment kernel with element copies)
enum BatchMode : int { kBatchMixedTau = 0, kBatchUnitTau = 1, kBatchMoment = 2, kBatchMomentElem = 3 };
inline TileCfg batch_tile(int prec, int stencil, int mode) {
  TileCfg t{32, (stencil == 4 && (prec != kF64 || mode == kBatchMomentElem)) ? 8 : 4, 0};
  t.kind = mode == kBatchMoment ? 5 : (mode == kBatchMomentElem ? 6 : 1);
  return t;
}
cudaError_t launch_batch_f64(int stencil, int mode, const BatchEntry* table, const BatchHeader* hdr,
                             int step, bool prepare, int* grid, cudaStream_t s);
cudaError_t launch_batch_f32(int stencil, int mode, const BatchEntry* table, const BatchHeader* hdr,
                             int step, bool prepare, int* grid, cudaStream_t s);
cudaError_t launch_batch_f16(int stencil, int mode, const BatchEntry* table, const BatchHeader* hdr,
                             int step, bool prepare, int* grid, cudaStream_t s);
inline cudaError_t launch_batch(int prec, int stencil, int mode, const BatchEntry* table,
                                const BatchHeader* hdr, int step, bool prepare, int* grid, cudaStream_t s) {
  if (prec == kF64) return launch_batch_f64(stencil, mode, table, hdr, step, prepare, grid, s);
  if (prec == kF32) return launch_batch_f32(stencil, mode, table, hdr, step, prepare, grid, s);
  if (prec == kF16) return launch_batch_f16(stencil, mode, table, hdr, step, prepare, grid, s);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- io / init (lbm_io.cu)
struct DropInit {
  double cx, cy, cz, R, rho_in, rho_out, width;
};
cudaError_t launch_init_drop(int prec, const LatticeDesc& d, const DropInit& di, cudaStream_t s);
cudaError_t launch_init_rho(int prec, const LatticeDesc& d, const double* rho_dev, cudaStream_t s);
// write population plane i of the stored state from f_i(x, t) (device doubles)
cudaError_t launch_set_plane(int prec, const LatticeDesc& d, int i, const double* f_dev,
                             cudaStream_t s);
// read population plane i of the current f_i(x, t) into device doubles
cudaError_t launch_get_plane(int prec, const LatticeDesc& d, int i, double* f_dev, cudaStream_t s);

// ---------------------------------------------------------------- observables (lbm_obs.cu)
struct PointOut {
  double n_in, n_out, P_in, P_out;
};
// centre node, farthest corner and the +x half axis: n, P^yy, P^xx (Eq. (9))
cudaError_t launch_point_obs(int prec, int stencil, const LatticeDesc& d, PointOut* pts,
                             double* n_line, double* PT_line, double* PN_line, cudaStream_t s);

struct FinalizeArgs {
  const FieldPartial* partials;
  long long n_partials;
  const PointOut* pts;
  const double* PT_line;
  int line_len;
  long long volume;
  double contrast0;       // |rho_in - rho_out| of the initial state (0: no collapse test)
  int center[3];          // centre node (nx/2, ny/2, nz/2)
  int have_u_old;
  long long steps;
  double* dP_prev;        // device: previous Delta P (NaN if none); updated
  const int* err;         // device: set when a step kernel's bounded wait ran out
  void* obs_out;          // device lbm_obs
};
cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t s);

}  // namespace lbm
