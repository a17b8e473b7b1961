// Launch helpers that instantiate the lattice kernels; each
// lbm_lattice_<prec>.cu includes this file for its own storage precision.
#pragma once

#include "lbm_kernels_chunk.cuh"
#include "lbm_kernels_moment.cuh"
#include "lbm_kernels_tma.cuh"
#include "lbm_launch.h"

namespace lbm {

template <int P, int ST, int BX, int BY, int MODE>
static cudaError_t launch_one(const LatticeDesc& d, int zchunk, bool prepare, const ObsArgs& oa,
                              cudaStream_t s) {
  using Sh = StepShape<P, ST, BX, BY>;
  auto kern = lattice_kernel<P, ST, BX, BY, MODE>;
  if (prepare)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Sh::smem_bytes);
  if (zchunk < 1) return cudaErrorInvalidValue;
  const int tiles = ((d.nx + BX - 1) / BX) * ((d.ny + BY - 1) / BY);
  const int chunks = (d.nz + zchunk - 1) / zchunk;
  dim3 grid(tiles, chunks);
  kern<<<grid, Sh::NT, Sh::smem_bytes, s>>>(d, zchunk, oa);
  return cudaGetLastError();
}

// (cost model: rounds x (chunk + 2R), the planes the slowest CTA loads when
// (chunk, column) items are handed out round-robin to `resident` CTAs)
inline int choose_zchunk(long long cols, int nz, int R, long long resident, int zchunk) {
  if (zchunk > 0) return zchunk < nz ? zchunk : nz;
  int best_zc = nz;
  long long best_cost = -1;
  for (int zc = 1; zc <= nz; ++zc) {
    const long long items = cols * ((nz + zc - 1) / zc);
    const long long rounds = (items + resident - 1) / resident;
    const long long cost = rounds * (zc + 2 * R);
    if (best_cost < 0 || cost <= best_cost) {
      best_cost = cost;
      best_zc = zc;
    }
  }
  return best_zc;
}

// Single-lattice step kernels whose CTAs take several work items in turn are
// launched with programmatic stream serialisation (each kernel begins with
// step_grid_enter): the next step's CTAs take the slots this step's CTAs free
// and wait on the device for its completion, so consecutive steps' launch
// latency and CTA ramp overlap the previous step's tail (256^3: 499 -> 488 us).
// A grid of one item per CTA has no such tail and measured 0.6 us slower with it
// (128^3), and the batch kernel measured 26% slower over a 144-lattice sweep, so
// both are launched plainly.
template <typename... KArgs, typename... Args>
static cudaError_t launch_step_kernel(void (*kern)(KArgs...), long long grid, int threads, size_t smem,
                                      cudaStream_t s, bool overlap, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = overlap ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename Kern>
static cudaError_t prepare_persistent(Kern kern, int threads, size_t smem, int* resident) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // (the default L1/shared carveout is kept: forcing all of it to shared
  //  memory measured 1.5x slower -- the element copies profit from L1)
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  *resident = (per_sm > 0 ? per_sm : 1) * sms;
  return cudaSuccess;
}

template <int P, int ST, int BX, int BY, int D, bool UNIT_TAU>
static cudaError_t launch_async_variant(const LatticeDesc& d, int zchunk, bool prepare,
                                        cudaStream_t s) {
  using Sh = AsyncShape<P, ST, BX, BY, D>;
  static_assert(Sh::smem_bytes == async_smem_bytes(sizeof(typename Sh::T), Sh::R, BX, BY, D),
                "host and device disagree on the pipelined kernel's shared memory");
  auto kern = lattice_async_kernel<P, ST, BX, BY, D, UNIT_TAU>;
  static int resident = 0;   // CTAs of this kernel resident on the whole GPU
  if (prepare || resident == 0) {
    cudaError_t e = prepare_persistent(kern, Sh::NT, Sh::smem_bytes, &resident);
    if (e != cudaSuccess || prepare) return e;
  }
  const long long cols = (long long)((d.nx + BX - 1) / BX) * ((d.ny + BY - 1) / BY);
  const int zc = choose_zchunk(cols, d.nz, Sh::R, resident, zchunk);
  const long long items = cols * ((d.nz + zc - 1) / zc);
  const long long grid = items < resident ? items : resident;
  return launch_step_kernel(kern, grid, Sh::NT, Sh::smem_bytes, s, items > grid, d, zc);
}

template <int P, int ST, int BX, int BY, int D, bool UNIT_TAU>
static cudaError_t launch_chunk_variant(const LatticeDesc& d, int zchunk, bool prepare,
                                        cudaStream_t s) {
  using Sh = ChunkShape<P, ST, BX, BY, D>;
  static_assert(Sh::smem_bytes == chunk_smem_bytes(sizeof(typename Sh::T), Sh::R, BX, BY, D),
                "host and device disagree on the chunked kernel's shared memory");
  auto kern = lattice_chunk_kernel<P, ST, BX, BY, D, UNIT_TAU>;
  static int resident = 0;
  if (prepare || resident == 0) {
    cudaError_t e = prepare_persistent(kern, Sh::NT, Sh::smem_bytes, &resident);
    if (e != cudaSuccess || prepare) return e;
  }
  if (d.nx % 4 != 0 || d.nx < BX + 8) return cudaErrorInvalidValue;
  const long long cols = (long long)((d.nx + BX - 1) / BX) * ((d.ny + BY - 1) / BY);
  const int zc = choose_zchunk(cols, d.nz, Sh::R, resident, zchunk);
  const long long items = cols * ((d.nz + zc - 1) / zc);
  const long long grid = items < resident ? items : resident;
  return launch_step_kernel(kern, grid, Sh::NT, Sh::smem_bytes, s, items > grid, d, zc);
}

template <int P, int ST, int BX, int BY, int D>
static cudaError_t launch_chunk(const LatticeDesc& d, int zchunk, bool prepare, cudaStream_t s) {
  if (prepare) {
    cudaError_t e = launch_chunk_variant<P, ST, BX, BY, D, true>(d, 0, true, s);
    if (e != cudaSuccess) return e;
    return launch_chunk_variant<P, ST, BX, BY, D, false>(d, 0, true, s);
  }
  if (d.omega == 1.0) return launch_chunk_variant<P, ST, BX, BY, D, true>(d, zchunk, false, s);
  return launch_chunk_variant<P, ST, BX, BY, D, false>(d, zchunk, false, s);
}

// unit-tau moment kernel; for tau != 1 the chunked kernel of the same shape runs
template <int P, int ST, int BX, int BY, int D>
static cudaError_t launch_moment(const LatticeDesc& d, int zchunk, bool prepare, cudaStream_t s) {
  using Sh = MomentShape<P, ST, BX, BY, D>;
  static_assert(Sh::smem_bytes == moment_smem_bytes(sizeof(typename Sh::S), sizeof(typename Sh::T),
                                                    Sh::R, BX, BY, D),
                "host and device disagree on the moment kernel's shared memory");
  auto kern = lattice_moment_kernel<P, ST, BX, BY, D>;
  static int resident = 0;
  if (prepare || resident == 0) {
    cudaError_t e = prepare_persistent(kern, Sh::NT, Sh::smem_bytes, &resident);
    if constexpr (P != kF16)   // the tau != 1 fallback (FP16 storage has none: tau = 1 only)
      if (e == cudaSuccess && prepare) e = launch_chunk<P, ST, BX, BY, D>(d, 0, true, s);
    if (e != cudaSuccess || prepare) return e;
  }
  if (d.omega != 1.0) {
    if constexpr (P == kF16) return cudaErrorInvalidValue;
    else return launch_chunk<P, ST, BX, BY, D>(d, zchunk, false, s);
  }
  if (d.nx % Sh::VE != 0 || d.nx < BX + 2 * Sh::APRON) return cudaErrorInvalidValue;
  const long long cols = (long long)((d.nx + BX - 1) / BX) * ((d.ny + BY - 1) / BY);
  const int zc = choose_zchunk(cols, d.nz, Sh::R, resident, zchunk);
  const long long items = cols * ((d.nz + zc - 1) / zc);
  const long long grid = items < resident ? items : resident;
  return launch_step_kernel(kern, grid, Sh::NT, Sh::smem_bytes, s, items > grid, d, zc);
}

template <int P, int ST>
static cudaError_t dispatch_moment(const LatticeDesc& d, TileCfg c, cudaStream_t s) {
  if constexpr (P == kF16) {   // FP16 storage: E4, 32 x 8 tiles
    if (ST == 4 && c.bx == 32 && c.by == 8 && c.depth == 1)
      return launch_moment<P, 4, 32, 8, 1>(d, c.zchunk, c.prepare, s);
    if (ST == 4 && c.bx == 32 && c.by == 8 && c.depth == 2)
      return launch_moment<P, 4, 32, 8, 2>(d, c.zchunk, c.prepare, s);
    return cudaErrorInvalidValue;
  } else {
    const bool prep = c.prepare;
    if (ST == 4) {
      if (c.bx == 32 && c.by == 8 && c.depth == 1) return launch_moment<P, 4, 32, 8, 1>(d, c.zchunk, prep, s);
      if (c.bx == 32 && c.by == 8 && c.depth == 2) return launch_moment<P, 4, 32, 8, 2>(d, c.zchunk, prep, s);
      if (c.bx == 32 && c.by == 4 && c.depth == 1) return launch_moment<P, 4, 32, 4, 1>(d, c.zchunk, prep, s);
      if (c.bx == 32 && c.by == 4 && c.depth == 2) return launch_moment<P, 4, 32, 4, 2>(d, c.zchunk, prep, s);
      if (c.bx == 64 && c.by == 4 && c.depth == 1) return launch_moment<P, 4, 64, 4, 1>(d, c.zchunk, prep, s);
    } else {
      if (c.bx == 32 && c.by == 4 && c.depth == 1) return launch_moment<P, ST, 32, 4, 1>(d, c.zchunk, prep, s);
    }
    return cudaErrorInvalidValue;
  }
}

template <int P, int ST>
static cudaError_t dispatch_chunk(const LatticeDesc& d, TileCfg c, cudaStream_t s) {
  if constexpr (P == kF16) {
    return cudaErrorInvalidValue;
  } else {
    const bool prep = c.prepare;
    if (ST == 4) {
      if (c.bx == 32 && c.by == 8 && c.depth == 1) return launch_chunk<P, 4, 32, 8, 1>(d, c.zchunk, prep, s);
      if (c.bx == 32 && c.by == 8 && c.depth == 2) return launch_chunk<P, 4, 32, 8, 2>(d, c.zchunk, prep, s);
      if (c.bx == 32 && c.by == 4 && c.depth == 1) return launch_chunk<P, 4, 32, 4, 1>(d, c.zchunk, prep, s);
      if (c.bx == 32 && c.by == 4 && c.depth == 2) return launch_chunk<P, 4, 32, 4, 2>(d, c.zchunk, prep, s);
      if (c.bx == 64 && c.by == 4 && c.depth == 1) return launch_chunk<P, 4, 64, 4, 1>(d, c.zchunk, prep, s);
    } else {
      if (c.bx == 32 && c.by == 4 && c.depth == 1) return launch_chunk<P, ST, 32, 4, 1>(d, c.zchunk, prep, s);
    }
    return cudaErrorInvalidValue;
  }
}

// Pipelined step kernel on a persistent grid of (resident CTAs per SM) x SMs;
// tau = 1 runs a specialised collision; prepare readies both variants.
template <int P, int ST, int BX, int BY, int D>
static cudaError_t launch_async(const LatticeDesc& d, int zchunk, bool prepare, cudaStream_t s) {
  if (prepare) {
    cudaError_t e = launch_async_variant<P, ST, BX, BY, D, true>(d, 0, true, s);
    if (e != cudaSuccess) return e;
    return launch_async_variant<P, ST, BX, BY, D, false>(d, 0, true, s);
  }
  if (d.omega == 1.0) return launch_async_variant<P, ST, BX, BY, D, true>(d, zchunk, false, s);
  return launch_async_variant<P, ST, BX, BY, D, false>(d, zchunk, false, s);
}

// the moment kernel with element copies (kind 6: any nx; tau = 1, else the
// pipelined kernel of the same shape).  Two CTAs per SM, and the shared-memory
// carveout set to what they need, so L1 keeps the rest for the element copies.
template <int P, int ST, int BX, int BY, int D>
static cudaError_t launch_moment_elem(const LatticeDesc& d, int zchunk, bool prepare, cudaStream_t s) {
  using Sh = MomentShape<P, ST, BX, BY, D, true>;
  static_assert(Sh::smem_bytes == moment_elem_smem_bytes(sizeof(typename Sh::S), sizeof(typename Sh::T),
                                                         Sh::R, BX, BY, D),
                "host and device disagree on the moment kernel's shared memory");
  auto kern = lattice_moment_kernel<P, ST, BX, BY, D, true>;
  static int resident = 0;
  if (prepare || resident == 0) {
    cudaError_t e = prepare_persistent(kern, Sh::NT, Sh::smem_bytes, &resident);
    if (e == cudaSuccess) {
      static_assert(2 * (Sh::smem_bytes + 1024) <= 228 * 1024, "two CTAs of kind 6 must fit an SM");
      const int pct = (int)((2 * (Sh::smem_bytes + 1024) * 100 + 228 * 1024 - 1) / (228 * 1024));
      e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
      int per_sm = 0, dev = 0, sms = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Sh::NT, Sh::smem_bytes);
      if (e == cudaSuccess) e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) resident = (per_sm < 2 ? (per_sm > 0 ? per_sm : 1) : 2) * sms;
    }
    if (e == cudaSuccess && prepare) e = launch_async<P, ST, BX, BY, D>(d, 0, true, s);
    if (e != cudaSuccess || prepare) return e;
  }
  if (d.omega != 1.0) return launch_async<P, ST, BX, BY, D>(d, zchunk, false, s);
  const long long cols = (long long)((d.nx + BX - 1) / BX) * ((d.ny + BY - 1) / BY);
  const int zc = choose_zchunk(cols, d.nz, Sh::R, resident, zchunk);
  const long long items = cols * ((d.nz + zc - 1) / zc);
  const long long grid = items < resident ? items : resident;
  return launch_step_kernel(kern, grid, Sh::NT, Sh::smem_bytes, s, items > grid, d, zc);
}

template <int P, int ST>
static cudaError_t dispatch_moment_elem(const LatticeDesc& d, TileCfg c, cudaStream_t s) {
  if constexpr (P == kF16) {
    return cudaErrorInvalidValue;
  } else {
    const bool prep = c.prepare;
    // shapes whose two CTAs fit an SM: E4 32 x 8 (depth 2 in FP32 only), wider
    // stencils 32 x 4
    if constexpr (ST == 4) {
      if (c.bx == 32 && c.by == 8 && c.depth == 1) return launch_moment_elem<P, 4, 32, 8, 1>(d, c.zchunk, prep, s);
      if constexpr (P == kF32)
        if (c.bx == 32 && c.by == 8 && c.depth == 2) return launch_moment_elem<P, 4, 32, 8, 2>(d, c.zchunk, prep, s);
    } else {
      if (c.bx == 32 && c.by == 4 && c.depth == 1) return launch_moment_elem<P, ST, 32, 4, 1>(d, c.zchunk, prep, s);
    }
    return cudaErrorInvalidValue;
  }
}

template <int P, int ST>
static cudaError_t dispatch_async(const LatticeDesc& d, TileCfg c, cudaStream_t s) {
  if constexpr (P == kF16) {
    return cudaErrorInvalidValue;
  } else {
    const bool prep = c.prepare;
    const int depth = c.depth;
    if (ST == 4) {
      if (c.bx == 32 && c.by == 8 && depth == 1) return launch_async<P, 4, 32, 8, 1>(d, c.zchunk, prep, s);
      if (c.bx == 32 && c.by == 8 && depth == 2) return launch_async<P, 4, 32, 8, 2>(d, c.zchunk, prep, s);
      if (c.bx == 32 && c.by == 4 && depth == 2) return launch_async<P, 4, 32, 4, 2>(d, c.zchunk, prep, s);
      if (c.bx == 32 && c.by == 4 && depth == 1) return launch_async<P, 4, 32, 4, 1>(d, c.zchunk, prep, s);
      if (c.bx == 64 && c.by == 4 && depth == 1) return launch_async<P, 4, 64, 4, 1>(d, c.zchunk, prep, s);
    } else {
      if (c.bx == 32 && c.by == 4 && depth == 1) return launch_async<P, ST, 32, 4, 1>(d, c.zchunk, prep, s);
      if (c.bx == 32 && c.by == 8 && depth == 1) return launch_async<P, ST, 32, 8, 1>(d, c.zchunk, prep, s);
    }
    return cudaErrorInvalidValue;
  }
}

template <int P, int ST, int BX, int BY, int D, bool MIXED_TAU>
static cudaError_t launch_batch_variant(const BatchEntry* table, const BatchHeader* hdr, int step,
                                        bool prepare, int* grid, cudaStream_t s) {
  using Sh = AsyncShape<P, ST, BX, BY, D>;
  auto kern = lattice_async_batch_kernel<P, ST, BX, BY, D, MIXED_TAU>;
  static int resident = 0;
  if (prepare || resident == 0) {
    cudaError_t e = prepare_persistent(kern, Sh::NT, Sh::smem_bytes, &resident);
    if (e != cudaSuccess) return e;
  }
  if (grid) *grid = resident;
  if (prepare) return cudaSuccess;
  return launch_step_kernel(kern, resident, Sh::NT, Sh::smem_bytes, s, false, table, hdr, step);
}

template <int P, int ST, int BX, int BY, int D, bool ELEM = false>
static cudaError_t launch_moment_batch_variant(const BatchEntry* table, const BatchHeader* hdr, int step,
                                               bool prepare, int* grid, cudaStream_t s) {
  using Sh = MomentShape<P, ST, BX, BY, D, ELEM>;
  auto kern = lattice_moment_batch_kernel<P, ST, BX, BY, D, ELEM>;
  static int resident = 0;
  if (prepare || resident == 0) {
    cudaError_t e = prepare_persistent(kern, Sh::NT, Sh::smem_bytes, &resident);
    if constexpr (ELEM) {   // two CTAs per SM, the rest of the SM's memory left to L1
      static_assert(2 * (Sh::smem_bytes + 1024) <= 228 * 1024, "two CTAs of kind 6 must fit an SM");
      const int pct = (int)((2 * (Sh::smem_bytes + 1024) * 100 + 228 * 1024 - 1) / (228 * 1024));
      if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
      int per_sm = 0, dev = 0, sms = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Sh::NT, Sh::smem_bytes);
      if (e == cudaSuccess) e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) resident = (per_sm < 2 ? (per_sm > 0 ? per_sm : 1) : 2) * sms;
    }
    if (e != cudaSuccess) return e;
  }
  if (grid) *grid = resident;
  if (prepare) return cudaSuccess;
  return launch_step_kernel(kern, resident, Sh::NT, Sh::smem_bytes, s, false, table, hdr, step);
}

// batches: the moment kernel when every lattice allows it, else the pipelined
// kernel; 32 x 8 tiles for FP32 E4, 32 x 4 otherwise (batch_tile)
template <int P, int ST>
static cudaError_t dispatch_batch(int mode, const BatchEntry* table, const BatchHeader* hdr,
                                  int step, bool prepare, int* grid, cudaStream_t s) {
  if constexpr (P == kF16) {   // FP16 storage: the moment kernel, E4, 32 x 8 tiles
    if (ST == 4 && mode == kBatchMoment)
      return launch_moment_batch_variant<P, 4, 32, 8, 1>(table, hdr, step, prepare, grid, s);
    return cudaErrorInvalidValue;
  } else if constexpr (P == kF32 && ST == 4) {
    if (mode == kBatchMoment) return launch_moment_batch_variant<P, ST, 32, 8, 1>(table, hdr, step, prepare, grid, s);
    if (mode == kBatchMomentElem)
      return launch_moment_batch_variant<P, ST, 32, 8, 1, true>(table, hdr, step, prepare, grid, s);
    if (mode == kBatchUnitTau) return launch_batch_variant<P, ST, 32, 8, 1, false>(table, hdr, step, prepare, grid, s);
    return launch_batch_variant<P, ST, 32, 8, 1, true>(table, hdr, step, prepare, grid, s);
  } else {
    if (mode == kBatchMomentElem) {
      if constexpr (ST == 4)   // FP64 E4: 32 x 8 tiles (the kind-6 shape)
        return launch_moment_batch_variant<P, ST, 32, 8, 1, true>(table, hdr, step, prepare, grid, s);
      else
        return launch_moment_batch_variant<P, ST, 32, 4, 1, true>(table, hdr, step, prepare, grid, s);
    }
    if (mode == kBatchMoment) return launch_moment_batch_variant<P, ST, 32, 4, 1>(table, hdr, step, prepare, grid, s);
    if (mode == kBatchUnitTau) return launch_batch_variant<P, ST, 32, 4, 1, false>(table, hdr, step, prepare, grid, s);
    return launch_batch_variant<P, ST, 32, 4, 1, true>(table, hdr, step, prepare, grid, s);
  }
}

template <int P>
static cudaError_t dispatch_batch_stencil(int stencil, int mode, const BatchEntry* table,
                                          const BatchHeader* hdr, int step, bool prepare, int* grid,
                                          cudaStream_t s) {
  if (stencil == 4) return dispatch_batch<P, 4>(mode, table, hdr, step, prepare, grid, s);
  if (stencil == 6) return dispatch_batch<P, 6>(mode, table, hdr, step, prepare, grid, s);
  if (stencil == 8) return dispatch_batch<P, 8>(mode, table, hdr, step, prepare, grid, s);
  return cudaErrorInvalidValue;
}

// the unit-tau moment kernel fed by TMA tensor-tile copies (kind 7; FP32 storage,
// tau = 1, the box rules of tma_box_ok, tensor maps encoded for this tile)
template <int ST, int BX, int BY>
static cudaError_t launch_tma(const LatticeDesc& d, int zchunk, bool prepare, cudaStream_t s) {
  using Sh = TmaShape<ST, BX, BY>;
  auto kern = lattice_tma_kernel<ST, BX, BY>;
  static int resident = 0;
  if (prepare || resident == 0) {
    cudaError_t e = prepare_persistent(kern, Sh::NT, Sh::smem_bytes, &resident);
    if (e != cudaSuccess || prepare) return e;
  }
  const TmaMaps* tm = static_cast<const TmaMaps*>(d.tma);
  if (!tm || !tm->ok || tm->bx != BX || tm->by != BY || d.omega != 1.0) return cudaErrorInvalidValue;
  if (!tma_box_ok(d.nx, d.ny, d.nz, BY)) return cudaErrorInvalidValue;
  const int b = d.src == tm->base[0] ? 0 : (d.src == tm->base[1] ? 1 : -1);
  if (b < 0) return cudaErrorInvalidValue;
  TmaMapSet maps;
  for (int k = 0; k < kMaxTmaMaps; ++k) maps.map[k] = tm->map[b][k];
  const long long cols = (long long)((d.nx + BX - 1) / BX) * (d.ny / BY);
  const int zc = choose_zchunk(cols, d.nz, Sh::R, resident, zchunk);
  const long long items = cols * ((d.nz + zc - 1) / zc);
  const long long grid = items < resident ? items : resident;
  return launch_step_kernel(kern, grid, Sh::NT, Sh::smem_bytes, s, items > grid, d, maps, zc);
}

template <int P, int ST>
static cudaError_t dispatch_tma(const LatticeDesc& d, TileCfg c, cudaStream_t s) {
  if constexpr (P == kF32 && ST == 4) {
    if (c.bx == 32 && c.by == 8 && c.depth == 1) return launch_tma<4, 32, 8>(d, c.zchunk, c.prepare, s);
  }
  return cudaErrorInvalidValue;
}

template <int P, int ST, int MODE>
static cudaError_t dispatch_shape(const LatticeDesc& d, TileCfg c, const ObsArgs& oa,
                                  cudaStream_t s) {
  if (c.bx == 32 && c.by == 4) return launch_one<P, ST, 32, 4, MODE>(d, c.zchunk, c.prepare, oa, s);
  if (c.bx == 32 && c.by == 8) return launch_one<P, ST, 32, 8, MODE>(d, c.zchunk, c.prepare, oa, s);
  if (ST == 4 && c.bx == 64 && c.by == 4)
    return launch_one<P, 4, 64, 4, MODE>(d, c.zchunk, c.prepare, oa, s);
  return cudaErrorInvalidValue;
}

template <int P>
static cudaError_t dispatch_lattice(int stencil, int mode, const LatticeDesc& d, TileCfg c,
                                    const ObsArgs& oa, cudaStream_t s) {
  if (c.zchunk < 0) return cudaErrorInvalidValue;
  if (mode == kModeStep && c.kind == 7) {
    if (stencil == 4) return dispatch_tma<P, 4>(d, c, s);
    return cudaErrorInvalidValue;
  }
  if (mode == kModeStep && c.kind == 6) {
    if (stencil == 4) return dispatch_moment_elem<P, 4>(d, c, s);
    if (stencil == 6) return dispatch_moment_elem<P, 6>(d, c, s);
    if (stencil == 8) return dispatch_moment_elem<P, 8>(d, c, s);
    return cudaErrorInvalidValue;
  }
  if (mode == kModeStep && c.kind == 5) {
    if (stencil == 4) return dispatch_moment<P, 4>(d, c, s);
    if (stencil == 6) return dispatch_moment<P, 6>(d, c, s);
    if (stencil == 8) return dispatch_moment<P, 8>(d, c, s);
    return cudaErrorInvalidValue;
  }
  if (mode == kModeStep && c.kind == 4) {
    if (stencil == 4) return dispatch_chunk<P, 4>(d, c, s);
    if (stencil == 6) return dispatch_chunk<P, 6>(d, c, s);
    if (stencil == 8) return dispatch_chunk<P, 8>(d, c, s);
    return cudaErrorInvalidValue;
  }
  if (mode == kModeStep && c.kind == 1) {
    if (stencil == 4) return dispatch_async<P, 4>(d, c, s);
    if (stencil == 6) return dispatch_async<P, 6>(d, c, s);
    if (stencil == 8) return dispatch_async<P, 8>(d, c, s);
    return cudaErrorInvalidValue;
  }
  if (mode == kModeStep) {
    if (stencil == 4) return dispatch_shape<P, 4, kModeStep>(d, c, oa, s);
    if (stencil == 6) return dispatch_shape<P, 6, kModeStep>(d, c, oa, s);
    if (stencil == 8) return dispatch_shape<P, 8, kModeStep>(d, c, oa, s);
  } else {
    // one shape for the field-observable pass
    TileCfg o{32, 4, c.zchunk};
    o.prepare = c.prepare;
    if (stencil == 4) return dispatch_shape<P, 4, kModeObs>(d, o, oa, s);
    if (stencil == 6) return dispatch_shape<P, 6, kModeObs>(d, o, oa, s);
    if (stencil == 8) return dispatch_shape<P, 8, kModeObs>(d, o, oa, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
