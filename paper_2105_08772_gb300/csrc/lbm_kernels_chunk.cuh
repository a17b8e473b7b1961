// Chunked variant of the pipelined Shan-Chen step (FP32 / FP64 storage).
//
// Same pipeline and arithmetic as lattice_async_kernel; the copies differ.
// Instead of one 4- or 8-byte cp.async per pulled population and padded node,
// a stage row of population i holds the 16-byte aligned x range
// [x0 - 4, x0 + BX + 4) of the source row, filled
// by 16-byte cp.async.cg copies (L2 only, no L1 allocation).  Because nx is a
// multiple of 4, every 16-byte chunk lies wholly inside the row or wholly in its
// periodic image, so a chunk wraps as a unit.  The pull shift in x becomes an
// index offset into the staged row.  Requirements: nx % 4 == 0, nx >= BX + 8.
//
// Per plane: 19 x (BY + 2R) x (BX + 8) / 4 (FP32) chunk copies per CTA instead of
// 19 x (BX + 2R)(BY + 2R) element copies: ~3.4x fewer copy instructions, each
// with its address one add away from per-thread constants.
#pragma once

#include "lbm_kernels_async.cuh"

namespace lbm {

constexpr int kChunkApron = 4;   // staged elements left of the tile (one 16-byte FP32 chunk)

template <int P, int ST, int BX, int BY, int D>
struct ChunkShape {
  using T = typename Storage<P>::T;
  static constexpr int R = stencil_radius<ST>();
  static constexpr int PX = BX + 2 * R;
  static constexpr int PY = BY + 2 * R;
  static constexpr int NPAD = PX * PY;
  static constexpr int NT = BX * BY;
  static constexpr int XW = BX + 2 * kChunkApron;       // staged row width
  static constexpr int VE = 16 / (int)sizeof(T);       // elements per chunk
  static constexpr int NCH = XW / VE;                  // chunks per staged row
  static constexpr int NS = R + 1 + D;
  static constexpr int NR = 2 * R + 1;
  static constexpr int NPER = (NPAD + NT - 1) / NT;
  static constexpr size_t stage_elems = (size_t)Q * PY * XW;
  static constexpr size_t smem_bytes = sizeof(T) * (NS * stage_elems + NR * NPAD);
  static_assert(XW % VE == 0, "staged rows are whole chunks");
  static_assert(R + 1 <= kChunkApron, "apron must cover the pull of the halo");
};

__device__ __forceinline__ void cp_async_chunk16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

template <int P, int ST, int BX, int BY, int D, bool UNIT_TAU>
__device__ __forceinline__ void chunk_process_item(const LatticeDesc& d, int zchunk, long long item,
                                                   unsigned char* smem_raw) {
  using Sh = ChunkShape<P, ST, BX, BY, D>;
  using T = typename Sh::T;
  using S = typename Storage<P>::S;
  static_assert(sizeof(S) == sizeof(T), "chunk path copies stored values unchanged");
  constexpr int R = Sh::R, PX = Sh::PX, PY = Sh::PY, NPAD = Sh::NPAD, NT = Sh::NT;
  constexpr int XW = Sh::XW, VE = Sh::VE, NCH = Sh::NCH, NS = Sh::NS, NR = Sh::NR;
  constexpr int NPER = Sh::NPER;
  T* stages = reinterpret_cast<T*>(smem_raw);
  T* ring = stages + NS * Sh::stage_elems;

  const int nx = d.nx, ny = d.ny, nz = d.nz;
  const long long plane = d.plane;
  const S* __restrict__ src = static_cast<const S*>(d.src);
  S* __restrict__ dst = static_cast<S*>(d.dst);
  const T n0 = dparam<T>(d.n0, d.n0f), G = dparam<T>(d.eos.G, d.eos.Gf), omega = dparam<T>(d.omega, d.omegaf);
  const int tiles_x = (nx + BX - 1) / BX;
  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int ncols = tiles_x * ((ny + BY - 1) / BY);

  const int col = (int)(item % ncols);
  const int z0 = (int)(item / ncols) * zchunk;
  const int zc = min(zchunk, nz - z0);
  const int x0 = (col % tiles_x) * BX, y0 = (col / tiles_x) * BY;
  const int w = min(BX, nx - x0), h = min(BY, ny - y0);
  const bool active = tx < w && ty < h;
  const int rows = h + 2 * R;
  const int xa = x0 - kChunkApron;

  // copy positions: a position is one 16-byte chunk (staged row jy, chunk k) of a
  // stage; a thread copies its position for a fixed range of populations, so
  // population, pull shift and plane offset are compile-time constants of the
  // unrolled copy loop.  With 2 POS <= NT two thread groups split the 19
  // populations; otherwise every position is copied for all 19 by one thread.
  constexpr int POS = PY * NCH;
  constexpr int NG = (2 * POS <= NT) ? 2 : 1;
  constexpr int NPP = NG == 2 ? 1 : (POS + NT - 1) / NT;
  constexpr int ISPLIT = NG == 2 ? 10 : Q;
  const int grp = NG == 2 ? tid / POS : 0;        // 0, 1 (or idle)
  const S* srcp[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) srcp[i] = src + i * plane;
  int prow[NPP][3], pgx[NPP], psm[NPP];
  bool pok[NPP];
#pragma unroll
  for (int pp = 0; pp < NPP; ++pp) {
    const int p = NG == 2 ? tid % POS : tid + pp * NT;
    const int jy = p / NCH, k = p % NCH;
    pok[pp] = (NG == 2 ? grp < 2 : p < POS) && jy < rows;
    const int y = wrap(y0 - R + (pok[pp] ? jy : 0), ny);
    prow[pp][0] = wrap(y + 1, ny) * nx;     // source row for c_y = -1
    prow[pp][1] = y * nx;
    prow[pp][2] = wrap(y - 1, ny) * nx;     // source row for c_y = +1
    pgx[pp] = wrap(xa + k * VE, nx);
    psm[pp] = jy * XW + k * VE;
  }
  bool valid[NPER];
#pragma unroll
  for (int s = 0; s < NPER; ++s) {
    const int j = tid + s * NT;
    valid[s] = j < NPAD && (j % PX) < w + 2 * R && (j / PX) < rows;
  }
  const int nplanes = zc + 2 * R;

  auto issue = [&](int q) {
    if (q < nplanes) {
      const int z = wrap(z0 - R + q, nz);
      const int zo[3] = {wrap(z + 1, nz) * ny * nx, z * ny * nx, wrap(z - 1, nz) * ny * nx};
      T* st = stages + (q % NS) * Sh::stage_elems;
#pragma unroll
      for (int pp = 0; pp < NPP; ++pp) {
        if (!pok[pp]) continue;
        if (grp == 0) {
#pragma unroll
          for (int i = 0; i < ISPLIT; ++i)
            cp_async_chunk16(st + i * PY * XW + psm[pp],
                             srcp[i] + (zo[cz(i) + 1] + prow[pp][cy(i) + 1] + pgx[pp]));
        } else if (NG == 2) {
#pragma unroll
          for (int i = ISPLIT; i < Q; ++i)
            cp_async_chunk16(st + i * PY * XW + psm[pp],
                             srcp[i] + (zo[cz(i) + 1] + prow[pp][cy(i) + 1] + pgx[pp]));
        }
      }
    }
    cp_async_commit();
  };

  __syncthreads();   // the previous item's readers are done with every stage
#pragma unroll 1
  for (int q = 0; q < D; ++q) issue(q);

#pragma unroll 1
  for (int qd = 0; qd < nplanes; ++qd) {
    cp_async_wait<D - 1>();
    __syncthreads();
    issue(qd + D);
    {  // density and psi of plane qd
      const T* st = stages + (qd % NS) * Sh::stage_elems;
      T* rs = ring + (qd % NR) * NPAD;
#pragma unroll
      for (int s = 0; s < NPER; ++s) {
        if (!valid[s]) continue;
        const int j = tid + s * NT;
        const int jx = j % PX, jy = j / PX;
        const T* row0 = st + jy * XW + jx + kChunkApron - R;
        T v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = row0[i * PY * XW - cx(i)];
        rs[j] = psi_of<T>(n0 + sum19(v), d.eos);
      }
    }
    __syncthreads();
    const int qc = qd - R;
    const int k = qc - R;
    if (k >= 0 && active) {
      const T* st = stages + (qc % NS) * Sh::stage_elems;
      const int jc = (ty + R) * PX + (tx + R);
      const T* row0 = st + (ty + R) * XW + tx + kChunkApron;
      T g[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] = row0[i * PY * XW - cx(i)];
      const T* planes[2 * R + 1];
#pragma unroll
      for (int dz = -R; dz <= R; ++dz) planes[dz + R] = ring + ((qc + dz) % NR) * NPAD + jc;
      T Fx, Fy, Fz;
      sc_force_pairs<T, ST, PX>(planes, G, Fx, Fy, Fz);
      T dn, jx, jy, jz;
      moments(g, dn, jx, jy, jz);
      const T n = n0 + dn;
      const T inv_n = (T)1 / n;
      const T ux = (jx + (T)0.5 * Fx) * inv_n;
      const T uy = (jy + (T)0.5 * Fy) * inv_n;
      const T uz = (jz + (T)0.5 * Fz) * inv_n;
      collide<T, true, UNIT_TAU>(g, dn, n, ux, uy, uz, Fx, Fy, Fz, omega);
      const long long node = ((long long)(z0 + k) * ny + (y0 + ty)) * nx + (x0 + tx);
#pragma unroll
      for (int i = 0; i < Q; ++i) dst[i * plane + node] = (S)g[i];
    }
  }
  cp_async_wait_all();
}

template <int P, int ST, int BX, int BY, int D, bool UNIT_TAU>
__global__ void __launch_bounds__(BX * BY, (async_min_blocks<BX * BY, ChunkShape<P, ST, BX, BY, D>::smem_bytes>()))
lattice_chunk_kernel(LatticeDesc d, int zchunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  step_grid_enter();
  const int ncols = ((d.nx + BX - 1) / BX) * ((d.ny + BY - 1) / BY);
  const long long items = (long long)ncols * ((d.nz + zchunk - 1) / zchunk);
#pragma unroll 1
  for (long long item = blockIdx.x; item < items; item += gridDim.x)
    chunk_process_item<P, ST, BX, BY, D, UNIT_TAU>(d, zchunk, item, smem_raw);
}

}  // namespace lbm
