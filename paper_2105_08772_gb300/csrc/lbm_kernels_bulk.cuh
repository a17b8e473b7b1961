// Row-bulk variant of the pipelined Shan-Chen step (FP32 / FP64 storage).
//
// Same arithmetic and pipeline as lattice_async_kernel, different copies: the
// pulled populations of a padded plane arrive as whole rows.  For population
// i and padded row jy the CTA needs x in [x0 - R - 1, x0 + BX + R + 1) of row
// (y0 - R + jy - c_y(i), z - c_z(i)); it copies the 16-byte aligned superset
// [x0 - 4, x0 + BX + 4) (XW = BX + 8 elements) with one cp.async.bulk, or two
// when the row crosses the periodic x boundary.  Requirements: nx % 4 == 0
// (16-byte aligned rows), nx >= XW (a row wraps at most once), x0 % 4 == 0.
// Every stage has an mbarrier; one thread posts the stage's byte count
// (expect_tx), the copies complete_tx against it, and every thread waits on
// the phase before reading.  Waits are bounded: after kMbarPolls polls a
// thread sets *d.err and the CTA returns instead of hanging.
//
// The density formed for the psi halo is kept (dn ring), so the collision
// takes dn from shared memory instead of re-summing the 19 populations.
#pragma once

#include <stdint.h>

#include "lbm_kernels_async.cuh"

namespace lbm {

constexpr int kBulkApron = 4;            // staged elements left of the tile
constexpr int kMbarPolls = 1 << 22;      // bound of every mbarrier wait

template <int P, int ST, int BX, int BY, int D>
struct BulkShape {
  using T = typename Storage<P>::T;
  static constexpr int R = stencil_radius<ST>();
  static constexpr int PX = BX + 2 * R;
  static constexpr int PY = BY + 2 * R;
  static constexpr int NPAD = PX * PY;
  static constexpr int NT = BX * BY;
  static constexpr int XW = BX + 2 * kBulkApron;   // staged row width
  static constexpr int NS = R + 1 + D;             // population stages
  static constexpr int NR = 2 * R + 1;             // psi / dn planes
  static constexpr int NPER = (NPAD + NT - 1) / NT;
  static constexpr size_t stage_elems = (size_t)Q * PY * XW;
  static constexpr size_t ring_elems = (size_t)NR * NPAD;
  static constexpr size_t mbar_offset =
      (sizeof(T) * (NS * stage_elems + 2 * ring_elems) + 15) / 16 * 16;
  static constexpr size_t smem_bytes = mbar_offset + 8 * NS;
  static_assert(R + 1 <= kBulkApron, "apron must cover the pull of the halo");
  static_assert(BX % 4 == 0, "tiles must start on 16-byte boundaries");
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                   smem_u32(m)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared bulk copy of `bytes` (multiple of 16, both ends 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* m) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(m))
      : "memory");
}

template <int P, int ST, int BX, int BY, int D, bool UNIT_TAU>
__global__ void __launch_bounds__(BX * BY)
lattice_bulk_kernel(LatticeDesc d, int zchunk) {
  using Sh = BulkShape<P, ST, BX, BY, D>;
  using T = typename Sh::T;
  using S = typename Storage<P>::S;
  static_assert(sizeof(S) == sizeof(T), "bulk path copies stored values unchanged");
  constexpr int R = Sh::R, PX = Sh::PX, PY = Sh::PY, NPAD = Sh::NPAD, NT = Sh::NT;
  constexpr int XW = Sh::XW, NS = Sh::NS, NR = Sh::NR, NPER = Sh::NPER;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stages = reinterpret_cast<T*>(smem_raw);
  T* ring = stages + NS * Sh::stage_elems;
  T* dnring = ring + Sh::ring_elems;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + Sh::mbar_offset);

  const int nx = d.nx, ny = d.ny, nz = d.nz;
  const long long plane = d.plane;
  const S* __restrict__ src = static_cast<const S*>(d.src);
  S* __restrict__ dst = static_cast<S*>(d.dst);
  const T n0 = (T)d.n0, G = (T)d.eos.G, omega = (T)d.omega;
  const int tiles_x = (nx + BX - 1) / BX;
  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int ncols = tiles_x * ((ny + BY - 1) / BY);
  const int nchunks = (nz + zchunk - 1) / zchunk;
  const long long items = (long long)ncols * nchunks;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&mbar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  unsigned issued = 0;   // planes this CTA has issued before the current item

#pragma unroll 1
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const int col = (int)(item % ncols);
    const int z0 = (int)(item / ncols) * zchunk;
    const int zc = min(zchunk, nz - z0);
    const int x0 = (col % tiles_x) * BX, y0 = (col / tiles_x) * BY;
    const int w = min(BX, nx - x0), h = min(BY, ny - y0);
    const bool active = tx < w && ty < h;
    const int rows = h + 2 * R;           // padded rows present in this tile
    const int nplanes = zc + 2 * R;       // plane q is z0 - R + q
    const int xa = x0 - kBulkApron;
    const unsigned stage_bytes = (unsigned)(Q * rows * XW * sizeof(T));

    bool valid[NPER];
#pragma unroll
    for (int s = 0; s < NPER; ++s) {
      const int j = tid + s * NT;
      valid[s] = j < NPAD && (j % PX) < w + 2 * R && (j / PX) < rows;
    }

    auto issue = [&](int q) {
      if (q >= nplanes) return;
      const unsigned g = issued + q;
      T* st = stages + (g % NS) * Sh::stage_elems;
      uint64_t* mb = &mbar[g % NS];
      if (tid == 0) mbar_expect_tx(mb, stage_bytes);
      const int z = wrap(z0 - R + q, nz);
      for (int r = tid; r < Q * rows; r += NT) {
        const int i = r / rows, jy = r % rows;
        const int gy = wrap(wrap(y0 - R + jy, ny) - cy_rt(i), ny);
        const int gz = wrap(z - cz_rt(i), nz);
        const S* rowp = src + i * plane + (gz * ny + gy) * nx;
        T* sp = st + (i * PY + jy) * XW;
        if (xa < 0) {                       // left part wraps to the end of the row
          bulk_g2s(sp, rowp + nx + xa, (unsigned)(-xa * sizeof(T)), mb);
          bulk_g2s(sp - xa, rowp, (unsigned)((XW + xa) * sizeof(T)), mb);
        } else if (xa + XW > nx) {          // right part wraps to the start of the row
          const int n1 = nx - xa;
          bulk_g2s(sp, rowp + xa, (unsigned)(n1 * sizeof(T)), mb);
          bulk_g2s(sp + n1, rowp, (unsigned)((XW - n1) * sizeof(T)), mb);
        } else {
          bulk_g2s(sp, rowp + xa, (unsigned)(XW * sizeof(T)), mb);
        }
      }
    };

    __syncthreads();   // the previous item's readers are done with every stage
#pragma unroll 1
    for (int q = 0; q < D; ++q) issue(q);

#pragma unroll 1
    for (int qd = 0; qd < nplanes; ++qd) {
      {
        const unsigned g = issued + qd;
        bool ok = false;
        for (int it = 0; it < kMbarPolls && !ok; ++it) ok = mbar_try_wait(&mbar[g % NS], (g / NS) & 1u);
        if (!ok) {
          if (d.err) atomicExch(d.err, 1);
          return;
        }
      }
      __syncthreads();
      issue(qd + D);
      {  // density, dn and psi of plane qd
        const unsigned g = issued + qd;
        const T* st = stages + (g % NS) * Sh::stage_elems;
        T* rs = ring + (qd % NR) * NPAD;
        T* ds = dnring + (qd % NR) * NPAD;
#pragma unroll
        for (int s = 0; s < NPER; ++s) {
          if (!valid[s]) continue;
          const int j = tid + s * NT;
          const int jx = j % PX, jy = j / PX;
          const T* row0 = st + jy * XW + jx + kBulkApron - R;
          T v[Q];
#pragma unroll
          for (int i = 0; i < Q; ++i) v[i] = row0[i * PY * XW - cx(i)];
          const T sum = sum19(v);
          ds[j] = sum;
          rs[j] = psi_of<T>(n0 + sum, d.eos);
        }
      }
      __syncthreads();
      const int qc = qd - R;   // plane collided now; its z is z0 + qc - R
      const int k = qc - R;
      if (k >= 0 && active) {
        const unsigned g = issued + qc;
        const T* st = stages + (g % NS) * Sh::stage_elems;
        const int jc = (ty + R) * PX + (tx + R);
        const T* row0 = st + (ty + R) * XW + tx + kBulkApron;
        T gq[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) gq[i] = row0[i * PY * XW - cx(i)];
        const T* planes[2 * R + 1];
#pragma unroll
        for (int dz = -R; dz <= R; ++dz) planes[dz + R] = ring + ((qc + dz) % NR) * NPAD + jc;
        T Fx, Fy, Fz;
        sc_force_pairs<T, ST, PX>(planes, G, Fx, Fy, Fz);
        T dn, jx, jy, jz;
        moments(gq, dn, jx, jy, jz);
        dn = dnring[(qc % NR) * NPAD + jc];   // the same value, formed in the density phase
        const T n = n0 + dn;
        const T inv_n = (T)1 / n;
        const T ux = (jx + (T)0.5 * Fx) * inv_n;
        const T uy = (jy + (T)0.5 * Fy) * inv_n;
        const T uz = (jz + (T)0.5 * Fz) * inv_n;
        collide<T, true, UNIT_TAU>(gq, dn, n, ux, uy, uz, Fx, Fy, Fz, omega);
        const int node = ((z0 + k) * ny + (y0 + ty)) * nx + (x0 + tx);
#pragma unroll
        for (int i = 0; i < Q; ++i) dst[i * plane + node] = (S)gq[i];
      }
    }
    issued += nplanes;
  }
}

}  // namespace lbm
