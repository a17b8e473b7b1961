// Pipelined variant of the fused Shan-Chen step (FP32 / FP64 storage).
//
// Same arithmetic as lattice_kernel (lbm_kernels.cuh), different data
// movement.  The pulled populations of a padded plane (tile + R halo) are
// copied global -> shared with cp.async into one of NS stages, D planes
// ahead of the plane whose density is being formed, so the HBM reads of the
// next planes are in flight while the current plane is collided and stored.
// Stage layout: stage[i][j], j = jy * PX + jx over the padded plane; element
// (i, j) holds f*_i at the pull source of padded node j, i.e. f_i(x_j, t).
//
// Work split: the box is cut into (BX x BY) columns and every column into
// the same z chunks.  Work items (chunk, column) are numbered with the column
// fastest and a persistent grid takes them round-robin, so the CTAs resident
// at any moment work on neighbouring columns at the same z: a halo row one
// CTA reads from HBM is read by its neighbour while it is still in L2.  The
// host picks the chunk length that makes the rounds of the grid fullest.
//
// Per plane (index qd in a segment, planes z0-R .. z0+zc+R-1):
//   wait for this thread's copies of plane qd; barrier
//   issue the copies of plane qd + D       (that stage was last read before the barrier)
//   density + psi of plane qd -> psi ring slot qd % NR; barrier
//   collide the plane with index qd - R (its psi neighbours qd-2R .. qd are ready)
// NS = R + 1 + D population stages and NR = 2R + 1 psi slots.  (A variant that
// collides one plane later needs one barrier per plane but one more stage,
// which halves the CTAs per SM; it measured slower.)
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

template <int P, int ST, int BX, int BY, int D>
struct AsyncShape {
  using T = typename Storage<P>::T;
  static constexpr int R = stencil_radius<ST>();
  static constexpr int PX = BX + 2 * R;
  static constexpr int PY = BY + 2 * R;
  static constexpr int NPAD = PX * PY;
  static constexpr int NT = BX * BY;
  static constexpr int NS = R + 1 + D;     // population stages
  static constexpr int NR = 2 * R + 1;     // psi planes
  static constexpr int NPER = (NPAD + NT - 1) / NT;
  static constexpr size_t stage_elems = (size_t)Q * NPAD;
  static constexpr size_t smem_bytes = sizeof(T) * (NS * stage_elems + NR * NPAD);
};

__device__ __forceinline__ void cp_async_elem4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_elem8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One work item (column col, z chunk starting at z0) of lattice d.
template <int P, int ST, int BX, int BY, int D, bool UNIT_TAU>
__device__ __forceinline__ void async_process_item(const LatticeDesc& d, int zchunk, long long item,
                                                   unsigned char* smem_raw) {
  using Sh = AsyncShape<P, ST, BX, BY, D>;
  using T = typename Sh::T;
  using S = typename Storage<P>::S;
  static_assert(sizeof(S) == sizeof(T), "async path copies stored values unchanged");
  constexpr int R = Sh::R, PX = Sh::PX, NPAD = Sh::NPAD, NT = Sh::NT, NS = Sh::NS, NR = Sh::NR;
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
  // per-population base pointers: each copy and store then needs one 32-bit
  // offset added to a register
  const S* srcp[Q];
  S* dstp[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    srcp[i] = src + i * plane;
    dstp[i] = dst + i * plane;
  }
  {

    const int col = (int)(item % ncols);
    const int z0 = (int)(item / ncols) * zchunk;
    const int zc = min(zchunk, nz - z0);
    const int x0 = (col % tiles_x) * BX, y0 = (col / tiles_x) * BY;
    const int w = min(BX, nx - x0), h = min(BY, ny - y0);
    const bool active = tx < w && ty < h;

    // per padded node of this thread: wrapped source columns / row offsets for
    // c = -1, 0, +1 (offsets inside one population plane fit 32 bits)
    int xs[NPER][3];
    int yrow[NPER][3];
    bool valid[NPER];
#pragma unroll
    for (int s = 0; s < NPER; ++s) {
      const int j = tid + s * NT;
      const int jx = j % PX, jy = j / PX;
      valid[s] = j < NPAD && jx < w + 2 * R && jy < h + 2 * R;
      const int gx = wrap(x0 + jx - R, nx), gy = wrap(y0 + (valid[s] ? jy : 0) - R, ny);
      xs[s][0] = wrap(gx + 1, nx);   // source x for c_x = -1
      xs[s][1] = gx;
      xs[s][2] = wrap(gx - 1, nx);   // source x for c_x = +1
      yrow[s][0] = wrap(gy + 1, ny) * nx;
      yrow[s][1] = gy * nx;
      yrow[s][2] = wrap(gy - 1, ny) * nx;
    }
    const int nplanes = zc + 2 * R;   // planes loaded; plane q is z0 - R + q

    auto issue = [&](int q) {
      if (q < nplanes) {
        const int z = wrap(z0 - R + q, nz);
        const int zo[3] = {wrap(z + 1, nz) * ny * nx, z * ny * nx, wrap(z - 1, nz) * ny * nx};
        T* st = stages + (q % NS) * Sh::stage_elems;
#pragma unroll
        for (int s = 0; s < NPER; ++s) {
          if (!valid[s]) continue;   // whole warps of the last pass skip
          const int j = tid + s * NT;
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const S* g = srcp[i] + (zo[cz(i) + 1] + yrow[s][cy(i) + 1] + xs[s][cx(i) + 1]);
            if (sizeof(T) == 8)
              cp_async_elem8(st + i * NPAD + j, g);
            else
              cp_async_elem4(st + i * NPAD + j, g);
          }
        }
      }
      cp_async_commit();
    };

    __syncthreads();   // the previous segment's readers are done with every stage
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
          T v[Q];
#pragma unroll
          for (int i = 0; i < Q; ++i) v[i] = st[i * NPAD + j];
          rs[j] = psi_of<T>(n0 + sum19(v), d.eos);
        }
      }
      __syncthreads();
      const int qc = qd - R;       // plane collided now; its z is z0 + qc - R
      const int k = qc - R;
      if (k >= 0 && active) {
        const T* st = stages + (qc % NS) * Sh::stage_elems;
        const int jc = (ty + R) * PX + (tx + R);
        T g[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = st[i * NPAD + jc];
        // force from the psi ring: plane qc + dz sits in slot (qc + dz) % NR
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
        const int node = ((z0 + k) * ny + (y0 + ty)) * nx + (x0 + tx);
#pragma unroll
        for (int i = 0; i < Q; ++i) dstp[i][node] = (S)g[i];
      }
    }
    cp_async_wait_all();
  }
}

// CTAs per SM a variant is compiled for: as many as its shared memory admits
// (228 KB per SM, 1 KB reserved per CTA), capped so that no thread is given
// fewer than 64 registers; __launch_bounds__ then caps the registers at
// 65536 / (threads x blocks), so registers never limit residency further.
template <int NT, size_t SMEM>
constexpr int async_min_blocks() {
  constexpr int by_smem = (int)((228u * 1024u) / (SMEM + 1024u));
  constexpr int by_regs = 65536 / (NT * 64);
  return by_smem < 1 ? 1 : (by_smem > by_regs ? by_regs : by_smem);
}

template <int P, int ST, int BX, int BY, int D, bool UNIT_TAU>
__global__ void __launch_bounds__(BX * BY, (async_min_blocks<BX * BY, AsyncShape<P, ST, BX, BY, D>::smem_bytes>()))
lattice_async_kernel(LatticeDesc d, int zchunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  step_grid_enter();
  const int ncols = ((d.nx + BX - 1) / BX) * ((d.ny + BY - 1) / BY);
  const long long items = (long long)ncols * ((d.nz + zchunk - 1) / zchunk);
#pragma unroll 1
  for (long long item = blockIdx.x; item < items; item += gridDim.x)
    async_process_item<P, ST, BX, BY, D, UNIT_TAU>(d, zchunk, item, smem_raw);
}

// A batch of independent lattices advanced by one launch: entry e owns global
// work items [item_begin, item_begin + its items); its current state is in
// d.src when (parity ^ step) is even and in d.dst otherwise.
struct BatchEntry {
  LatticeDesc d;
  long long item_begin;
  int zchunk;
  int parity;
};
struct BatchHeader {
  int n;                 // active entries
  long long total_items;
};

// MIXED_TAU: the batch holds tau = 1 and other lattices; each item then takes
// the collision variant of its own lattice, so every lattice evolves bitwise as
// it would alone.
template <int P, int ST, int BX, int BY, int D, bool MIXED_TAU>
__global__ void __launch_bounds__(BX * BY)
lattice_async_batch_kernel(const BatchEntry* __restrict__ table, const BatchHeader* __restrict__ hdr,
                           int step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  step_grid_enter();
  const int n = hdr->n;
  const long long total = hdr->total_items;
#pragma unroll 1
  for (long long item = blockIdx.x; item < total; item += gridDim.x) {
    int lo = 0, hi = n - 1;          // last entry with item_begin <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (table[mid].item_begin <= item) lo = mid; else hi = mid - 1;
    }
    LatticeDesc d = table[lo].d;
    if ((table[lo].parity ^ step) & 1) {
      const void* t = d.src;
      d.src = d.dst;
      d.dst = const_cast<void*>(t);
    }
    if (!MIXED_TAU || d.omega == 1.0)
      async_process_item<P, ST, BX, BY, D, true>(d, table[lo].zchunk, item - table[lo].item_begin, smem_raw);
    else
      async_process_item<P, ST, BX, BY, D, false>(d, table[lo].zchunk, item - table[lo].item_begin, smem_raw);
  }
}

}  // namespace lbm
