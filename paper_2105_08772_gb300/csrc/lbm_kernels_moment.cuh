// Unit-relaxation-time variant of the pipelined Shan-Chen step (FP32 / FP64).
//
// With tau = 1 the BGK update of Eq. (4) loses its f_i term:
//     f*_i = f_i - (f_i - f_i^eq) + F_i = f_i^eq(n, u) + F_i,
// so a node's post-collision populations depend on its own populations only
// through n and the momentum j = sum_i xi_i f_i (u = (j + F/2)/n, Eq. (7)).
// The collision of plane z therefore needs, from its stage, just four numbers
// per node -- and those can be formed in the same pass that forms the density
// for psi.  The kernel keeps them in registers until psi of plane z + R exists,
// so a population stage is free as soon as its densities are formed: NS = 1 + D
// stages instead of R + 1 + D.  The smaller footprint fits more CTAs per SM, and
// one spare psi plane lets a plane's densities and an earlier plane's collision
// share one barrier.
//
// Copies: the 16-byte row chunks of the chunked kernel (lbm_kernels_chunk.cuh),
// staged in the storage type (FP16 storage: half the shared memory, a 16-byte
// chunk is 8 values, so the apron is 8 and nx % 8 == 0 is needed); or, for
// rows that do not split into chunks (odd or narrow nx; ELEM), the pipelined
// kernel's 4/8-byte element copies of each pulled population straight to its
// padded node, two CTAs per SM so that L1 keeps room for them.
// Thread roles in the density pass: each thread forms its own column's padded
// node (ty + R, tx + R) -- its interior node, whose moments it keeps -- and
// the NPAD - NT nodes of the halo ring are dealt out to the threads (to warps
// that do not copy, where the tile allows it).
// The arithmetic per node is the chunked kernel's (same sums, same collide), so
// fields are bitwise equal to it.
#pragma once

#include "lbm_kernels_chunk.cuh"

namespace lbm {

template <int P, int ST, int BX, int BY, int D, bool ELEM = false>
struct MomentShape {
  using T = typename Storage<P>::T;
  static constexpr int R = stencil_radius<ST>();
  static constexpr int PX = BX + 2 * R;
  static constexpr int PY = BY + 2 * R;
  static constexpr int NPAD = PX * PY;
  static constexpr int NT = BX * BY;
  static constexpr int NH = NPAD - NT;                 // halo ring nodes
  static constexpr int NHPER = (NH + NT - 1) / NT;     // halo nodes per thread
  using S = typename Storage<P>::S;                    // stored (and staged) type
  static constexpr int VE = 16 / (int)sizeof(S);       // elements per 16-byte chunk
  static constexpr int APRON = VE > kChunkApron ? VE : kChunkApron;   // staged left of the tile
  static constexpr int XW = BX + 2 * APRON;
  // staged row pitch: XW, or XW + 4 for FP32 32 x 8 E4 tiles, whose rows 44 floats
  // apart put the halo ring's side columns (read by one warp) on distinct banks
  static constexpr int XWS = (sizeof(S) == 4 && !ELEM && BX == 32 && BY == 8 && R == 1) ? XW + 4 : XW;
  static constexpr int NCH = XW / VE;
  static constexpr int NS = 1 + D;
  static constexpr int NR = 2 * R + 2;                 // psi planes (one spare: one barrier per plane)
  static constexpr int NPER = (NPAD + NT - 1) / NT;   // padded nodes a thread copies (ELEM)
  // ELEM: stage[i][j] holds population i pulled to padded node j (4- or 8-byte
  // element copies, any nx); else staged rows of XW values (16-byte chunks)
  static constexpr size_t stage_elems = ELEM ? (size_t)Q * NPAD : (size_t)Q * PY * XWS;
  static constexpr size_t smem_bytes = sizeof(S) * NS * stage_elems + sizeof(T) * NR * NPAD;
  // ELEM variants run 2 CTAs per SM: the element copies go through L1, which
  // needs the capacity that more CTAs' shared memory would take
  static constexpr int MIN_BLOCKS = ELEM ? 2 : async_min_blocks<NT, smem_bytes>();
  static_assert(R + 1 <= APRON, "apron must cover the pull of the halo");
  static_assert((sizeof(S) * NS * stage_elems) % 16 == 0, "psi ring stays aligned");
};

// a staged (stored) value as an arithmetic value, still scaled by FP16 storage's
// 2^k: the density pass sums the scaled values and scales the sums once, which
// gives bitwise the same sums (a power-of-two factor commutes with rounding)
template <int P>
__device__ __forceinline__ typename Storage<P>::T staged_value(typename Storage<P>::S x) {
  if constexpr (P == kF16) return __half2float(x);
  else return x;
}

// padded index of the h-th node of the halo ring: R full rows on top, R on the
// bottom, then R columns on each side of the BY middle rows
template <int R, int PX, int PY>
__device__ __forceinline__ int halo_node(int h) {
  if (h < R * PX) return h;
  h -= R * PX;
  if (h < R * PX) return (PY - R) * PX + h;
  h -= R * PX;
  const int row = R + h / (2 * R), c = h % (2 * R);
  return row * PX + (c < R ? c : PX - 2 * R + c);
}

// The same ring dealt to four halo warps, for 32-wide tiles with R = 1 and the
// staged rows 44 floats apart: warp 0 reads the top halo row's first 32 nodes,
// warp 1 the bottom row's, warp 2 the 16 side-column nodes (rows 1..8, x = 0 and
// x = 33: 16 distinct banks), warp 3 the four remaining row-end nodes.  Each warp's
// reads of one population hit distinct banks (a row 8 apart is 352 floats, a
// multiple of 32, so the row-end nodes would share banks with the side columns
// if one warp read both).  -1: lane without a node.
template <int BX, int BY, int R>
__device__ __forceinline__ int halo_node_warps(int h) {
  static_assert(BX == 32 && BY == 8 && R == 1, "four-warp halo order is defined for 32 x 8 tiles and R = 1");
  constexpr int PX = BX + 2 * R, PY = BY + 2 * R;
  if (h < 0) return -1;
  if (h < 32) return h;
  if (h < 64) return (PY - 1) * PX + (h - 32);
  if (h < 80) return (1 + (h - 64) / 2) * PX + ((h & 1) ? PX - 1 : 0);
  if (h >= 96 && h < 100) return ((h - 96) < 2 ? 0 : (PY - 1) * PX) + 32 + (h & 1);
  return -1;
}

template <int P, int ST, int BX, int BY, int D, bool ELEM = false>
__device__ __forceinline__ void moment_process_item(const LatticeDesc& d, int zchunk, long long item,
                                                    unsigned char* smem_raw) {
  using Sh = MomentShape<P, ST, BX, BY, D, ELEM>;
  using T = typename Sh::T;
  using S = typename Storage<P>::S;
  constexpr int APRON = Sh::APRON;
  constexpr int R = Sh::R, PX = Sh::PX, PY = Sh::PY, NPAD = Sh::NPAD, NT = Sh::NT, NH = Sh::NH;
  constexpr int NHPER = Sh::NHPER;
  constexpr int XWS = Sh::XWS, VE = Sh::VE, NCH = Sh::NCH, NS = Sh::NS, NR = Sh::NR;
  S* stages = reinterpret_cast<S*>(smem_raw);
  T* ring = reinterpret_cast<T*>(stages + NS * Sh::stage_elems);

  const int nx = d.nx, ny = d.ny, nz = d.nz;
  const long long plane = d.plane;
  const S* __restrict__ src = static_cast<const S*>(d.src);
  S* __restrict__ dst = static_cast<S*>(d.dst);
  const T n0 = dparam<T>(d.n0, d.n0f), G = dparam<T>(d.eos.G, d.eos.Gf);
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
  const int xa = x0 - APRON;
  const T inv_scale = dparam<T>(1.0 / d.scale, d.inv_scalef), scale = dparam<T>(d.scale, d.scalef);

  // Copy positions are the chunked kernel's (one 16-byte chunk of a staged row).
  // Thread roles.  When the copy positions and the halo nodes fit in disjoint
  // whole warps (SPLIT), the first warps copy (one position, all 19 populations)
  // and the last warps form the halo densities, so no warp carries both extra
  // loads to the barrier; otherwise two thread groups split the populations of
  // each position and the halo nodes go to the first threads.
  constexpr int POS = PY * NCH;
  constexpr int POSW = (POS + 31) / 32 * 32;
  constexpr bool HALO4 = !ELEM && BX == 32 && BY == 8 && R == 1 && POSW + 128 <= NT;   // halo_node_warps
  constexpr int NHW = HALO4 ? 128 : (NH + 31) / 32 * 32;
  constexpr bool SPLIT = !ELEM && POSW + NHW <= NT;
  constexpr int NG = SPLIT ? 1 : ((2 * POS <= NT) ? 2 : 1);
  constexpr int NPP = NG == 2 ? 1 : (POS + NT - 1) / NT;
  constexpr int ISPLIT = NG == 2 ? 10 : Q;
  const int grp = NG == 2 ? tid / POS : 0;
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
    prow[pp][0] = wrap(y + 1, ny) * nx;
    prow[pp][1] = y * nx;
    prow[pp][2] = wrap(y - 1, ny) * nx;
    pgx[pp] = wrap(xa + k * VE, nx);
    psm[pp] = jy * XWS + k * VE;
  }
  // ELEM copies (as in the pipelined kernel): padded nodes tid + s NT, their
  // wrapped source columns and row offsets for c = -1, 0, +1
  constexpr int NPER = Sh::NPER;
  int exs[ELEM ? NPER : 1][3], eyr[ELEM ? NPER : 1][3];
  bool ecv[ELEM ? NPER : 1];
  if constexpr (ELEM) {
#pragma unroll
    for (int s = 0; s < NPER; ++s) {
      const int j = tid + s * NT;
      const int jx = j % PX, jy = j / PX;
      ecv[s] = j < NPAD && jx < w + 2 * R && jy < rows;
      const int gx = wrap(x0 + jx - R, nx), gy = wrap(y0 + (ecv[s] ? jy : 0) - R, ny);
      exs[s][0] = wrap(gx + 1, nx);
      exs[s][1] = gx;
      exs[s][2] = wrap(gx - 1, nx);
      eyr[s][0] = wrap(gy + 1, ny) * nx;
      eyr[s][1] = gy * nx;
      eyr[s][2] = wrap(gy - 1, ny) * nx;
    }
  }
  // density-pass nodes: own column's node (padded (ty + R, tx + R)) and halo ring nodes
  const int j0 = (ty + R) * PX + (tx + R);
  const bool valid0 = tx < w + R && ty < h + R;
  int jh[NHPER];
  bool validh[NHPER];
#pragma unroll
  for (int s = 0; s < NHPER; ++s) {
    const int hh = SPLIT ? (s == 0 ? tid - (NT - NHW) : -1) : tid + s * NT;
    bool mine;
    if constexpr (HALO4) {   // bank-conflict-free halo warps
      const int node = halo_node_warps<BX, BY, R>(hh);
      mine = node >= 0;
      jh[s] = mine ? node : 0;
    } else {
      mine = hh >= 0 && hh < NH;
      jh[s] = mine ? halo_node<R, PX, PY>(hh) : 0;
    }
    validh[s] = mine && (jh[s] % PX) < w + 2 * R && (jh[s] / PX) < rows;
  }
  const int nplanes = zc + 2 * R;

  auto issue = [&](int q) {
    if (q < nplanes) {
      const int z = wrap(z0 - R + q, nz);
      const int zo[3] = {wrap(z + 1, nz) * ny * nx, z * ny * nx, wrap(z - 1, nz) * ny * nx};
      S* st = stages + (q % NS) * Sh::stage_elems;
      if constexpr (ELEM) {
#pragma unroll
        for (int s = 0; s < NPER; ++s) {
          if (!ecv[s]) continue;
          const int j = tid + s * NT;
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const S* gsrc = srcp[i] + (zo[cz(i) + 1] + eyr[s][cy(i) + 1] + exs[s][cx(i) + 1]);
            if constexpr (sizeof(S) == 8) cp_async_elem8(st + i * NPAD + j, gsrc);
            else cp_async_elem4(st + i * NPAD + j, gsrc);
          }
        }
      } else {
#pragma unroll
      for (int pp = 0; pp < NPP; ++pp) {
        if (!pok[pp]) continue;
        if (grp == 0) {
#pragma unroll
          for (int i = 0; i < ISPLIT; ++i)
            cp_async_chunk16(st + i * PY * XWS + psm[pp],
                             srcp[i] + (zo[cz(i) + 1] + prow[pp][cy(i) + 1] + pgx[pp]));
        } else if (NG == 2) {
#pragma unroll
          for (int i = ISPLIT; i < Q; ++i)
            cp_async_chunk16(st + i * PY * XWS + psm[pp],
                             srcp[i] + (zo[cz(i) + 1] + prow[pp][cy(i) + 1] + pgx[pp]));
        }
      }
      }
    }
    cp_async_commit();
  };

  // moments of the own interior node for the last R + 1 planes: m[0] newest
  T mdn[R + 1], mjx[R + 1], mjy[R + 1], mjz[R + 1];
#pragma unroll
  for (int r = 0; r <= R; ++r) mdn[r] = mjx[r] = mjy[r] = mjz[r] = (T)0;
  // psi of the own interior node for the last 2R + 1 planes: pz[2R] newest; at
  // the collision of plane qc, pz[dz + R] is plane qc + dz (the force's own
  // column and centre, kept in registers)
  T pz[2 * R + 1];
#pragma unroll
  for (int r = 0; r <= 2 * R; ++r) pz[r] = (T)0;

  __syncthreads();   // the previous item's readers are done with every stage and psi plane
#pragma unroll 1
  for (int q = 0; q < D; ++q) issue(q);

  // One barrier per plane.  Iteration qd collides plane qc = qd - 1 - R, whose psi
  // neighbours qc - R .. qc + R = qd - 1 were all formed before this iteration's
  // barrier, and then forms the densities of plane qd.  The density pass writes
  // psi slot qd % (2R + 2), which none of those 2R + 1 planes occupies; the stage
  // it reads is not the one issue() refills (that held plane qd - 1, read before
  // the barrier).  The collision goes first so that the warps' shared-memory load
  // bursts (density pass) and arithmetic (collision) overlap across warps.  One
  // extra iteration collides the last plane.
#pragma unroll 1
  for (int qd = 0; qd <= nplanes; ++qd) {
    cp_async_wait<D - 1>();
    __syncthreads();
    issue(qd + D);
    const int qc = qd - 1 - R;
    const int k = qc - R;
    if (k >= 0 && active) {
      const T* planes[2 * R + 1];
#pragma unroll
      for (int dz = -R; dz <= R; ++dz) planes[dz + R] = ring + ((qc + dz) % NR) * NPAD + j0;
      T Fx, Fy, Fz;
      sc_force_pairs<T, ST, PX, true>(planes, G, Fx, Fy, Fz, pz);
      const T dn = mdn[R];       // plane qc = qd - 1 - R: R planes before the newest
      const T n = n0 + dn;
      const T inv_n = (T)1 / n;
      const T ux = (mjx[R] + (T)0.5 * Fx) * inv_n;
      const T uy = (mjy[R] + (T)0.5 * Fy) * inv_n;
      const T uz = (mjz[R] + (T)0.5 * Fz) * inv_n;
      T g[Q];     // written, never read, by the unit-tau collision
      // FP16: the collision returns the populations times the storage scale
      collide<T, true, true, P == kF16>(g, dn, n, ux, uy, uz, Fx, Fy, Fz, (T)1, scale);
      const long long node = ((long long)(z0 + k) * ny + (y0 + ty)) * nx + (x0 + tx);
      S* q = dst + node;   // population i's plane is i * plane further on
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if constexpr (P == kF16) *q = __float2half_rn(g[i]);   // already scaled
        else Storage<P>::store(q, g[i], scale);
        q += plane;
      }
    }
#pragma unroll
    for (int r = R; r > 0; --r) {
      mdn[r] = mdn[r - 1];
      mjx[r] = mjx[r - 1];
      mjy[r] = mjy[r - 1];
      mjz[r] = mjz[r - 1];
    }
#pragma unroll
    for (int r = 0; r < 2 * R; ++r) pz[r] = pz[r + 1];
    if (qd < nplanes) {  // densities, psi and own moments of plane qd
      const S* st = stages + (qd % NS) * Sh::stage_elems;
      T* rs = ring + (qd % NR) * NPAD;
      if (valid0) {
        T v[Q];
        if constexpr (ELEM) {
#pragma unroll
          for (int i = 0; i < Q; ++i) v[i] = staged_value<P>(st[i * NPAD + j0]);
        } else {
          const S* row0 = st + (ty + R) * XWS + tx + APRON;
#pragma unroll
          for (int i = 0; i < Q; ++i) v[i] = staged_value<P>(row0[i * PY * XWS - cx(i)]);
        }
        T dn, jx, jy, jz;
        moments(v, dn, jx, jy, jz);
        if constexpr (P == kF16) {
          dn *= inv_scale;
          jx *= inv_scale;
          jy *= inv_scale;
          jz *= inv_scale;
        }
        const T p = psi_of<T>(n0 + dn, d.eos);
        rs[j0] = p;
        pz[2 * R] = p;
        mdn[0] = dn;
        mjx[0] = jx;
        mjy[0] = jy;
        mjz[0] = jz;
      }
#pragma unroll
      for (int s = 0; s < NHPER; ++s) {
        if (!validh[s]) continue;
        T v[Q];
        if constexpr (ELEM) {
#pragma unroll
          for (int i = 0; i < Q; ++i) v[i] = staged_value<P>(st[i * NPAD + jh[s]]);
        } else {
          const int hx = jh[s] % PX, hy = jh[s] / PX;
          const S* row0 = st + hy * XWS + hx + APRON - R;
#pragma unroll
          for (int i = 0; i < Q; ++i) v[i] = staged_value<P>(row0[i * PY * XWS - cx(i)]);
        }
        rs[jh[s]] = psi_of<T>(n0 + (P == kF16 ? sum19(v) * inv_scale : sum19(v)), d.eos);
      }
    }
  }
  cp_async_wait_all();
}

template <int P, int ST, int BX, int BY, int D, bool ELEM = false>
__global__ void __launch_bounds__(BX * BY, (MomentShape<P, ST, BX, BY, D, ELEM>::MIN_BLOCKS))
lattice_moment_kernel(LatticeDesc d, int zchunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  step_grid_enter();
  const int ncols = ((d.nx + BX - 1) / BX) * ((d.ny + BY - 1) / BY);
  const long long items = (long long)ncols * ((d.nz + zchunk - 1) / zchunk);
#pragma unroll 1
  for (long long item = blockIdx.x; item < items; item += gridDim.x)
    moment_process_item<P, ST, BX, BY, D, ELEM>(d, zchunk, item, smem_raw);
}

// A batch of tau = 1 lattices (see lattice_async_batch_kernel for the table):
// every lattice takes the moment kernel's path.
template <int P, int ST, int BX, int BY, int D, bool ELEM = false>
__global__ void __launch_bounds__(BX * BY, (MomentShape<P, ST, BX, BY, D, ELEM>::MIN_BLOCKS))
lattice_moment_batch_kernel(const BatchEntry* __restrict__ table, const BatchHeader* __restrict__ hdr,
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
    moment_process_item<P, ST, BX, BY, D, ELEM>(d, table[lo].zchunk, item - table[lo].item_begin, smem_raw);
  }
}

}  // namespace lbm
