// Unit-tau moment kernel fed by TMA tensor-tile copies (FP32 storage, kind 7).
//
// The arithmetic is the moment kernel's (lbm_kernels_moment.cuh): at tau = 1 the
// post-collision populations depend on a node's own populations only through n
// and j, so a plane's stage is free once its densities are formed, and the
// fields are bitwise those of kinds 4-6.  What differs is how the pulled
// populations reach shared memory.  Instead of threads issuing 16-byte cp.async
// chunks (an address computation and an L1 request per chunk), lane i of warp 0
// issues one cp.async.bulk.tensor box per population i and plane: XW x PY floats
// of a 4-D tensor map over the population buffer (x, y, z, i), rows
// y0 - R - c_y(i) ... of plane z - c_z(i), columns [x0 - APRON, x0 - APRON + XW).
// The boxes complete on one mbarrier per stage (expect_tx of the stage's bytes)
// and every thread waits on the stage's phase.  Stage row j of population i then
// holds source row y0 - R - c_y(i) + j; the pull shift in x is an index offset.
//
// Periodic wrap.  A tensor box reads the fill value (zero) outside the tensor;
// the lattice is periodic.  Every box starts on a 128-byte shared-memory boundary,
// so a box cannot be split at an arbitrary staged row; instead:
//  * y: for the first and last row of tiles the rows beyond the box's range
//    (R + c_y(i) above, R - c_y(i) below, per population) are copied by extra
//    boxes of those heights, from their periodic images, into a small buffer
//    (one 128-byte aligned slot per population); after the stage's mbarrier
//    completes, threads copy them (16-byte chunks whose x lies in [0, nx)) over
//    the zero-filled stage rows;
//  * x: for the first and last tile column the cells outside [0, nx) that the
//    density pass reads (R + c_x(i) left, R - c_x(i) right per population and
//    staged row) are loaded by threads from their periodic images one plane
//    ahead into registers and stored into the stage after the mbarrier wait.
// The two kinds of fix-up write disjoint cells (x inside vs outside [0, nx)), both
// before the barrier that precedes the density pass; the writers then fence their
// generic writes against the next asynchronous copy into the same stage.
//
// Requirements (host-checked): nx % 4 == 0 (16-byte rows and box origins),
// nx >= 64 (no tile column wraps on both sides), ny % BY == 0 and ny >= 2 BY (no
// ragged tile rows; a tile wraps at most one way in y), and the tensor maps.
//
// Bounded waits: every mbarrier wait gives up after kTmaPolls polls; the barrier
// that follows is a __syncthreads_or on the give-up flag, so the whole CTA sees it
// at once: it sets *d.err, waits (again bounded) for its copies in flight and
// leaves the kernel.
//
// Shared memory: NS = 2 stages of Q population regions (PY rows of XW = BX + 8
// floats, each region padded to a 128-byte multiple), the psi ring of 2R + 2
// padded planes, the wrapped-row buffer, two mbarriers: 72.9 KB for 32 x 8 E4
// tiles, three CTAs per SM.
#pragma once

#include <cuda.h>

#include "lbm_kernels_moment.cuh"

namespace lbm {

constexpr int kTmaPolls = 1 << 20;   // bound of every mbarrier wait (about a second)

// tensor maps of one population buffer: map[0] is the XW x PY box, map[k] the
// XW x k box of k wrapped rows (k = 1 .. R + 1), map[R + 2] the 4 x PY box of an
// x apron (16 bytes of each staged row); passed by value as a __grid_constant__
// kernel parameter
struct TmaMapSet {
  CUtensorMap map[kMaxTmaMaps];
};

__host__ __device__ constexpr int tma_align128(int bytes) { return (bytes + 127) / 128 * 128; }

// Periodic wrap, counted per population i (R = 1 for the kernel below):
//  * wrapped rows of a tile at the top (yside = +1: R + c_y rows above the box)
//    or the bottom (yside = -1: R - c_y rows below it);
//  * x-wrapped cells per staged row of a tile at the left (xside = +1: R + c_x
//    cells left of x = 0) or the right (xside = -1: R - c_x cells right of nx - 1).
// Each side's list (wrapped rows of a tile, x cells of one staged row) has 19 R
// entries, population by population; the lists are packed into 64-bit constants
// (6 bits an entry: population << 1 | index) so that a thread decodes its entry
// with a shift and a mask, without a table in memory.
__host__ __device__ constexpr int tma_wrap_rows(int R, int side, int i) {
  return R + side * cy_rt(i) > 0 ? R + side * cy_rt(i) : 0;
}
__host__ __device__ constexpr int tma_wrap_cols(int R, int side, int i) {
  return R + side * cx_rt(i) > 0 ? R + side * cx_rt(i) : 0;
}
// entry j of a side's list (rows if `rows`, else columns), population << 1 | index
__host__ __device__ constexpr int tma_list_entry(bool rows, int side, int j) {
  int n = 0;
  for (int i = 0; i < Q; ++i) {
    const int c = rows ? tma_wrap_rows(1, side, i) : tma_wrap_cols(1, side, i);
    for (int m = 0; m < c; ++m, ++n)
      if (n == j) return (i << 1) | m;
  }
  return 0;
}
// ten 6-bit entries j0 .. j0 + 9 of a list in one constant
__host__ __device__ constexpr unsigned long long tma_list_pack(bool rows, int side, int j0) {
  unsigned long long v = 0;
  for (int k = 0; k < 10; ++k) v |= (unsigned long long)tma_list_entry(rows, side, j0 + k) << (6 * k);
  return v;
}
// entry j (0 <= j < 19) of a side's list, decoded from the packed constants
__device__ __forceinline__ int tma_list(bool rows, int side, int j) {
  constexpr unsigned long long r0p = tma_list_pack(true, 1, 0), r1p = tma_list_pack(true, 1, 10);
  constexpr unsigned long long r0m = tma_list_pack(true, -1, 0), r1m = tma_list_pack(true, -1, 10);
  constexpr unsigned long long c0p = tma_list_pack(false, 1, 0), c1p = tma_list_pack(false, 1, 10);
  constexpr unsigned long long c0m = tma_list_pack(false, -1, 0), c1m = tma_list_pack(false, -1, 10);
  const unsigned long long t = rows ? (side > 0 ? (j < 10 ? r0p : r1p) : (j < 10 ? r0m : r1m))
                                    : (side > 0 ? (j < 10 ? c0p : c1p) : (j < 10 ? c0m : c1m));
  return (int)((t >> (6 * (j < 10 ? j : j - 10))) & 63ull);
}
// byte offset of population i's slot in the wrapped-row buffer
__host__ __device__ constexpr int tma_wrap_offset(int R, int XW, int side, int i) {
  int off = 0;
  for (int j = 0; j < i; ++j) off += tma_align128(tma_wrap_rows(R, side, j) * XW * 4);
  return off;
}
__host__ __device__ constexpr unsigned long long tma_wrap_slots_pack(int XW, int side, int i0) {
  unsigned long long v = 0;
  for (int k = 0; k < 10 && i0 + k < Q; ++k)
    v |= (unsigned long long)(tma_wrap_offset(1, XW, side, i0 + k) / 128) << (6 * k);
  return v;
}
template <int XW>
__device__ __forceinline__ int tma_wrap_slot_bytes(int side, int i) {
  constexpr unsigned long long p0 = tma_wrap_slots_pack(XW, 1, 0), p1 = tma_wrap_slots_pack(XW, 1, 10);
  constexpr unsigned long long m0 = tma_wrap_slots_pack(XW, -1, 0), m1 = tma_wrap_slots_pack(XW, -1, 10);
  const unsigned long long t = side > 0 ? (i < 10 ? p0 : p1) : (i < 10 ? m0 : m1);
  return 128 * (int)((t >> (6 * (i < 10 ? i : i - 10))) & 63ull);
}
__host__ __device__ constexpr int tma_wrap_bytes(int R, int XW) {
  const int a = tma_wrap_offset(R, XW, 1, Q), b = tma_wrap_offset(R, XW, -1, Q);
  return a > b ? a : b;
}
// populations with x-wrapped cells on a side, as a bit mask; the x-apron slot of
// population i is the number of such populations before it
__host__ __device__ constexpr unsigned tma_xpops(int R, int side) {
  unsigned m = 0;
  for (int i = 0; i < Q; ++i)
    if (tma_wrap_cols(R, side, i) > 0) m |= 1u << i;
  return m;
}
__host__ __device__ constexpr int tma_popcount(unsigned m) {
  int n = 0;
  for (; m; m &= m - 1) ++n;
  return n;
}
// cells both x- and y-wrapped (corner tiles): wrap rows x wrap columns per
// population; entry t of the list is population << 2 | row index << 1 | column index
__host__ __device__ constexpr int tma_corner_entry(int xside, int yside, int t) {
  int n = 0;
  for (int i = 0; i < Q; ++i)
    for (int v = 0; v < tma_wrap_rows(1, yside, i); ++v)
      for (int m = 0; m < tma_wrap_cols(1, xside, i); ++m, ++n)
        if (n == t) return (i << 2) | (v << 1) | m;
  return 0;
}
__host__ __device__ constexpr int tma_corner_count(int xside, int yside) {
  int n = 0;
  for (int i = 0; i < Q; ++i) n += tma_wrap_rows(1, yside, i) * tma_wrap_cols(1, xside, i);
  return n;
}
// nine 7-bit corner entries t0 .. t0 + 8 in one constant
__host__ __device__ constexpr unsigned long long tma_corner_pack(int xside, int yside, int t0) {
  unsigned long long v = 0;
  for (int k = 0; k < 9; ++k) v |= (unsigned long long)tma_corner_entry(xside, yside, t0 + k) << (7 * k);
  return v;
}
template <int XS, int YS>
__device__ __forceinline__ unsigned long long tma_corner_word(int w) {
  constexpr unsigned long long a = tma_corner_pack(XS, YS, 0), b = tma_corner_pack(XS, YS, 9),
                               c = tma_corner_pack(XS, YS, 18);
  return w == 0 ? a : (w == 1 ? b : c);
}
__device__ __forceinline__ int tma_corner(int xside, int yside, int t) {
  const int w = t / 9, k = t % 9;
  const unsigned long long v = xside > 0 ? (yside > 0 ? tma_corner_word<1, 1>(w) : tma_corner_word<1, -1>(w))
                                         : (yside > 0 ? tma_corner_word<-1, 1>(w) : tma_corner_word<-1, -1>(w));
  return (int)((v >> (7 * k)) & 127ull);
}

template <int ST, int BX, int BY>
struct TmaShape {
  static constexpr int R = stencil_radius<ST>();
  static constexpr int PX = BX + 2 * R;
  static constexpr int PY = BY + 2 * R;
  static constexpr int NPAD = PX * PY;
  static constexpr int NT = BX * BY;
  static constexpr int NH = NPAD - NT;
  static constexpr int NHPER = (NH + NT - 1) / NT;
  static constexpr int APRON = 4;                  // one 16-byte FP32 chunk left of the tile
  static constexpr int XW = BX + 8;                // box width
  static constexpr int POP = (PY * XW + 31) / 32 * 32;   // population region: 128-byte multiple
  static constexpr int NS = 2;
  static constexpr int NR = 2 * R + 2;
  static constexpr int NMAPS = R + 3;
  static constexpr int LIST = Q * R;               // wrapped rows of a tile, x cells of a staged row
  static constexpr int XPOPS = tma_popcount(tma_xpops(R, 1));   // populations with an x apron
  static constexpr int XBOX = 4 * PY * 4;                      // bytes of one x-apron box
  static constexpr int XSLOT = tma_align128(XBOX);               // its slot (the tail holds corner values)
  static constexpr int NCORNER = tma_corner_count(1, 1);
  static constexpr size_t stage_elems = (size_t)Q * POP;
  static constexpr size_t ring_off = sizeof(float) * NS * stage_elems;
  static constexpr size_t wrap_off = (ring_off + sizeof(float) * NR * NPAD + 127) / 128 * 128;
  static constexpr size_t xa_off = wrap_off + tma_wrap_bytes(R, XW);
  static constexpr size_t bar_off = xa_off + (size_t)XPOPS * XSLOT;
  static constexpr size_t smem_bytes = bar_off + 8 * NS + 128;   // + 128: the base is aligned at run time
  static constexpr int MIN_BLOCKS = 3;
  static_assert(R == 1, "the packed wrap lists are written for R = 1 (E4)");
  static_assert(XW % 4 == 0 && XW >= APRON + BX + R + 1, "box covers the pull of the halo");
  static_assert(APRON >= R + 1, "apron covers the pull of the halo");
  static_assert(NMAPS <= kMaxTmaMaps, "tensor maps per buffer");
  static_assert((sizeof(float) * stage_elems) % 128 == 0, "stages on 128-byte boundaries");
  static_assert(LIST * (XW / 4) <= NT && PY * LIST <= NT && NCORNER <= NT && NCORNER <= 27,
                "one fix-up of each kind per thread");
  static_assert(XPOPS == tma_popcount(tma_xpops(R, -1)), "both x sides have as many apron boxes");
  static_assert(XPOPS >= 2 && XSLOT - XBOX >= 4 * NCORNER, "corner buffers fit the slot tails");
  static_assert(NCORNER == tma_corner_count(-1, 1) && NCORNER == tma_corner_count(1, -1) &&
                    NCORNER == tma_corner_count(-1, -1), "corners alike");
};

__device__ __forceinline__ unsigned tma_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(tma_smem(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void tma_mbar_expect(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tma_smem(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool tma_mbar_try(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(tma_smem(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// one box of a 4-D tensor map (x, y, z, population) into shared memory
__device__ __forceinline__ void tma_load_box(void* dst, const CUtensorMap* m, int x, int y, int z, int i,
                                             unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];\n" ::"r"(tma_smem(dst)),
      "l"((unsigned long long)m), "r"(x), "r"(y), "r"(z), "r"(i), "r"(tma_smem(bar))
      : "memory");
}
__device__ __forceinline__ void tma_fence_generic_to_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Wait for the phase of `bar` with parity `par`; false if kTmaPolls polls passed.
__device__ __forceinline__ bool tma_wait(unsigned long long* bar, unsigned par) {
  for (int k = 0; k < kTmaPolls; ++k)
    if (tma_mbar_try(bar, par)) return true;
  return false;
}

// One work item (column, z chunk).  Returns false when a wait gave up.
// The halo ring in warp-row order, for 32-wide tiles with R = 1: the first 32
// nodes of the top halo row, the first 32 of the bottom row, the two remaining
// nodes of each, then the side columns row by row (each of the first two warps
// reads one contiguous row).
template <int BX, int BY, int R>
__device__ __forceinline__ int tma_halo_node_rows(int h) {
  static_assert(BX == 32 && R == 1, "warp-row order is defined for 32-wide tiles and R = 1");
  constexpr int PX = BX + 2 * R, PY = BY + 2 * R;
  if (h < 32) return h;
  h -= 32;
  if (h < 32) return (PY - 1) * PX + h;
  h -= 32;
  if (h < PX - 32) return 32 + h;
  h -= PX - 32;
  if (h < PX - 32) return (PY - 1) * PX + 32 + h;
  h -= PX - 32;
  const int row = 1 + h / 2, c = h % 2;
  return row * PX + (c == 0 ? 0 : PX - 1);
}

template <int ST, int BX, int BY>
__device__ __forceinline__ bool tma_process_item(const LatticeDesc& d, const TmaMapSet& maps, int zchunk,
                                                 long long item, unsigned char* smem, unsigned& phase_bits) {
  using Sh = TmaShape<ST, BX, BY>;
  using T = float;
  constexpr int R = Sh::R, PX = Sh::PX, PY = Sh::PY, NPAD = Sh::NPAD, NT = Sh::NT, NH = Sh::NH;
  constexpr int NHPER = Sh::NHPER, APRON = Sh::APRON, XW = Sh::XW, POP = Sh::POP, NS = Sh::NS,
                NR = Sh::NR;
  constexpr int XC = XW / 4;   // 16-byte chunks per staged row
  float* stages = reinterpret_cast<float*>(smem);
  T* ring = reinterpret_cast<T*>(smem + Sh::ring_off);
  unsigned char* wbuf = smem + Sh::wrap_off;
  unsigned char* xbuf = smem + Sh::xa_off;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + Sh::bar_off);

  const int nx = d.nx, ny = d.ny, nz = d.nz;
  const long long plane = d.plane;
  const float* __restrict__ src = static_cast<const float*>(d.src);
  float* __restrict__ dst = static_cast<float*>(d.dst);
  const T n0 = dparam<T>(d.n0, d.n0f), G = dparam<T>(d.eos.G, d.eos.Gf);
  const int tiles_x = (nx + BX - 1) / BX;
  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int ncols = tiles_x * (ny / BY);

  const int col = (int)(item % ncols);
  const int z0 = (int)(item / ncols) * zchunk;
  const int zc = min(zchunk, nz - z0);
  const int x0 = (col % tiles_x) * BX, y0 = (col / tiles_x) * BY;
  const int w = min(BX, nx - x0);
  const bool active = tx < w;
  const int nplanes = zc + 2 * R;

  // density-pass nodes: own column (padded (ty + R, tx + R)) and the halo ring,
  // dealt to the last warps (warp-row order for 32 x 8 E4 tiles)
  const int j0 = (ty + R) * PX + (tx + R);
  const bool valid0 = tx < w + R;
  constexpr int NHW = (NH + 31) / 32 * 32;
  int jh[NHPER];
  bool validh[NHPER];
#pragma unroll
  for (int s = 0; s < NHPER; ++s) {
    const int hh = NHW <= NT ? (s == 0 ? tid - (NT - NHW) : -1) : tid + s * NT;
    const bool mine = hh >= 0 && hh < NH;
    int j = 0;
    if (mine) {
      if constexpr (BX == 32 && BY == 8 && R == 1) j = tma_halo_node_rows<BX, BY, R>(hh);
      else j = halo_node<R, PX, PY>(hh);
    }
    jh[s] = j;
    validh[s] = mine && (j % PX) < w + 2 * R;
  }

  // Periodic wrap of this item (see the file comment): y for the first (yside +1)
  // or last (-1) row of tiles, x for the first (xside +1) or last (-1) column.
  const int yside = y0 == 0 ? 1 : (y0 + BY == ny ? -1 : 0);
  const int xside = x0 < R + 1 ? 1 : (x0 + w + R + 1 > nx ? -1 : 0);
  // x-apron slot of population i on this item's x side
  auto xslot = [&](int i) {
    constexpr unsigned left = tma_xpops(R, 1), right = tma_xpops(R, -1);
    return Sh::XSLOT * __popc((xside > 0 ? left : right) & ((1u << i) - 1u));
  };

  // corner cells (x- and y-wrapped; 19 per plane of a corner tile): thread t < 19
  // copies its cell's periodic image two planes ahead of its use, with a 4-byte
  // cp.async, into one of two 19-float buffers kept in the unused tails of the
  // first two x-apron slots (even and odd planes); it waits for that copy group
  // before storing the value into the stage.  (One plane ahead, in a register,
  // the copy's latency stalled the corner tiles and with them the whole grid.)
  const bool corner = xside != 0 && yside != 0 && tid < Sh::NCORNER;
  auto corner_cell = [&](int& pop, int& yx) {   // staged index, population, periodic image
    const int e = tma_corner(xside, yside, tid);
    pop = e >> 2;
    const int v = (e >> 1) & 1, m = e & 1;
    const int k = tma_wrap_rows(R, yside, pop);
    const int r = yside > 0 ? v : PY - k + v;                               // staged row
    const int c = xside > 0 ? APRON - R - cx_rt(pop) + m : APRON + w + m;   // staged column
    yx = wrap(y0 - R - cy_rt(pop) + r, ny) * nx + wrap(x0 - APRON + c, nx);
    return pop * POP + r * XW + c;
  };
  auto corner_buf = [&](int q) {
    return reinterpret_cast<float*>(xbuf + (q & 1) * Sh::XSLOT + Sh::XBOX);
  };
  auto corner_load = [&](int q) {   // one cp.async group per plane slot, possibly empty
    if (!corner) return;
    if (q < nplanes) {
      int pop, yx;
      corner_cell(pop, yx);
      const int zs = wrap(wrap(z0 - R + q, nz) - cz_rt(pop), nz);
      cp_async_elem4(corner_buf(q) + tid, src + (long long)pop * plane + (long long)zs * ny * nx + yx);
    }
    cp_async_commit();
  };

  // TMA copies of plane q into stage q % NS, the wrapped rows into their buffer and
  // the x aprons into theirs: lane i of warp 0 copies population i
  auto issue = [&](int q) {
    if (q >= nplanes || tid >= 32) return;
    const int s = q % NS;
    unsigned long long* bar = bars + s;
    if (tid == 0)
      tma_mbar_expect(bar, (unsigned)(sizeof(float) * (XW * (Q * PY + (yside != 0 ? Sh::LIST : 0)) +
                                                        (xside != 0 ? 4 * PY * Sh::XPOPS : 0))));
    __syncwarp();
    if (tid < Q) {
      const int i = tid;
      const int z = wrap(z0 - R + q, nz);
      const int zs = wrap(z - cz_rt(i), nz);
      const int xb = x0 - APRON, yb = y0 - R - cy_rt(i);
      tma_load_box(stages + s * Sh::stage_elems + i * POP, &maps.map[0], xb, yb, zs, i, bar);
      if (yside != 0) {
        const int k = tma_wrap_rows(R, yside, i);
        if (k > 0)
          tma_load_box(wbuf + tma_wrap_slot_bytes<XW>(yside, i), &maps.map[k], xb, yside > 0 ? ny - k : 0, zs,
                       i, bar);
      }
      if (xside != 0 && tma_wrap_cols(R, xside, i) > 0)
        tma_load_box(xbuf + xslot(i), &maps.map[R + 2],
                     xside > 0 ? nx - 4 : 0, yb, zs, i, bar);
    }
  };

  // After a stage's copies have landed: the wrapped rows (16-byte chunks inside
  // [0, nx)) and the x-apron cells of unwrapped rows go from their buffers into the
  // stage; corner cells come from registers.  The three sets of cells are disjoint.
  auto fix_stage = [&](float* st, int q) {
    bool wrote = false;
    if (yside != 0 && tid < Sh::LIST * XC) {
      const int rho = tid / XC, c4 = tid % XC;
      const int e = tma_list(true, yside, rho);
      const int pop = e >> 1, v = e & 1;
      const int xs = x0 - APRON + 4 * c4;
      if (xs >= 0 && xs + 4 <= nx) {
        const int k = tma_wrap_rows(R, yside, pop);
        *reinterpret_cast<float4*>(st + pop * POP + (yside > 0 ? v : PY - k + v) * XW + 4 * c4) =
            *reinterpret_cast<const float4*>(
                reinterpret_cast<const float*>(wbuf + tma_wrap_slot_bytes<XW>(yside, pop)) + v * XW + 4 * c4);
        wrote = true;
      }
    }
    if (xside != 0 && tid < PY * Sh::LIST) {
      const int r = tid / Sh::LIST, j = tid % Sh::LIST;
      const int e = tma_list(false, xside, j);
      const int pop = e >> 1, m = e & 1;
      const int k = yside != 0 ? tma_wrap_rows(R, yside, pop) : 0;
      const bool row_wrapped = yside > 0 ? r < k : (yside < 0 ? r >= PY - k : false);
      if (!row_wrapped) {
        const int c = xside > 0 ? APRON - R - cx_rt(pop) + m : APRON + w + m;   // staged column
        const int bc = xside > 0 ? c : m;                                       // column in the box
        st[pop * POP + r * XW + c] =
            reinterpret_cast<const float*>(xbuf + xslot(pop))[r * 4 + bc];
        wrote = true;
      }
    }
    if (corner) {
      cp_async_wait<1>();   // this thread's copy of plane q (the copy of q + 1 may still be in flight)
      int pop, yx;
      st[corner_cell(pop, yx)] = corner_buf(q)[tid];
      wrote = true;
    }
    if (wrote) tma_fence_generic_to_async();
  };

  T mdn[R + 1], mjx[R + 1], mjy[R + 1], mjz[R + 1];
#pragma unroll
  for (int r = 0; r <= R; ++r) mdn[r] = mjx[r] = mjy[r] = mjz[r] = (T)0;
  T pz[2 * R + 1];
#pragma unroll
  for (int r = 0; r <= 2 * R; ++r) pz[r] = (T)0;

  // the previous item's readers are done with every stage, psi plane and the
  // wrapped-row buffer
  __syncthreads();
  issue(0);
  corner_load(0);
  corner_load(1);

  // One barrier per plane (the moment kernel's schedule).  Iteration qd waits for
  // plane qd's copies, writes its fix-ups, passes the barrier, issues plane qd + 1
  // (into the stage last read in iteration qd - 1; the wrapped-row buffer was read
  // before the barrier), collides plane qd - 1 - R and forms plane qd's densities.
  // one plane; false when a wait gave up
  auto plane_step = [&](int qd) -> bool {
    bool gave_up = false;
    if (qd < nplanes) {
      const int s = qd % NS;
      const unsigned par = (phase_bits >> s) & 1u;
      gave_up = !tma_wait(bars + s, par);
      phase_bits ^= 1u << s;
      if (xside != 0 || yside != 0) fix_stage(stages + s * Sh::stage_elems, qd);
    }
    if (__syncthreads_or(gave_up)) {
      // a copy never completed: flag it, wait (bounded) once more for the copies
      // in flight, leave every remaining item
      if (tid == 0 && d.err) atomicExch(d.err, 1);
      const int s = qd % NS;
      tma_wait(bars + s, ((phase_bits >> s) & 1u) ^ 1u);
      return false;
    }
    issue(qd + 1);
    corner_load(qd + 2);
    const int qc = qd - 1 - R;
    const int k = qc - R;
    if (k >= 0 && active) {
      const T* planes[2 * R + 1];
#pragma unroll
      for (int dz = -R; dz <= R; ++dz) planes[dz + R] = ring + ((qc + dz) % NR) * NPAD + j0;
      T Fx, Fy, Fz;
      sc_force_pairs<T, ST, PX, true>(planes, G, Fx, Fy, Fz, pz);
      const T dn = mdn[R];
      const T n = n0 + dn;
      const T inv_n = (T)1 / n;
      const T ux = (mjx[R] + (T)0.5 * Fx) * inv_n;
      const T uy = (mjy[R] + (T)0.5 * Fy) * inv_n;
      const T uz = (mjz[R] + (T)0.5 * Fz) * inv_n;
      float* out = dst + (((long long)(z0 + k) * ny + (y0 + ty)) * nx + (x0 + tx));
      collide_unit_tau_store<T>(dn, n, ux, uy, uz, Fx, Fy, Fz,
                                [&](int i, T v) { out[i * plane] = v; });
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
    if (qd < nplanes) {
      const float* st = stages + (qd % NS) * Sh::stage_elems;
      T* rs = ring + (qd % NR) * NPAD;
      if (valid0) {
        T v[Q];
        const float* row0 = st + (ty + R) * XW + tx + APRON;
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = row0[i * POP - cx(i)];
        T dn, jx, jy, jz;
        moments(v, dn, jx, jy, jz);
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
        const int hx = jh[s] % PX, hy = jh[s] / PX;
        const float* row0 = st + hy * XW + hx + APRON - R;
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = row0[i * POP - cx(i)];
        rs[jh[s]] = psi_of<T>(n0 + sum19(v), d.eos);
      }
    }
    return true;
  };
#pragma unroll 1
  for (int qd = 0; qd <= nplanes; ++qd)
    if (!plane_step(qd)) {
      cp_async_wait_all();
      return false;
    }
  cp_async_wait_all();   // (only empty groups can remain: no copy targets a plane past the chunk)
  return true;
}

template <int ST, int BX, int BY>
__global__ void __launch_bounds__(BX * BY, (TmaShape<ST, BX, BY>::MIN_BLOCKS))
lattice_tma_kernel(LatticeDesc d, const __grid_constant__ TmaMapSet maps, int zchunk) {
  using Sh = TmaShape<ST, BX, BY>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // every box lands on a 128-byte boundary of the CTA's shared window
  const unsigned base = tma_smem(smem_raw);
  unsigned char* smem = smem_raw + ((128u - (base & 127u)) & 127u);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + Sh::bar_off);
  if (threadIdx.x == 0) {
    for (int s = 0; s < Sh::NS; ++s) tma_mbar_init(bars + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (threadIdx.x < Sh::NMAPS)
    asm volatile("prefetch.tensormap [%0];\n" ::"l"((unsigned long long)&maps.map[threadIdx.x]) : "memory");
  step_grid_enter();
  __syncthreads();
  unsigned phase_bits = 0;
  const int ncols = ((d.nx + BX - 1) / BX) * (d.ny / BY);
  const long long items = (long long)ncols * ((d.nz + zchunk - 1) / zchunk);
#pragma unroll 1
  for (long long item = blockIdx.x; item < items; item += gridDim.x)
    if (!tma_process_item<ST, BX, BY>(d, maps, zchunk, item, smem, phase_bits)) break;
}

}  // namespace lbm
