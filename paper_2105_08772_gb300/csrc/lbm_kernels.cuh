// Fused Shan-Chen step and field-observable kernels (templated; included by
// one translation unit per storage precision).
//
// One time step of Sec. II, Eq. (3):
//   pull      f_i(x, t) = f*_i(x - xi_i, t - 1)                 (streaming)
//   moments   n = sum_i f_i, j = sum_i xi_i f_i
//   force     F = -G c_s^2 psi(x) sum_a W_a psi(x + xi_a) xi_a   Eq. (8)
//   velocity  u = (j + F/2) / n                                  Eq. (7)
//   collide   f*_i = f_i - (f_i - f_i^eq)/tau + F_i              Eqs. (4)-(6)
//   store     f*_i(x, t) at x (read by the next step's pull).
//
// The force needs psi at the stencil neighbours, i.e. the density of the
// neighbours at the same time step.  A CTA owns a BX x BY column of the box
// and marches through a chunk of z planes.  For each plane it pulls the 19
// populations of the tile plus an R-node xy halo, forms n and psi there and
// keeps them in a ring of 2R+1 psi planes in shared memory; the tile's own
// pulled populations are parked in shared memory until the plane is
// collided R planes later.  Density and psi never touch HBM: every step
// moves 19 loads + 19 stores per node, the halo re-reads hit L2.  Two
// population buffers alternate (the halo reads of one CTA may not race with
// another CTA's in-place writes).
#pragma once

#include "lbm_common.cuh"

namespace lbm {

// shell weights W(|xi|^2) of the forcing stencils (Sec. II; wider stencils
// are the isotropic ones the paper cites): 0 where a vector is not used
template <int ST>
__host__ __device__ constexpr double shell_weight(int s) {
  if (ST == 4) return s == 1 ? 1.0 / 6.0 : (s == 2 ? 1.0 / 12.0 : 0.0);
  if (ST == 6)
    return s == 1 ? 2.0 / 15.0 : s == 2 ? 1.0 / 15.0 : s == 3 ? 1.0 / 60.0 : s == 4 ? 1.0 / 120.0 : 0.0;
  // E8
  return s == 1 ? 4.0 / 45.0
       : s == 2 ? 1.0 / 21.0
       : s == 3 ? 2.0 / 105.0
       : s == 4 ? 5.0 / 504.0
       : s == 5 ? 1.0 / 315.0
       : s == 6 ? 1.0 / 630.0
       : s == 8 ? 1.0 / 5040.0
       : 0.0;
}
template <int ST> constexpr int stencil_radius() { return ST == 4 ? 1 : 2; }

// per-CTA reduction record of the field-observable pass
struct FieldPartial {
  double mass;        // sum n
  double wsum;        // sum (n - n_out)
  double wd[3];       // sum (n - n_out) d_alpha (minimum image about the centre)
  double du;          // sum_x sum_alpha |u - u_old|
  double max_u;       // max |u|
  double bad;         // count of non-finite or non-positive densities
};

struct ObsArgs {
  const double* n_out;     // device scalar: density at the farthest corner
  void* u_old;             // velocity snapshot, 3 planes (double for F64, float otherwise)
  int have_u_old;          // 0 right after an init: skip the delta-u sum
  FieldPartial* partials;  // one record per CTA
  double* rho_out;         // optional full density field (doubles), may be null
  double* u_out;           // optional full velocity field (3 planes of doubles), may be null
  int write_u_old;         // 1: replace the snapshot by the current velocity
};

template <int P, int ST, int BX, int BY>
struct StepShape {
  using T = typename Storage<P>::T;
  static constexpr int R = stencil_radius<ST>();
  static constexpr int PX = BX + 2 * R;
  static constexpr int PY = BY + 2 * R;
  static constexpr int NT = BX * BY;
  static constexpr int NR = 2 * R + 1;   // psi planes in the ring
  static constexpr int NP = R + 1;       // parked population planes
  static constexpr size_t ring_bytes = sizeof(T) * NR * PX * PY;
  static constexpr size_t pops_bytes = sizeof(T) * NP * Q * NT;
  static constexpr size_t smem_bytes = ring_bytes + pops_bytes;
};

// Mirror-exact summation.  The box, the droplet and its initial profile are
// symmetric under the three reflections x -> -x, y -> -y, z -> -z about the centre
// node, and so is the exact dynamics; floating-point sums keep that symmetry only
// if each reflection maps every sum onto the same operations.  A reflection
// permutes the populations (x: 1<->2, 7<->10, 8<->9, 11<->14, 12<->13; y: 3<->4,
// 7<->9, 8<->10, 15<->18, 16<->17; z: 5<->6, 11<->13, 12<->14, 15<->17, 16<->18), so
// the sums below add opposite pairs first and then exactly the pair sums a
// reflection swaps; a + b = b + a and a - b = -(b - a) hold exactly, so a mirrored
// state gives bitwise mirrored densities, momenta and forces, the drop's centre of
// mass stays on the centre node, and rounding (FP16 storage above all) cannot push
// the drop off it.
//
// sum of the nine opposite-pair sums g_i + g_ibar, grouped by the reflections
template <typename T>
__device__ __forceinline__ T pair_sum9(T p12, T p34, T p56, T p78, T p910, T p1112, T p1314, T p1516, T p1718) {
  return ((p12 + p34) + p56) + (((p78 + p910) + (p1112 + p1314)) + (p1516 + p1718));
}

// density: rest population plus the mirror-exact sum of the pair sums (the order
// is fixed, so every kernel forms bitwise the same density)
template <typename T>
__device__ __forceinline__ T sum19(const T* v) {
  return v[0] + pair_sum9<T>(v[1] + v[2], v[3] + v[4], v[5] + v[6], v[7] + v[8], v[9] + v[10],
                             v[11] + v[12], v[13] + v[14], v[15] + v[16], v[17] + v[18]);
}

// Pull the 19 populations of every node of one padded plane (tile + R halo),
// form psi into the ring slot, park the interior populations if asked.
template <int P, int ST, int BX, int BY>
__device__ __forceinline__ void load_plane(const LatticeDesc& d, int x0, int y0, int w, int h,
                                           int zg, typename Storage<P>::T* ring_slot,
                                           typename Storage<P>::T* pops_slot, bool keep) {
  using Sh = StepShape<P, ST, BX, BY>;
  using T = typename Sh::T;
  using S = typename Storage<P>::S;
  constexpr int R = Sh::R, PX = Sh::PX, PY = Sh::PY, NT = Sh::NT;
  const S* __restrict__ src = static_cast<const S*>(d.src);
  const int nx = d.nx, ny = d.ny, nz = d.nz;
  const long long plane = d.plane;
  const T inv_scale = dparam<T>(1.0 / d.scale, d.inv_scalef);
  const T n0 = dparam<T>(d.n0, d.n0f);
  const int z = wrap(zg, nz);
  const int zm = wrap(z - 1, nz), zp = wrap(z + 1, nz);
  const int tid = threadIdx.x;
  for (int j = tid; j < PX * PY; j += NT) {
    const int jx = j % PX, jy = j / PX;
    if (jx >= w + 2 * R || jy >= h + 2 * R) continue;
    const int gx = wrap(x0 + jx - R, nx), gy = wrap(y0 + jy - R, ny);
    const int xs[3] = {wrap(gx + 1, nx), gx, wrap(gx - 1, nx)};   // source x for c_x = -1, 0, +1
    const int ys[3] = {wrap(gy + 1, ny), gy, wrap(gy - 1, ny)};
    const int zs[3] = {zp, z, zm};
    const bool interior = keep && jx >= R && jx < R + w && jy >= R && jy < R + h;
    const int li = (jy - R) * BX + (jx - R);
    T v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const long long idx = (long long)i * plane +
                            ((long long)zs[cz(i) + 1] * ny + ys[cy(i) + 1]) * nx + xs[cx(i) + 1];
      v[i] = Storage<P>::load(src + idx, inv_scale);
      if (interior) pops_slot[i * NT + li] = v[i];
    }
    ring_slot[jy * PX + jx] = psi_of<T>(n0 + sum19(v), d.eos);
  }
}

// Shan-Chen force (Eq. (8)) from psi planes in shared memory.  planes[dz + R]
// points at the node's own position in the psi plane at offset dz; rows are PX
// apart.  The stencil is summed through the differences D(xi) = psi(x + xi) -
// psi(x - xi), so that two psi values cancel before they are scaled: a uniform
// region gives exactly F = 0 and the rounding error scales with F, not with the
// psi values.  (Summing the 18 terms one by one in raster order lets FP32 rounding
// build a spurious force that grows the density error of a 1000-step droplet run
// tenfold.)
// Mirror-exact order: component a of the force is, per shell, a sum over the
// orbits of the stencil vectors with xi_a > 0 under the two reflections that
// leave axis a alone -- {(xi_a, +-b, +-c)} -- each orbit summed as
// ((D(a,b,c) + D(a,-b,c)) + (D(a,b,-c) + D(a,-b,-c))); the shells are then
// weighted and added in a fixed order.  A reflection of the field maps every
// orbit sum onto itself (reordered by exactly commuting additions) or onto its
// negative, so mirrored psi gives a bitwise mirrored force (see sum19).
// OWN: own[dz + R] holds psi of the node's own column at offset dz (the caller
// formed those values and kept them in registers); differences along the node's
// own column take them from there instead of from shared memory.
template <typename T, int ST, int PX, bool OWN>
__device__ __forceinline__ T sc_diff(const T* const* planes, const T* own, int dx, int dy, int dz) {
  constexpr int R = stencil_radius<ST>();
  if (OWN && dx == 0 && dy == 0) return own[R + dz] - own[R - dz];
  return planes[R + dz][dy * PX + dx] - planes[R - dz][-dy * PX - dx];
}

template <typename T, int ST, int PX, bool OWN>
__device__ __forceinline__ T sc_force_axis(const T* const* planes, const T* own, int axis) {
  constexpr int R = stencil_radius<ST>();
  T F = (T)0;
  bool any_shell = false;
#pragma unroll
  for (int sh = 1; sh <= 3 * R * R; ++sh) {
    const double W = shell_weight<ST>(sh);
    if (W == 0.0) continue;
    T S = (T)0;
    bool any = false;
#pragma unroll
    for (int a = 1; a <= R; ++a) {
#pragma unroll
      for (int b = 0; b <= R; ++b) {
#pragma unroll
        for (int c = 0; c <= R; ++c) {
          if (a * a + b * b + c * c != sh) continue;
          // the vector (a, b, c) in the frame of `axis`: a along it, b and c along the
          // other two axes in increasing order
          auto D = [&](int bb, int cc) {
            return axis == 0 ? sc_diff<T, ST, PX, OWN>(planes, own, a, bb, cc)
                 : axis == 1 ? sc_diff<T, ST, PX, OWN>(planes, own, bb, a, cc)
                             : sc_diff<T, ST, PX, OWN>(planes, own, bb, cc, a);
          };
          T O;
          if (b > 0 && c > 0) O = (D(b, c) + D(-b, c)) + (D(b, -c) + D(-b, -c));
          else if (b > 0) O = D(b, 0) + D(-b, 0);
          else if (c > 0) O = D(0, c) + D(0, -c);
          else O = D(0, 0);
          if (a != 1) O = (T)a * O;
          S = any ? S + O : O;
          any = true;
        }
      }
    }
    if (!any) continue;
    F = any_shell ? F + (T)W * S : (T)W * S;
    any_shell = true;
  }
  return F;
}

template <typename T, int ST, int PX, bool OWN = false>
__device__ __forceinline__ void sc_force_pairs(const T* const* planes, T G, T& Fx, T& Fy, T& Fz,
                                               const T* own = nullptr) {
  constexpr int R = stencil_radius<ST>();
  const T k = -G * (T)(1.0 / 3.0) * (OWN ? own[R] : planes[R][0]);
  Fx = k * sc_force_axis<T, ST, PX, OWN>(planes, own, 0);
  Fy = k * sc_force_axis<T, ST, PX, OWN>(planes, own, 1);
  Fz = k * sc_force_axis<T, ST, PX, OWN>(planes, own, 2);
}

// Force at interior node (tx, ty) of the current plane from the psi ring;
// slots[k] is the ring slot of plane z + k - R.
template <int P, int ST, int BX, int BY>
__device__ __forceinline__ void sc_force(const typename Storage<P>::T* ring, const int* slots, int tx,
                                         int ty, typename Storage<P>::T G,
                                         typename Storage<P>::T& Fx, typename Storage<P>::T& Fy,
                                         typename Storage<P>::T& Fz) {
  using Sh = StepShape<P, ST, BX, BY>;
  using T = typename Sh::T;
  constexpr int R = Sh::R, PX = Sh::PX, PY = Sh::PY;
  const T* planes[2 * R + 1];
#pragma unroll
  for (int k = 0; k <= 2 * R; ++k) planes[k] = ring + slots[k] * (PX * PY) + (ty + R) * PX + (tx + R);
  sc_force_pairs<T, ST, PX>(planes, G, Fx, Fy, Fz);
}

// BGK + Guo collision of one node in shifted form, g_i = f_i - w_i n0:
//   g*_i = (1 - omega) g_i + omega g_i^eq + F_i
//   g_i^eq = w_i [dn + n (3 e.u + 9/2 (e.u)^2 - 3/2 u.u)]          Eq. (6)
//   F_i    = (1 - omega/2) w_i [3 e.F + 9 (e.u)(e.F) - 3 u.F]       Eq. (5)
// Opposite velocities share the even part; the odd part flips sign.
// CLOSE_MASS: the collision conserves mass exactly (sum g*_i = dn), but the
// rounded weights do not sum to exactly 1 (FP32: 1 + 1.5e-8), which would
// add a systematic error proportional to n - n0 to every node every step; the
// rest population is set to dn - sum_{i>0} g*_i instead (the same value in
// exact arithmetic), so mass changes only by uncorrelated rounding.
// UNIT_TAU: tau = 1 (the relaxation time the method uses); then 1 - omega = 0
// and the post-collision populations depend on the old ones only through n, j.
// SCALED: the outputs come multiplied by wscale, a power of two (FP16 storage's
// 2^k), folded into the weights and the mass closure; a power-of-two factor
// commutes with every rounding, so the values are bitwise those of the
// unscaled collision times wscale.
template <typename T, bool CLOSE_MASS, bool UNIT_TAU = false, bool SCALED = false>
__device__ __forceinline__ void collide(T* g, T dn, T n, T ux, T uy, T uz, T Fx, T Fy, T Fz,
                                        T omega_in, T wscale = (T)1) {
  const T omega = UNIT_TAU ? (T)1 : omega_in;
  const T uu = ux * ux + uy * uy + uz * uz;
  const T uF = ux * Fx + uy * Fy + uz * Fz;
  const T cg = (T)1 - (T)0.5 * omega;     // 1 - 1/(2 tau)
  const T om1 = (T)1 - omega;
  const T base = omega * (dn - (T)1.5 * n * uu) - (T)3 * cg * uF;
  g[0] = UNIT_TAU ? (T)(1.0 / 3.0) * base : om1 * g[0] + (T)(1.0 / 3.0) * base;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const T eu = (T)cx(i) * ux + (T)cy(i) * uy + (T)cz(i) * uz;
    const T eF = (T)cx(i) * Fx + (T)cy(i) * Fy + (T)cz(i) * Fz;
    const T wi = SCALED ? (T)wq(i) * wscale : (T)wq(i);
    const T even = base + omega * (T)4.5 * n * eu * eu + (T)9 * cg * eu * eF;
    const T odd = (T)3 * (omega * n * eu + cg * eF);
    if (UNIT_TAU) {
      g[i] = wi * (even + odd);
      g[i + 1] = wi * (even - odd);
    } else {
      g[i] = om1 * g[i] + wi * (even + odd);
      g[i + 1] = om1 * g[i + 1] + wi * (even - odd);
    }
  }
  if (CLOSE_MASS) {
    // pair sums first (their odd parts cancel), then the mirror-exact grouping
    g[0] = (SCALED ? dn * wscale : dn) -
           pair_sum9<T>(g[1] + g[2], g[3] + g[4], g[5] + g[6], g[7] + g[8], g[9] + g[10], g[11] + g[12],
                        g[13] + g[14], g[15] + g[16], g[17] + g[18]);
  }
}

// The unit-tau collision of `collide<T, true, true>` with each post-collision
// population stored as soon as it is formed (store(i, g_i)): only the nine pair
// sums stay live for the mass closure, not all nineteen values.  Same operations
// in the same order, so the stored values are bitwise those of collide().
template <typename T, typename Store>
__device__ __forceinline__ void collide_unit_tau_store(T dn, T n, T ux, T uy, T uz, T Fx, T Fy, T Fz,
                                                       Store store) {
  const T uu = ux * ux + uy * uy + uz * uz;
  const T uF = ux * Fx + uy * Fy + uz * Fz;
  const T cg = (T)1 - (T)0.5 * (T)1;
  const T base = (T)1 * (dn - (T)1.5 * n * uu) - (T)3 * cg * uF;
  T p[9];
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const T eu = (T)cx(i) * ux + (T)cy(i) * uy + (T)cz(i) * uz;
    const T eF = (T)cx(i) * Fx + (T)cy(i) * Fy + (T)cz(i) * Fz;
    const T wi = (T)wq(i);
    const T even = base + (T)1 * (T)4.5 * n * eu * eu + (T)9 * cg * eu * eF;
    const T odd = (T)3 * ((T)1 * n * eu + cg * eF);
    const T ga = wi * (even + odd), gb = wi * (even - odd);
    store(i, ga);
    store(i + 1, gb);
    p[i / 2] = ga + gb;
  }
  store(0, dn - pair_sum9<T>(p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], p[8]));
}

// density and momentum of one node: momentum from the differences of the nine
// opposite pairs (1,2), (3,4), ..., (17,18) of the population order
template <typename T>
__device__ __forceinline__ void moments(const T* g, T& dn, T& jx, T& jy, T& jz) {
  dn = sum19(g);
  const T d12 = g[1] - g[2], d34 = g[3] - g[4], d56 = g[5] - g[6];
  const T d78 = g[7] - g[8], d910 = g[9] - g[10], d1112 = g[11] - g[12];
  const T d1314 = g[13] - g[14], d1516 = g[15] - g[16], d1718 = g[17] - g[18];
  // x: 1 (+), 7 (+), 9 (+), 11 (+), 13 (+); y: 3, 7, 10, 15, 17 (+); z: 5, 11, 14, 15, 18 (+);
  // the differences a reflection swaps are added (or subtracted) first: mirror-exact
  jx = (d12 + (d78 + d910)) + (d1112 + d1314);
  jy = (d34 + (d78 - d910)) + (d1516 + d1718);
  jz = (d56 + (d1112 - d1314)) + (d1516 - d1718);
}

template <typename T>
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

enum Mode : int { kModeStep = 0, kModeObs = 1 };

// One CTA: tile (blockIdx.x over tiles), z chunk (blockIdx.y).
template <int P, int ST, int BX, int BY, int MODE>
__global__ void __launch_bounds__(BX * BY)
lattice_kernel(LatticeDesc d, int zchunk, ObsArgs oa) {
  using Sh = StepShape<P, ST, BX, BY>;
  using T = typename Sh::T;
  using S = typename Storage<P>::S;
  constexpr int R = Sh::R, NR = Sh::NR, NP = Sh::NP, NT = Sh::NT, PX = Sh::PX, PY = Sh::PY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);
  T* pops = reinterpret_cast<T*>(smem_raw + Sh::ring_bytes);

  const int tiles_x = (d.nx + BX - 1) / BX;
  const int x0 = (blockIdx.x % tiles_x) * BX;
  const int y0 = (blockIdx.x / tiles_x) * BY;
  const int w = min(BX, d.nx - x0), h = min(BY, d.ny - y0);
  const int z0 = blockIdx.y * zchunk;
  const int zc = min(zchunk, d.nz - z0);
  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const bool active = tx < w && ty < h;

  // prologue: planes z0-R .. z0+R-1 (q = 0 .. 2R-1); populations kept for z0 .. z0+R-1
#pragma unroll 1
  for (int q = 0; q < 2 * R; ++q) {
    const int kk = q - R;   // plane index relative to z0
    load_plane<P, ST, BX, BY>(d, x0, y0, w, h, z0 + kk, ring + (q % NR) * PX * PY,
                              pops + ((kk + NP) % NP) * Q * NT, kk >= 0 && kk < zc);
  }

  const T G = dparam<T>(d.eos.G, d.eos.Gf), omega = dparam<T>(d.omega, d.omegaf), n0 = dparam<T>(d.n0, d.n0f);
  const T scale = dparam<T>(d.scale, d.scalef);
  const long long plane = d.plane;
  double acc_mass = 0, acc_w = 0, acc_wd0 = 0, acc_wd1 = 0, acc_wd2 = 0, acc_du = 0, acc_max = 0,
         acc_bad = 0;
  double nout = 0;
  if (MODE == kModeObs) nout = *oa.n_out;

#pragma unroll 1
  for (int k = 0; k < zc; ++k) {
    // lead plane z0 + k + R (q = k + 2R)
    {
      const int q = k + 2 * R;
      const int kk = k + R;
      load_plane<P, ST, BX, BY>(d, x0, y0, w, h, z0 + kk, ring + (q % NR) * PX * PY,
                                pops + (kk % NP) * Q * NT, kk < zc);
    }
    __syncthreads();
    if (active) {
      int slots[2 * R + 1];
#pragma unroll
      for (int s = 0; s <= 2 * R; ++s) slots[s] = (k + s) % NR;
      const T* pk = pops + (k % NP) * Q * NT;
      T g[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] = pk[i * NT + tid];
      T Fx, Fy, Fz;
      sc_force<P, ST, BX, BY>(ring, slots, tx, ty, G, Fx, Fy, Fz);
      const int z = z0 + k;
      const long long node = ((long long)z * d.ny + (y0 + ty)) * d.nx + (x0 + tx);
      if (MODE == kModeStep) {
        T dn, jx, jy, jz;
        moments(g, dn, jx, jy, jz);
        const T n = n0 + dn;
        const T inv_n = (T)1 / n;
        const T ux = (jx + (T)0.5 * Fx) * inv_n;
        const T uy = (jy + (T)0.5 * Fy) * inv_n;
        const T uz = (jz + (T)0.5 * Fz) * inv_n;
        collide<T, true>(g, dn, n, ux, uy, uz, Fx, Fy, Fz, omega);
        S* __restrict__ dst = static_cast<S*>(d.dst);
#pragma unroll
        for (int i = 0; i < Q; ++i) Storage<P>::store(dst + (long long)i * plane + node, g[i], scale);
      } else {
        // observables: moments and velocity accumulated in FP64 whatever the storage
        double gd[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) gd[i] = (double)g[i];
        double dnd, jxd, jyd, jzd;
        moments(gd, dnd, jxd, jyd, jzd);
        const double nd = d.n0 + dnd;
        const double uxd = (jxd + 0.5 * (double)Fx) / nd;
        const double uyd = (jyd + 0.5 * (double)Fy) / nd;
        const double uzd = (jzd + 0.5 * (double)Fz) / nd;
        acc_mass += nd;
        if (!(nd > 0.0) || !isfinite(nd) || !isfinite(uxd) || !isfinite(uyd) || !isfinite(uzd))
          acc_bad += 1.0;
        const double wgt = nd - nout;
        acc_w += wgt;
        // minimum-image displacement from the centre node; the plane at exactly
        // half the box (even sizes) is both images and counts as 0
        const int X = x0 + tx, Y = y0 + ty, Z = z;
        int dxi = X - d.nx / 2, dyi = Y - d.ny / 2, dzi = Z - d.nz / 2;
        if (2 * dxi >= d.nx) dxi -= d.nx; else if (2 * dxi < -d.nx) dxi += d.nx;
        if (2 * dyi >= d.ny) dyi -= d.ny; else if (2 * dyi < -d.ny) dyi += d.ny;
        if (2 * dzi >= d.nz) dzi -= d.nz; else if (2 * dzi < -d.nz) dzi += d.nz;
        if (2 * dxi == -d.nx) dxi = 0;
        if (2 * dyi == -d.ny) dyi = 0;
        if (2 * dzi == -d.nz) dzi = 0;
        acc_wd0 += wgt * dxi;
        acc_wd1 += wgt * dyi;
        acc_wd2 += wgt * dzi;
        acc_max = fmax(acc_max, sqrt(uxd * uxd + uyd * uyd + uzd * uzd));
        if (P == kF64) {
          double* uo = static_cast<double*>(oa.u_old);
          if (oa.have_u_old)
            acc_du += fabs(uxd - uo[node]) + fabs(uyd - uo[plane + node]) + fabs(uzd - uo[2 * plane + node]);
          if (oa.write_u_old) {
            uo[node] = uxd;
            uo[plane + node] = uyd;
            uo[2 * plane + node] = uzd;
          }
        } else {
          float* uo = static_cast<float*>(oa.u_old);
          if (oa.have_u_old)
            acc_du += fabs(uxd - (double)uo[node]) + fabs(uyd - (double)uo[plane + node]) +
                      fabs(uzd - (double)uo[2 * plane + node]);
          if (oa.write_u_old) {
            uo[node] = (float)uxd;
            uo[plane + node] = (float)uyd;
            uo[2 * plane + node] = (float)uzd;
          }
        }
        if (oa.rho_out) oa.rho_out[node] = nd;
        if (oa.u_out) {
          oa.u_out[node] = uxd;
          oa.u_out[plane + node] = uyd;
          oa.u_out[2 * plane + node] = uzd;
        }
      }
    }
    __syncthreads();
  }

  if (MODE == kModeObs) {
    __shared__ double red[8][NT / 32];
    double v[8] = {acc_mass, acc_w, acc_wd0, acc_wd1, acc_wd2, acc_du, acc_bad, acc_max};
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int q = 0; q < 7; ++q) v[q] = warp_sum<double>(v[q]);
    v[7] = warp_max(v[7]);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) red[q][warp] = v[q];
    }
    __syncthreads();
    if (tid == 0) {
      double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int wi = 0; wi < NT / 32; ++wi) {
#pragma unroll
        for (int q = 0; q < 7; ++q) s[q] += red[q][wi];
        s[7] = fmax(s[7], red[7][wi]);
      }
      FieldPartial& out = oa.partials[blockIdx.y * gridDim.x + blockIdx.x];
      out.mass = s[0];
      out.wsum = s[1];
      out.wd[0] = s[2];
      out.wd[1] = s[3];
      out.wd[2] = s[4];
      out.du = s[5];
      out.bad = s[6];
      out.max_u = s[7];
    }
  }
}

}  // namespace lbm
