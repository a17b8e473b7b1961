// Shared device definitions of the GB300 Shan-Chen LBM library.
//
// D3Q19 velocity set and weights (Sec. II; c_s^2 = 1/3), the forcing
// stencils of Eq. (8), the pseudopotentials psi(n) and the storage
// precisions.  The population order is the one documented in include/lbm.h.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

constexpr int Q = 19;

// velocity components, population order of include/lbm.h
__host__ __device__ constexpr int cx(int i) {
  constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
  return t[i];
}
__host__ __device__ constexpr int cy(int i) {
  constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
  return t[i];
}
__host__ __device__ constexpr int cz(int i) {
  constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
  return t[i];
}
// the same components for an index known only at run time: component + 1 of
// velocity i in two bits at bit 2i of a packed constant (no memory access)
__host__ __device__ constexpr unsigned long long pack_component(int axis) {
  unsigned long long p = 0;
  for (int i = 0; i < Q; ++i) {
    const int c = axis == 0 ? cx(i) : (axis == 1 ? cy(i) : cz(i));
    p |= (unsigned long long)(c + 1) << (2 * i);
  }
  return p;
}
__host__ __device__ constexpr int cx_rt(int i) { return (int)((pack_component(0) >> (2 * i)) & 3ull) - 1; }
__host__ __device__ constexpr int cy_rt(int i) { return (int)((pack_component(1) >> (2 * i)) & 3ull) - 1; }
__host__ __device__ constexpr int cz_rt(int i) { return (int)((pack_component(2) >> (2 * i)) & 3ull) - 1; }

// D3Q19 weights: 1/3 rest, 1/18 axis, 1/36 diagonal
__host__ __device__ constexpr double wq(int i) {
  return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// ---------------------------------------------------------------- stencils
// Forcing-stencil vectors, grouped by shell |xi|^2, with the shell weights
// W(|xi|^2) that make the stencil isotropic to 4th (E4), 6th (E6) and 8th
// (E8) order with e_2 = 1.  E4: W(1) = 1/6, W(2) = 1/12 (Sec. II).
struct StencilVec { int8_t x, y, z; };

constexpr int kE4Count = 18;
constexpr int kE6Count = 32;
constexpr int kE8Count = 92;

enum PsiKind : int { kPsiExpInv = 0, kPsiOneMinusExp = 1, kPsiCS = 2 };

struct EosParams {
  int kind;
  double G;       // coupling (Eq. (8))
  double a, b, Rgas, T;  // Carnahan-Starling constants (kind == kPsiCS)
  // the same constants rounded to float on the host (set_float_params), so that
  // FP32 kernels take them straight from the parameter bank and convert nothing
  float Gf, af, bf, RTf;
};

template <typename T>
__device__ __forceinline__ T psi_of(T n, const EosParams& e);

template <>
__device__ __forceinline__ double psi_of<double>(double n, const EosParams& e) {
  if (e.kind == kPsiOneMinusExp) return -expm1(-n);
  if (e.kind == kPsiExpInv) return exp(-1.0 / n);
  // Carnahan-Starling mapped: psi = sqrt(2 (p_CS - n c_s^2) / (G c_s^2))
  const double q = e.b * n * 0.25;
  const double om = 1.0 - q;
  const double p = n * e.Rgas * e.T * (1.0 + q + q * q - q * q * q) / (om * om * om) - e.a * n * n;
  return sqrt(2.0 * (p - n * (1.0 / 3.0)) / (e.G * (1.0 / 3.0)));
}

// FP32: 1 - exp(-n) through the hardware exponential (__expf, a few ulp): at the
// densities of the method (n >= 0.05) its absolute error, ~1e-7, is below the
// rounding of the FP32-shifted populations, and it costs a few instructions
// where expm1f costs a few dozen (the step is issue-limited at small boxes).
template <>
__device__ __forceinline__ float psi_of<float>(float n, const EosParams& e) {
  if (e.kind == kPsiOneMinusExp) return 1.0f - __expf(-n);
  if (e.kind == kPsiExpInv) return expf(-1.0f / n);
  const float q = e.bf * n * 0.25f;
  const float om = 1.0f - q;
  const float p = n * e.RTf * (1.0f + q + q * q - q * q * q) / (om * om * om) - e.af * n * n;
  return sqrtf(2.0f * (p - n * (1.0f / 3.0f)) / (e.Gf * (1.0f / 3.0f)));
}

// ---------------------------------------------------------------- storage
enum Prec : int { kF64 = 0, kF32 = 1, kF16 = 2 };

template <int P> struct Storage;
template <> struct Storage<kF64> {
  using S = double;   // stored type
  using T = double;   // arithmetic type
  static __device__ __forceinline__ T load(const S* p, T /*inv_scale*/) { return __ldg(p); }
  static __device__ __forceinline__ void store(S* p, T v, T /*scale*/) { *p = v; }
};
template <> struct Storage<kF32> {
  using S = float;
  using T = float;
  static __device__ __forceinline__ T load(const S* p, T) { return __ldg(p); }
  static __device__ __forceinline__ void store(S* p, T v, T) { *p = v; }
};
template <> struct Storage<kF16> {
  using S = __half;
  using T = float;
  static __device__ __forceinline__ T load(const S* p, T inv_scale) {
    return __half2float(__ldg(p)) * inv_scale;
  }
  static __device__ __forceinline__ void store(S* p, T v, T scale) {
    *p = __float2half_rn(v * scale);
  }
};

// One lattice as the kernels see it.  Populations are stored post-collision
// and pre-streaming: slot i of node x holds f*_i(x, t-1), so the
// pre-collision f_i(x, t) of Eq. (3) is slot i of node x - xi_i.
struct LatticeDesc {
  const void* src;      // populations read this step (19 planes)
  void* dst;            // populations written this step
  int nx, ny, nz;
  long long plane;      // nx*ny*nz
  double omega;         // 1/tau
  double n0;            // storage shift (0 for F64)
  double scale;         // storage scale (1 for F64/F32)
  EosParams eos;
  float n0f, omegaf, scalef, inv_scalef;   // n0, omega, scale, 1/scale rounded to float (host)
  int* err;             // device flag set by a kernel whose bounded wait ran out (may be null)
  const void* tma;      // host: the lattice's TMA tensor maps (TmaMaps) or null; kernels ignore it
};

// The float copies of a descriptor's double parameters; call after setting them.
inline void set_float_params(LatticeDesc& d) {
  d.n0f = (float)d.n0;
  d.omegaf = (float)d.omega;
  d.scalef = (float)d.scale;
  d.inv_scalef = (float)(1.0 / d.scale);
  d.eos.Gf = (float)d.eos.G;
  d.eos.af = (float)d.eos.a;
  d.eos.bf = (float)d.eos.b;
  d.eos.RTf = (float)(d.eos.Rgas * d.eos.T);
}

// A descriptor parameter in the kernel's arithmetic type: the host-rounded float
// copy for FP32 arithmetic, the double itself for FP64.
template <typename T>
__device__ __forceinline__ T dparam(double v, float f) {
  if constexpr (sizeof(T) == 4) return f;
  else return v;
}

constexpr int kMaxTmaMaps = 4;   // tensor maps per population buffer (TMA step kernel)

__host__ __device__ __forceinline__ int wrap(int g, int n) {
  return g < 0 ? g + n : (g >= n ? g - n : g);
}

// Programmatic dependent launch (sm_90 and later).  The step kernels are
// launched with programmatic stream serialisation, so the next step's CTAs are
// scheduled into the slots this step's CTAs free instead of after the whole
// grid has drained.  Each CTA first allows its own successor to be scheduled,
// then waits until the previous grid has completed and its writes are visible;
// no global memory is touched before that wait.  Without the launch attribute
// both instructions are no-ops.
__device__ __forceinline__ void step_grid_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

}  // namespace lbm
