// Observables of one lattice: point samples of the lattice pressure tensor
// and the closing FP64 reduction + closed forms.
//
// Point pass (one thread per sampled node): n and P^xx, P^yy of Eq. (9)
//   P^{mu nu}(x) = n c_s^2 delta + (G c_s^2 / 2) psi(x) sum_a W_a psi(x + xi_a) xi_a^mu xi_a^nu
// at the centre node c (P_in), the farthest corner (P_out) and along the +x
// half axis c + r e_x, r = 0..nx/2 (P_T(r) = P^yy, Sec. III below Eq. (22);
// P_N(r) = P^xx, used by the flat interface's sigma_0, Eq. (25)).
//
// Finalize (one CTA, fixed reduction order, so the result is deterministic):
//   mass M, centre of mass of n - n_out, delta u (Sec. IV), max |u|,
//   R_e from M = 4 pi R_e^3 n_in/3 + (V - 4 pi R_e^3/3) n_out (Sec. IV),
//   C = int r^2 (P_out - P_T) dr, D = int r (P_out - P_T) dr (trapezoid on the
//   nodes), R_s = (6 C / dP)^(1/3) -- the minimum of
//   sigma[R] = dP R / 3 + C / R^2, Eq. (21) with the step P_J integrated
//   exactly -- and sigma_s = dP R_s / 2 (Eq. (12)).
#include <math.h>

#include "lbm.h"
#include "lbm_launch.h"

namespace lbm {

namespace {

template <int P>
__device__ double density_at(const LatticeDesc& d, int x, int y, int z) {
  using S = typename Storage<P>::S;
  using T = typename Storage<P>::T;
  const S* src = static_cast<const S*>(d.src);
  const T inv_scale = (T)(1.0 / d.scale);
  double sum = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int xx = wrap(x - cx(i), d.nx), yy = wrap(y - cy(i), d.ny), zz = wrap(z - cz(i), d.nz);
    sum += (double)Storage<P>::load(src + (long long)i * d.plane + ((long long)zz * d.ny + yy) * d.nx + xx,
                                    inv_scale);
  }
  return d.n0 + sum;
}

template <int P, int ST>
__global__ void point_obs_kernel(LatticeDesc d, PointOut* pts, double* n_line, double* PT_line,
                                 double* PN_line, int line_len) {
  constexpr int R = stencil_radius<ST>();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 + line_len) return;
  const int c[3] = {d.nx / 2, d.ny / 2, d.nz / 2};
  int p[3];
  if (t == 0) {
    p[0] = c[0]; p[1] = c[1]; p[2] = c[2];
  } else if (t == 1) {
    p[0] = (c[0] + d.nx / 2) % d.nx;
    p[1] = (c[1] + d.ny / 2) % d.ny;
    p[2] = (c[2] + d.nz / 2) % d.nz;
  } else {
    p[0] = (c[0] + (t - 2)) % d.nx; p[1] = c[1]; p[2] = c[2];
  }
  const double n = density_at<P>(d, p[0], p[1], p[2]);
  const double psic = psi_of<double>(n, d.eos);
  double sxx = 0.0, syy = 0.0;
  for (int dz = -R; dz <= R; ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        const double W = shell_weight<ST>(dx * dx + dy * dy + dz * dz);
        if (W == 0.0 || (dx == 0 && dy == 0 && dz == 0)) continue;
        const double nb = density_at<P>(d, wrap(p[0] + dx, d.nx), wrap(p[1] + dy, d.ny),
                                        wrap(p[2] + dz, d.nz));
        const double ps = psi_of<double>(nb, d.eos);
        sxx += W * ps * (double)(dx * dx);
        syy += W * ps * (double)(dy * dy);
      }
  const double k = 0.5 * d.eos.G * (1.0 / 3.0) * psic;
  const double Pxx = n * (1.0 / 3.0) + k * sxx;
  const double Pyy = n * (1.0 / 3.0) + k * syy;
  if (t == 0) { pts->n_in = n; pts->P_in = Pxx; }
  else if (t == 1) { pts->n_out = n; pts->P_out = Pxx; }
  else { n_line[t - 2] = n; PT_line[t - 2] = Pyy; PN_line[t - 2] = Pxx; }
}

__global__ void finalize_kernel(FinalizeArgs a) {
  constexpr int NT = 256;
  __shared__ double red[8][NT];
  const int t = threadIdx.x;
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // mass, wsum, wd0, wd1, wd2, du, bad, max_u
  for (long long k = t; k < a.n_partials; k += NT) {
    const FieldPartial& p = a.partials[k];
    s[0] += p.mass; s[1] += p.wsum; s[2] += p.wd[0]; s[3] += p.wd[1]; s[4] += p.wd[2];
    s[5] += p.du; s[6] += p.bad; s[7] = fmax(s[7], p.max_u);
  }
  for (int q = 0; q < 8; ++q) red[q][t] = s[q];
  __syncthreads();
  for (int off = NT / 2; off > 0; off >>= 1) {
    if (t < off) {
      for (int q = 0; q < 7; ++q) red[q][t] += red[q][t + off];
      red[7][t] = fmax(red[7][t], red[7][t + off]);
    }
    __syncthreads();
  }
  if (t != 0) return;
  lbm_obs o;
  const PointOut pt = *a.pts;
  o.n_in = pt.n_in;
  o.n_out = pt.n_out;
  o.P_in = pt.P_in;
  o.P_out = pt.P_out;
  o.dP = pt.P_in - pt.P_out;
  o.mass = red[0][0];
  const double wsum = red[1][0];
  // centre of mass of n - n_out: centre node + mean minimum-image displacement
  double rel[3] = {red[2][0] / wsum, red[3][0] / wsum, red[4][0] / wsum};
  for (int k = 0; k < 3; ++k) o.com[k] = (double)a.center[k] + rel[k];
  const double V = (double)a.volume;
  o.R_e = cbrt(3.0 * (o.mass - V * o.n_out) / (4.0 * M_PI * (o.n_in - o.n_out)));
  // trapezoid rule on r = 0..line_len-1
  double C = 0.0, D = 0.0;
  for (int r = 0; r < a.line_len; ++r) {
    const double g = o.P_out - a.PT_line[r];
    const double wt = (r == 0 || r == a.line_len - 1) ? 0.5 : 1.0;
    C += wt * (double)r * (double)r * g;
    D += wt * (double)r * g;
  }
  o.C = C;
  o.D = D;
  const double q = (o.dP != 0.0) ? C / o.dP : -1.0;
  unsigned st = 0;
  if (q > 0.0) {
    o.R_s = cbrt(6.0 * q);
    o.sigma_s = 0.5 * o.dP * o.R_s;
  } else {
    o.R_s = NAN;
    o.sigma_s = NAN;
    st |= 1u;
  }
  if (a.contrast0 > 0.0 && fabs(o.n_in - o.n_out) < 1e-2 * a.contrast0) st |= 2u;
  for (int k = 0; k < 3; ++k)
    if (!(fabs(rel[k]) <= 1e-3)) st |= 4u;
  if (red[6][0] > 0.0 || !isfinite(o.mass)) st |= 8u;
  if (a.err && *a.err) st |= 16u;
  o.max_u = red[7][0];
  o.du = a.have_u_old ? red[5][0] / V : 0.0;
  const double prev = *a.dP_prev;
  o.dP_rel_change = isnan(prev) ? NAN : fabs(o.dP - prev) / fabs(prev);
  *a.dP_prev = o.dP;
  o.steps = a.steps;
  o.status_bits = st;
  o.criterion = 0;
  *static_cast<lbm_obs*>(a.obs_out) = o;
}

}  // namespace

cudaError_t launch_point_obs(int prec, int stencil, const LatticeDesc& d, PointOut* pts,
                             double* n_line, double* PT_line, double* PN_line, cudaStream_t s) {
  const int line_len = d.nx / 2 + 1;
  const int n = 2 + line_len;
  const dim3 grid((n + 63) / 64);
#define LBM_POINT(PR, STC) \
  point_obs_kernel<PR, STC><<<grid, 64, 0, s>>>(d, pts, n_line, PT_line, PN_line, line_len)
  if (stencil != 4 && stencil != 6 && stencil != 8) return cudaErrorInvalidValue;
  switch (prec) {
    case kF64: if (stencil == 4) LBM_POINT(kF64, 4); else if (stencil == 6) LBM_POINT(kF64, 6); else LBM_POINT(kF64, 8); break;
    case kF32: if (stencil == 4) LBM_POINT(kF32, 4); else if (stencil == 6) LBM_POINT(kF32, 6); else LBM_POINT(kF32, 8); break;
    case kF16: if (stencil == 4) LBM_POINT(kF16, 4); else if (stencil == 6) LBM_POINT(kF16, 6); else LBM_POINT(kF16, 8); break;
    default: return cudaErrorInvalidValue;
  }
#undef LBM_POINT
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t s) {
  finalize_kernel<<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lbm
