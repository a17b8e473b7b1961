"""Observables of a droplet / bubble field (oracle, test infrastructure).

Paper references:

* lattice pressure tensor, Eq. (9):
      P^{mu nu}(x) = n c_s^2 delta^{mu nu}
                     + (G c_s^2/2) psi(x) sum_a W_a psi(x + xi_a) xi_a^mu xi_a^nu
* Sec. IV: P_in at the centre node (floor(L/2), floor(L/2), floor(L/2)), P_out
  at the farthest corner, Delta P = P_in - P_out (Sec. III, below Eq. (11));
  the centre of mass must lie within 1e-3 of the centre; convergence every
  2^11 steps on |Delta P(t) - Delta P(t + dt)| / Delta P(t) < 1e-5 or
  delta u = L^-3 sum_x sum_alpha |u^alpha(t + dt) - u^alpha(t)| < 1e-12.
* Sec. IV, last paragraph: the equimolar radius from
  M = 4 pi R_e^3 n_in / 3 + (V - 4 pi R_e^3 / 3) n_out.
* Eq. (21): sigma[R] = int_0^inf (r/R)^2 [P_J(r;R) - P_T(r)] dr, with the
  pressure-jump function P_J = P_in for r < R and P_out for r > R
  (Sec. III, above Eq. (18)), P_T = P^yy sampled along the +x axis from the
  centre (Sec. III below Eq. (22)).  Eq. (22) gives [d sigma/dR].  R_s is
  the minimum of sigma[R]; sigma_s = sigma[R_s] = Delta P R_s / 2 (Eq. (12)).

Readings (the paper is silent on them):

* Even box sizes: the "farthest corner" is (c + floor(L/2)) mod L per axis,
  which is the paper's (L-1, L-1, L-1) for the odd L it uses.
* Centre of mass: of n - n_out with minimum-image displacements from the
  centre node, so the uniform outer phase does not contribute; for even L
  the plane at distance exactly L/2 is both images and counts as 0.
* Integrals along r: P_J is a step, integrated exactly; P_T is known on the
  integer nodes r = 0..floor(L/2) and integrated by the trapezoid rule.  With
  C = int r^2 (P_out - P_T) dr and D = int r (P_out - P_T) dr:
      sigma[R]     = Delta P R / 3 + C / R^2                     (Eq. (21))
      [dsigma/dR]  = Delta P / 3 - 2 C / R^3 + 2 D / R^2          (Eq. (22))
  so the minimum is R_s = (6 C / Delta P)^(1/3) when C / Delta P > 0 and
  otherwise there is none (status NO_MINIMUM).  D vanishes at mechanical
  equilibrium (the n = d - 1 identity of Eq. (17)), so the two forms of
  sigma' agree there.
* The paper's own route, "interpolating the position of the minimum", is
  ``sigma_min_by_grid``: sigma[R] on a grid with P_T linearly interpolated,
  a parabola through the three lowest grid points.  Its R_s differs from the
  closed form only by the quadrature of the P_T part (node trapezoid vs
  interpolated fine grid): below 1% for interfaces a few nodes wide.
* Bubbles enter the Tolman fit with negative curvature (Sec. IV): R_s -> -R_s.
* hat-delta (Sec. IV, last paragraph; Fig. 4): hat-delta_+- = +-(R_e - R_s), + for
  droplets and - for bubbles.  Its flat limit is taken as the intercept of one
  least-squares straight line in the signed curvature x = +-1/R_s through the
  droplets and the bubbles together (the paper does not say how its flat-limit
  points were obtained).
* Collapse: |n_in - n_out| below 1e-2 of the initial contrast.

Parity: Eq. (9) pinned by the uniform field (P = P(n) delta exactly) and the
flat run; sigma[R] pinned by the universal curve, sigma'(R_s) = 0 and the
generalised Laplace law Eq. (11); R_e by a sharp-sphere field.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import eos as _eos
from . import lbm3d

CS2 = 1.0 / 3.0

ST_NO_MINIMUM = 1
ST_COLLAPSED = 2
ST_OFF_CENTER = 4


def pressure_tensor(n, psi, G, vectors, weights):
    """Eq. (9) on the whole field, shape [3, 3, z, y, x]."""
    acc = np.zeros((3, 3) + n.shape)
    for xi, w in zip(vectors, weights):
        nb = lbm3d.shift(psi, xi)
        for mu in range(3):
            for nu in range(3):
                if xi[mu] != 0 and xi[nu] != 0:
                    acc[mu, nu] += w * xi[mu] * xi[nu] * nb
    P = 0.5 * G * CS2 * psi * acc
    for mu in range(3):
        P[mu, mu] += n * CS2
    return P


def centre_node(shape_zyx):
    nz, ny, nx = shape_zyx
    return (nx // 2, ny // 2, nz // 2)


def far_node(shape_zyx):
    nz, ny, nx = shape_zyx
    c = centre_node(shape_zyx)
    return ((c[0] + nx // 2) % nx, (c[1] + ny // 2) % ny, (c[2] + nz // 2) % nz)


@dataclass
class Obs:
    n_in: float
    n_out: float
    P_in: float
    P_out: float
    dP: float
    mass: float
    com: np.ndarray
    R_e: float
    C: float
    D: float
    R_s: float
    sigma_s: float
    max_u: float
    status: int
    PT_line: np.ndarray = field(repr=False)
    n_line: np.ndarray = field(repr=False)


def line_integrals(PT_line, P_out):
    """(C, D) = (int r^2 (P_out - P_T) dr, int r (P_out - P_T) dr), trapezoid on r = 0..r_max."""
    r = np.arange(len(PT_line), dtype=np.float64)
    g = P_out - PT_line
    return float(np.trapezoid(r * r * g, r)), float(np.trapezoid(r * g, r))


def sigma_of_R(R, dP, C, D):
    """(sigma[R], [dsigma/dR]) from Eqs. (21), (22) with the module's quadrature."""
    R = np.asarray(R, dtype=np.float64)
    return dP * R / 3.0 + C / R ** 2, dP / 3.0 - 2.0 * C / R ** 3 + 2.0 * D / R ** 2


def surface_of_tension(dP, C):
    """R_s = (6 C / Delta P)^(1/3), or NaN when sigma[R] has no minimum."""
    q = C / dP if dP != 0 else -1.0
    return float(np.cbrt(6.0 * q)) if q > 0 else float("nan")


def sigma_min_by_grid(PT_line, P_in, P_out, R_lo, R_hi, m=20001, sub=64):
    """The paper's route: sigma[R] of Eq. (21) on an R grid, minimum by a parabola.

    P_T is linearly interpolated between nodes onto a grid ``sub`` times finer
    in r and its part of the integrand, (r/R)^2 (P_out - P_T), is summed by the
    trapezoid rule; the step part (r/R)^2 (P_J - P_out) is integrated exactly
    (dP R / 3), since a sampled step makes sigma[R] saw-toothed in R.  The
    minimum of the sampled sigma[R] is refined by a parabola through the three
    lowest grid points.  Returns (R_s, sigma_s).
    """
    rmax = len(PT_line) - 1
    r = np.linspace(0.0, rmax, rmax * sub + 1)
    PT = np.interp(r, np.arange(rmax + 1), PT_line)
    Cg = np.trapezoid(r * r * (P_out - PT), r)
    Rg = np.linspace(R_lo, R_hi, m)
    sig = (P_in - P_out) * Rg / 3.0 + Cg / Rg ** 2
    k = int(np.argmin(sig))
    k = min(max(k, 1), m - 2)
    x0, x1, x2 = Rg[k - 1:k + 2]
    y0, y1, y2 = sig[k - 1:k + 2]
    den = (x0 - x1) * (x0 - x2) * (x1 - x2)
    a = (x2 * (y1 - y0) + x1 * (y0 - y2) + x0 * (y2 - y1)) / den
    b = (x2 * x2 * (y0 - y1) + x1 * x1 * (y2 - y0) + x0 * x0 * (y1 - y2)) / den
    c = (x1 * x2 * (x1 - x2) * y0 + x2 * x0 * (x2 - x0) * y1 + x0 * x1 * (x0 - x1) * y2) / den
    xs = -b / (2 * a)
    return float(xs), float(a * xs * xs + b * xs + c)


def equimolar_radius(mass, volume, n_in, n_out):
    """Sec. IV: solve M = 4 pi R^3 n_in/3 + (V - 4 pi R^3/3) n_out for R."""
    return float(np.cbrt(3.0 * (mass - volume * n_out) / (4.0 * np.pi * (n_in - n_out))))


def centre_of_mass(n, n_out):
    """Centre of mass of n - n_out, minimum-image about the centre node (x, y, z)."""
    nz, ny, nx = n.shape
    c = centre_node(n.shape)
    wgt = n - n_out
    tot = wgt.sum()
    out = []
    for axis, (L, cc) in zip((2, 1, 0), ((nx, c[0]), (ny, c[1]), (nz, c[2]))):
        d = lbm3d.min_image(np.arange(L, dtype=np.float64), cc, L)
        d[np.abs(d) == 0.5 * L] = 0.0     # even L: the plane at L/2 is both images
        shape = [1, 1, 1]
        shape[axis] = L
        out.append(cc + float((wgt * d.reshape(shape)).sum() / tot))
    return np.array(out)


def observe(f, m: lbm3d.Model, contrast0: float | None = None) -> Obs:
    """All per-run observables of the current populations."""
    n, psi, F, u = lbm3d.macroscopic(f, m)
    vecs, wts = m.stencil_arrays()
    P = pressure_tensor(n, psi, m.G, vecs, wts)
    shape = n.shape
    cx, cy, cz = centre_node(shape)
    fx, fy, fz = far_node(shape)
    n_in, n_out = float(n[cz, cy, cx]), float(n[fz, fy, fx])
    P_in, P_out = float(P[0, 0, cz, cy, cx]), float(P[0, 0, fz, fy, fx])
    dP = P_in - P_out
    nz, ny, nx = shape
    idx = (cx + np.arange(nx // 2 + 1)) % nx
    PT_line = P[1, 1, cz, cy, idx].copy()
    n_line = n[cz, cy, idx].copy()
    C, D = line_integrals(PT_line, P_out)
    R_s = surface_of_tension(dP, C)
    mass = float(n.sum())
    com = centre_of_mass(n, n_out)
    R_e = equimolar_radius(mass, float(n.size), n_in, n_out)
    max_u = float(np.sqrt((u * u).sum(axis=0)).max())
    status = 0
    if not np.isfinite(R_s):
        status |= ST_NO_MINIMUM
    if contrast0 is not None and abs(n_in - n_out) < 1e-2 * abs(contrast0):
        status |= ST_COLLAPSED
    if np.any(np.abs(com - np.array([cx, cy, cz], dtype=np.float64)) > 1e-3):
        status |= ST_OFF_CENTER
    sigma_s = 0.5 * dP * R_s if np.isfinite(R_s) else float("nan")
    return Obs(n_in, n_out, P_in, P_out, dP, mass, com, R_e, C, D, R_s, sigma_s, max_u,
               status, PT_line, n_line)


def velocity(f, m: lbm3d.Model):
    return lbm3d.macroscopic(f, m)[3]


def delta_u(u_new, u_old):
    """Sec. IV: delta u = L^-3 sum_x sum_alpha |u_new - u_old|."""
    return float(np.abs(u_new - u_old).sum() / u_new[0].size)


@dataclass
class RunResult:
    f: np.ndarray
    steps: int
    criterion: str        # "dP", "du" or "" (not converged)
    dP_hist: list
    du_hist: list


def run_to_convergence(f, m: lbm3d.Model, max_steps=50_000, check_every=2048,
                       tol_dP_rel=1e-5, tol_du=1e-12) -> RunResult:
    """Sec. IV convergence loop: check every ``check_every`` steps, stop on either test."""
    steps = 0
    obs = observe(f, m)
    dP_prev, u_prev = obs.dP, velocity(f, m)
    dP_hist, du_hist = [dP_prev], []
    crit = ""
    while steps < max_steps:
        f = lbm3d.run(f, m, check_every)
        steps += check_every
        obs = observe(f, m)
        u = velocity(f, m)
        du = delta_u(u, u_prev)
        dP_hist.append(obs.dP)
        du_hist.append(du)
        if abs(dP_prev - obs.dP) / abs(dP_prev) < tol_dP_rel:
            crit = "dP"
            break
        if du < tol_du:
            crit = "du"
            break
        dP_prev, u_prev = obs.dP, u
    return RunResult(f, steps, crit, dP_hist, du_hist)


def delta_hat(R_e, R_s, bubble):
    """Sec. IV: hat-delta_+- = +-(R_e - R_s), + for droplets, - for bubbles."""
    sign = np.where(np.asarray(bubble, dtype=bool), -1.0, 1.0)
    return sign * (np.asarray(R_e, dtype=np.float64) - np.asarray(R_s, dtype=np.float64))


def delta_hat_flat_limit(R_e, R_s, bubble):
    """hat-delta at 1/R_s -> 0: intercept of the least-squares line of hat-delta_+-
    against the signed curvature x = +-1/R_s (bubbles negative), droplets and
    bubbles in one fit."""
    R_s = np.asarray(R_s, dtype=np.float64)
    b = np.asarray(bubble, dtype=bool)
    x = np.where(b, -1.0, 1.0) / R_s
    A = np.stack([np.ones_like(x), x], axis=1)
    coef, *_ = np.linalg.lstsq(A, delta_hat(R_e, R_s, b), rcond=None)
    return float(coef[0])


def tolman_fit(R_s, sigma_s, bubble, quadratic=True):
    """Eqs. (2)/(12): least squares of sigma_s on x = 1/R_s (bubbles: x < 0).

    Returns (sigma_0, delta, c) with sigma_s = sigma_0 (1 - 2 delta x + c x^2);
    c = 0 for the linear fit.
    """
    R_s = np.asarray(R_s, dtype=np.float64)
    s = np.asarray(sigma_s, dtype=np.float64)
    x = np.where(np.asarray(bubble, dtype=bool), -1.0, 1.0) / R_s
    cols = [np.ones_like(x), x] + ([x * x] if quadratic else [])
    A = np.stack(cols, axis=1)
    coef, *_ = np.linalg.lstsq(A, s, rcond=None)
    a0, a1 = coef[0], coef[1]
    a2 = coef[2] if quadratic else 0.0
    return float(a0), float(-a1 / (2 * a0)), float(a2 / a0)
