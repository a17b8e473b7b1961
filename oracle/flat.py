"""Flat-interface run and sigma_0 (oracle, test infrastructure).

Paper, Sec. IV: the flat-interface simulations run on a 2-D strip
(D2Q9, L_x = 100, L_y = 4, forcing weights projected to W(1) = 1/3,
W(2) = 1/12) initialised with the strip profile of Eq. (24) (gas strip of
width L_x/2 centred at x_0 = L_x/2), and sigma_0 is the integral of
P_N - P_T over the right half, Eq. (25).  Their bulk densities n_g, n_l
initialise the droplets and bubbles (Sec. IV, below Eq. (23)).

A field that varies only along x makes the D3Q19 (or D2Q9) dynamics of
Sec. II collapse exactly onto D1Q3: the populations with the same xi_x sum
to D1Q3 populations with weights (2/3, 1/6, 1/6), the equilibrium and Guo
term depend on xi only through xi_x (u and F point along x), and only the
x-shift of streaming changes anything.  The force of Eq. (8) on such a field
is F^x(x) = -G c_s^2 psi(x) sum_a W_a psi(x + xi_a^x) xi_a^x over the 3-D
stencil; for E4 the weight of each x-neighbour lumps to W(1) + 4 W(2) = 1/2,
the same as the paper's D2Q9 projection W(1) + 2 W(2) = 1/2.  This module
runs that exact 1-D reduction (tests check it against the 3-D oracle).

The lattice pressure tensor (Eq. (9)) on the flat field gives
    P_N(x) = P^xx = n c_s^2 + (G c_s^2/2) psi(x) sum_a W_a psi(x + xi_a^x) (xi_a^x)^2
    P_T(x) = P^yy = n c_s^2 + (G c_s^2/2) psi(x) sum_a W_a psi(x + xi_a^x) (xi_a^y)^2.

Convergence: the run stops when, over one check interval, the bulk
densities move by less than ``tol_n`` and P_N is flat to ``tol_pn``.

Parity: pinned by the paper's statement that P_N is constant to machine
precision (Sec. II below Eq. (9)), by zero velocity at equilibrium, and by
the continuum coexistence construction of ``eos``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import eos as _eos
from . import lattice as _lat

CS2 = 1.0 / 3.0
XI1 = np.array([0, 1, -1])
W1 = _lat.d1q3_weights()


def strip_density(Lx: int, n_l: float, n_g: float, x0: float | None = None,
                  w: float | None = None) -> np.ndarray:
    """Eq. (24): liquid outside, gas strip of width w centred at x0."""
    x = np.arange(Lx, dtype=np.float64)
    x0 = 0.5 * Lx if x0 is None else x0
    w = 0.5 * Lx if w is None else w
    return (0.5 * (n_l + n_g) - 0.5 * (n_l - n_g) * np.tanh(x - (x0 - 0.5 * w))
            + 0.5 * (n_l - n_g) * (np.tanh(x - (x0 + 0.5 * w)) + 1.0))


def _shift(a, s):
    """a(x + s) on the periodic 1-D lattice (last axis)."""
    return np.roll(a, -int(s), axis=-1)


def force_x(psi, G, vectors, weights):
    acc = np.zeros_like(psi)
    for xi, w in zip(vectors, weights):
        if xi[0] != 0:
            acc += w * xi[0] * _shift(psi, xi[0])
    return -G * CS2 * psi * acc


def pressure_NT(n, psi, G, vectors, weights):
    """(P_N, P_T) of Eq. (9) on a field varying only along x."""
    sN = np.zeros_like(psi)
    sT = np.zeros_like(psi)
    for xi, w in zip(vectors, weights):
        nb = _shift(psi, xi[0])
        sN += w * xi[0] * xi[0] * nb
        sT += w * xi[1] * xi[1] * nb
    return n * CS2 + 0.5 * G * CS2 * psi * sN, n * CS2 + 0.5 * G * CS2 * psi * sT


def step(f, G, tau, eos, vectors, weights):
    """One D1Q3 step of Eqs. (3)-(8); f has shape [3, ..., Lx]."""
    n = f.sum(axis=0)
    psi = _eos.psi(n, eos, G)
    F = force_x(psi, G, vectors, weights)
    u = (f[1] - f[2] + 0.5 * F) / n
    out = np.empty_like(f)
    for i in range(3):
        eu = XI1[i] * u
        feq = W1[i] * n * (1.0 + eu / CS2 + eu * eu / (2 * CS2 * CS2) - u * u / (2 * CS2))
        eF = XI1[i] * F
        Fi = (1.0 - 0.5 / tau) * W1[i] * (eF / CS2 + (eu * eF - CS2 * u * F) / (CS2 * CS2))
        post = f[i] - (f[i] - feq) / tau + Fi
        out[i] = np.roll(post, int(XI1[i]), axis=-1)
    return out


@dataclass
class FlatResult:
    n: np.ndarray          # final density profile
    n_g: float
    n_l: float
    sigma0: float          # Eq. (25)
    pn_spread: float       # max P_N - min P_N
    max_u: float
    steps: int
    converged: bool


def run_flat(G: float, eos: _eos.EOS, stencil: str = "E4", tau: float = 1.0, Lx: int = 100,
             n_l0: float | None = None, n_g0: float | None = None, check_every: int = 2048,
             max_steps: int = 600_000, tol_n: float = 1e-12, tol_pn: float = 1e-13) -> FlatResult:
    """Run the flat strip to its steady state and measure n_g, n_l, sigma_0."""
    vectors, weights = _lat.stencil(stencil)
    if n_l0 is None or n_g0 is None:
        n_g0, n_l0, _ = _eos.coexistence(eos, G)
    n = strip_density(Lx, n_l0, n_g0)
    f = np.stack([W1[i] * n for i in range(3)])
    i_gas, i_liq = Lx // 2, 0          # strip centre (gas) and the far edge (liquid)
    prev = None
    steps = 0
    converged = False
    while steps < max_steps:
        for _ in range(check_every):
            f = step(f, G, tau, eos, vectors, weights)
        steps += check_every
        n = f.sum(axis=0)
        psi = _eos.psi(n, eos, G)
        PN, _ = pressure_NT(n, psi, G, vectors, weights)
        cur = np.array([n[i_gas], n[i_liq]])
        if prev is not None and np.max(np.abs(cur - prev)) < tol_n and np.ptp(PN) < tol_pn:
            converged = True
            break
        prev = cur
    n = f.sum(axis=0)
    psi = _eos.psi(n, eos, G)
    PN, PT = pressure_NT(n, psi, G, vectors, weights)
    F = force_x(psi, G, vectors, weights)
    u = (f[1] - f[2] + 0.5 * F) / n
    half = np.arange(Lx // 2, Lx)
    # Eq. (25) over [L_x/2, L_x): trapezoid on the nodes, closing the periodic
    # interval with the node at L_x = node 0 (bulk liquid there)
    g = np.append((PN - PT)[half], (PN - PT)[0])
    sigma0 = float(np.trapezoid(g, dx=1.0))
    return FlatResult(n=n, n_g=float(n[i_gas]), n_l=float(n[i_liq]), sigma0=sigma0,
                      pn_spread=float(np.ptp(PN)), max_u=float(np.max(np.abs(u))),
                      steps=steps, converged=converged)
