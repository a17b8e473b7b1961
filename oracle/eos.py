"""Pseudopotentials, bulk pressure, critical coupling, coexistence (oracle).

Paper: Sec. II, Eq. (10): P(n) = n c_s^2 + (G c_s^2 e_2 / 2) psi(n)^2 with
e_2 = 1; phase coexistence needs G < G_c, the coupling where dP/dn and
d^2P/dn^2 vanish together.  Sec. IV uses psi = exp(-1/n) and
psi = 1 - exp(-n) and prints G_c c_s^2 = -2.463 and -1.333 for them.

A third, Carnahan-Starling-mapped pseudopotential (a = 1, b = 4, R = 1,
G = -1) is included for the wider-stencil workload:
psi = sqrt(2 (p_CS(n) - n c_s^2) / (G c_s^2)), so that Eq. (10) returns
p_CS exactly.

Coexistence: for a flat interface the lattice pressure tensor of Eq. (9)
keeps P_N constant.  To leading order in gradients Eq. (9) gives
P_N = P(n) + (G c_s^2 / 4) psi psi''; multiplying P_N = p_0 by psi'/psi and
integrating across the interface gives the construction solved here:
    P(n_g) = P(n_l) = p_0,   int_{n_g}^{n_l} (p_0 - P(n)) psi'(n)/psi(n) dn = 0.
It is the continuum limit of the lattice run in ``flat`` (pinned against it
to the size of the neglected higher-order terms).

Parity: G_c pinned to the paper's printed values; P(n) pinned by the
uniform-field pressure tensor; coexistence pinned by the lattice flat run.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy import integrate, optimize

CS2 = 1.0 / 3.0

KINDS = ("exp_inv", "one_minus_exp", "cs")


@dataclass(frozen=True)
class EOS:
    """psi kind plus the Carnahan-Starling constants (used by kind 'cs' only)."""
    kind: str = "one_minus_exp"
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    T: float = 0.0


def p_cs(n, eos: EOS):
    """Carnahan-Starling pressure  n R T (1+e+e^2-e^3)/(1-e)^3 - a n^2, e = b n / 4."""
    e = eos.b * n / 4.0
    return n * eos.R * eos.T * (1.0 + e + e * e - e ** 3) / (1.0 - e) ** 3 - eos.a * n * n


def dp_cs(n, eos: EOS):
    """d p_CS / dn (derivative of the expression above, by hand)."""
    e = eos.b * n / 4.0
    g = (1.0 + e + e * e - e ** 3) / (1.0 - e) ** 3
    dg_de = ((1.0 + 2 * e - 3 * e * e) * (1.0 - e) + 3 * (1.0 + e + e * e - e ** 3)) / (1.0 - e) ** 4
    return eos.R * eos.T * (g + n * dg_de * eos.b / 4.0) - 2.0 * eos.a * n


def psi(n, eos: EOS, G: float):
    """psi(n) (Sec. II below Eq. (8); Sec. IV for the two closed forms)."""
    if eos.kind == "exp_inv":
        return np.exp(-1.0 / n)
    if eos.kind == "one_minus_exp":
        return 1.0 - np.exp(-n)
    if eos.kind == "cs":
        return np.sqrt(2.0 * (p_cs(n, eos) - n * CS2) / (G * CS2))
    raise ValueError(eos.kind)


def dpsi_over_psi(n, eos: EOS, G: float):
    """psi'(n)/psi(n)."""
    if eos.kind == "exp_inv":
        return 1.0 / (n * n)
    if eos.kind == "one_minus_exp":
        return np.exp(-n) / (1.0 - np.exp(-n))
    if eos.kind == "cs":
        return (dp_cs(n, eos) - CS2) / (2.0 * (p_cs(n, eos) - n * CS2))
    raise ValueError(eos.kind)


def bulk_pressure(n, eos: EOS, G: float, e2: float = 1.0):
    """Eq. (10):  P(n) = n c_s^2 + G c_s^2 e_2 psi(n)^2 / 2."""
    return n * CS2 + 0.5 * G * CS2 * e2 * psi(n, eos, G) ** 2


def _d1(fun, n, h=1e-5):
    return (fun(n + h) - fun(n - h)) / (2 * h)


def critical_point(eos: EOS):
    """(n_c, G_c) with dP/dn = d^2P/dn^2 = 0 (Sec. II below Eq. (10)).

    psi kinds only (the CS kind has G fixed; see ``cs_critical_temperature``).
    dP/dn = c_s^2 + G c_s^2 psi psi'  and  d^2P/dn^2 = G c_s^2 (psi'^2 + psi psi''),
    so n_c is the root of psi'^2 + psi psi'' (G-independent) and then
    G_c = -1 / (psi psi')(n_c).  Derivatives of psi by central differences.
    """
    if eos.kind == "cs":
        raise ValueError("use cs_critical_temperature")
    f = lambda n: psi(n, eos, 0.0)
    d1 = lambda n: _d1(f, n)
    d2 = lambda n: (f(n + 1e-4) - 2 * f(n) + f(n - 1e-4)) / 1e-8
    curv = lambda n: d1(n) ** 2 + f(n) * d2(n)
    grid = np.linspace(0.05, 5.0, 2000)
    vals = np.array([curv(x) for x in grid])
    k = int(np.nonzero(np.sign(vals[:-1]) != np.sign(vals[1:]))[0][0])
    n_c = optimize.brentq(curv, grid[k], grid[k + 1], xtol=1e-14)
    G_c = -1.0 / (f(n_c) * d1(n_c))
    return n_c, G_c


def cs_critical_temperature(eos: EOS):
    """(n_c, T_c) of the Carnahan-Starling EOS: dp/dn = d^2p/dn^2 = 0."""
    def eqs(x):
        n, T = x
        e = EOS("cs", eos.a, eos.b, eos.R, T)
        return [dp_cs(n, e), _d1(lambda m: dp_cs(m, e), n)]
    n_c, T_c = optimize.fsolve(eqs, [0.13, 0.094], xtol=1e-14)
    return float(n_c), float(T_c)


def _spinodals(eos, G, lo, hi):
    """(n_sg, n_sl): local maximum (gas spinodal) and minimum (liquid) of P(n)."""
    grid = np.linspace(lo, hi, 20000)
    P = bulk_pressure(grid, eos, G)
    dP = np.diff(P)
    turn = np.nonzero(np.sign(dP[:-1]) != np.sign(dP[1:]))[0]
    if len(turn) < 2:
        raise ValueError("no van der Waals loop: G above G_c")
    a, b = grid[turn[0]], grid[turn[0] + 2]
    n_sg = optimize.minimize_scalar(lambda n: -bulk_pressure(n, eos, G), bounds=(a, b),
                                    method="bounded", options={"xatol": 1e-13}).x
    a, b = grid[turn[1]], grid[turn[1] + 2]
    n_sl = optimize.minimize_scalar(lambda n: bulk_pressure(n, eos, G), bounds=(a, b),
                                    method="bounded", options={"xatol": 1e-13}).x
    return n_sg, n_sl


def coexistence(eos: EOS, G: float, lo: float = 1e-3, hi: float = 4.0):
    """(n_g, n_l, p_0) from the psi'/psi construction stated in the module doc.

    p_0 is found by bisection between the spinodal pressures; for each trial
    p_0 the gas root (on the rising branch below the gas spinodal) and the
    liquid root (on the rising branch above the liquid spinodal) bound the
    area integral.
    """
    n_sg, n_sl = _spinodals(eos, G, lo, hi)
    P = lambda n: bulk_pressure(n, eos, G)

    def roots(p0):
        ng = optimize.brentq(lambda n: P(n) - p0, lo, n_sg, xtol=1e-15, rtol=1e-15)
        nl = optimize.brentq(lambda n: P(n) - p0, n_sl, hi, xtol=1e-15, rtol=1e-15)
        return ng, nl

    def area(p0):
        ng, nl = roots(p0)
        val, _ = integrate.quad(lambda n: (p0 - P(n)) * dpsi_over_psi(n, eos, G),
                                ng, nl, epsabs=1e-14, epsrel=1e-13, limit=400)
        return val

    p_hi, p_lo = P(n_sg), max(P(n_sl), P(lo))
    span = p_hi - p_lo
    a_lo, a_hi = area(p_lo + 1e-10 * span), area(p_hi - 1e-10 * span)
    if np.sign(a_lo) == np.sign(a_hi):
        raise ValueError("psi'/psi construction has no root between the spinodal pressures")
    p0 = optimize.brentq(area, p_lo + 1e-10 * span, p_hi - 1e-10 * span, xtol=1e-16, rtol=1e-15)
    ng, nl = roots(p0)
    return ng, nl, p0
