"""D3Q19 Shan-Chen BGK + Guo-forcing step, FP64 (oracle, test infrastructure).

Paper, Sec. II.  One time step, in the paper's order:

  n = sum_i f_i,  n u = sum_i xi_i f_i                      (moments, Sec. II)
  F^mu = -G c_s^2 psi(x) sum_a W(|xi_a|^2) psi(x+xi_a) xi_a^mu        Eq. (8)
  u_eq = (sum_i xi_i f_i)/n + F/(2n)                                  Eq. (7)
  f_i^eq = w_i n [1 + xi.u/c_s^2 + (xi.u)^2/(2 c_s^4) - u.u/(2 c_s^2)] Eq. (6)
  F_i = (1 - 1/(2 tau)) w_i [xi_i.F/c_s^2
                              + ((xi_i.u)(xi_i.F) - c_s^2 u.F)/c_s^4]  Eq. (5)
  Omega_i = -(f_i - f_i^eq)/tau                                       Eq. (4)
  f_i(x + xi_i, t+1) = f_i(x, t) + Omega_i + F_i                      Eq. (3)

on a box periodic in all three axes.  Reading: Eq. (6) as printed lacks the
factor 1/2 on (xi.u)^2/c_s^4; the second-order Hermite equilibrium (the one
whose second moment is n c_s^2 delta + n u u) has it, and it is used here.
All velocities that enter Eqs. (5) and (6) are u_eq of Eq. (7).

Arrays: populations f[i, z, y, x] (i in the D3Q19 order of ``lattice``),
fields [z, y, x]; shifts by np.roll.

Initial condition (Sec. IV, Eq. (23)): radial tanh profile around a centre
node, f = f^eq(n, u = 0).  Reading: the paper's profile has unit width; a
width w enters as tanh((r - R)/w) (w = 1 is the paper's).  r is the
minimum-image distance on the periodic box.

Parity: mass and total momentum conservation, the uniform-field fixed point,
the exact reduction to the 1-D flat run, cubic symmetry and a node-by-node
evaluation on a tiny box pin the step; the transient is pinned by linear
acoustics of a uniform phase (a small standing wave oscillates at
c^2 = dP/dn of Eq. (10) and decays at the lattice viscosity c_s^2 (tau - 1/2),
both closed forms, to 0.1-0.3%).  The paper prints no 3-D field values.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import eos as _eos
from . import lattice as _lat

CS2 = 1.0 / 3.0
XI = _lat.D3Q19                       # [19, 3] (x, y, z)
W = _lat.d3q19_weights()              # [19]


@dataclass
class Model:
    """Parameters of one lattice: relaxation time, coupling, psi and stencil."""
    tau: float = 1.0
    G: float = -5.0
    eos: _eos.EOS = field(default_factory=_eos.EOS)
    stencil: str = "E4"

    def stencil_arrays(self):
        return _lat.stencil(self.stencil)


def shift(field: np.ndarray, xi) -> np.ndarray:
    """field(x + xi) on the periodic box; field indexed [z, y, x]."""
    return np.roll(field, shift=(-int(xi[2]), -int(xi[1]), -int(xi[0])), axis=(0, 1, 2))


def density(f: np.ndarray) -> np.ndarray:
    """n = sum_i f_i."""
    return f.sum(axis=0)


def momentum(f: np.ndarray) -> np.ndarray:
    """sum_i xi_i f_i, shape [3, z, y, x]."""
    return np.einsum("ia,izyx->azyx", XI.astype(np.float64), f)


def sc_force(psi: np.ndarray, G: float, vectors: np.ndarray, weights: np.ndarray) -> np.ndarray:
    """Eq. (8): F^mu = -G c_s^2 psi(x) sum_a W_a psi(x + xi_a) xi_a^mu, shape [3, ...]."""
    acc = np.zeros((3,) + psi.shape)
    for xi, w in zip(vectors, weights):
        nb = shift(psi, xi)
        for mu in range(3):
            if xi[mu] != 0:
                acc[mu] += w * xi[mu] * nb
    return -G * CS2 * psi * acc


def equilibrium(n: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Eq. (6) with the Hermite 1/2 (module doc): f_i^eq, shape [19, ...]."""
    uu = (u * u).sum(axis=0)
    feq = np.empty((19,) + n.shape)
    for i in range(19):
        eu = sum(XI[i, a] * u[a] for a in range(3))
        feq[i] = W[i] * n * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2))
    return feq


def guo_source(u: np.ndarray, F: np.ndarray, tau: float) -> np.ndarray:
    """Eq. (5): F_i = (1 - 1/2tau) w_i [xi.F/c_s^2 + ((xi.u)(xi.F) - c_s^2 u.F)/c_s^4]."""
    uF = (u * F).sum(axis=0)
    out = np.empty((19,) + uF.shape)
    for i in range(19):
        eu = sum(XI[i, a] * u[a] for a in range(3))
        eF = sum(XI[i, a] * F[a] for a in range(3))
        out[i] = (1.0 - 0.5 / tau) * W[i] * (eF / CS2 + (eu * eF - CS2 * uF) / (CS2 * CS2))
    return out


def macroscopic(f: np.ndarray, m: Model):
    """(n, psi, F, u_eq) of the current populations (Eqs. (7), (8))."""
    n = density(f)
    psi = _eos.psi(n, m.eos, m.G)
    vecs, wts = m.stencil_arrays()
    F = sc_force(psi, m.G, vecs, wts)
    u = (momentum(f) + 0.5 * F) / n
    return n, psi, F, u


def step(f: np.ndarray, m: Model) -> np.ndarray:
    """One time step, Eq. (3): collide (Eqs. (4)-(8)) then stream."""
    n, psi, F, u = macroscopic(f, m)
    feq = equilibrium(n, u)
    post = f - (f - feq) / m.tau + guo_source(u, F, m.tau)
    out = np.empty_like(f)
    for i in range(19):
        out[i] = np.roll(post[i], shift=(int(XI[i, 2]), int(XI[i, 1]), int(XI[i, 0])), axis=(0, 1, 2))
    return out


def run(f: np.ndarray, m: Model, steps: int) -> np.ndarray:
    for _ in range(steps):
        f = step(f, m)
    return f


def min_image(coord: np.ndarray, c: float, L: int) -> np.ndarray:
    """Minimum-image displacement coord - c on a periodic axis of length L, in [-L/2, L/2)."""
    return np.mod(coord - c + 0.5 * L, L) - 0.5 * L


def drop_density(shape_zyx, center_xyz, R, n_in, n_out, width=1.0) -> np.ndarray:
    """Eq. (23): n(r) = (n_in + n_out)/2 - (n_in - n_out)/2 tanh((r - R)/width)."""
    nz, ny, nx = shape_zyx
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dx = min_image(x.astype(np.float64), center_xyz[0], nx)
    dy = min_image(y.astype(np.float64), center_xyz[1], ny)
    dz = min_image(z.astype(np.float64), center_xyz[2], nz)
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    return 0.5 * (n_in + n_out) - 0.5 * (n_in - n_out) * np.tanh((r - R) / width)


def init_from_density(n: np.ndarray) -> np.ndarray:
    """f = f^eq(n, u = 0) (Sec. IV: the fluid starts at rest)."""
    return equilibrium(n, np.zeros((3,) + n.shape))
