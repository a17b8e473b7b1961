"""Seeded synthetic inputs shared by the oracle and the CUDA path in tests.

Holds none of the method's arithmetic: it only draws numbers.  A state is a
smooth radial density bump (droplet-like, or inverted for a bubble) split
over the 19 populations with random positive fractions, so it is far from
equilibrium and exercises every term of the step.
"""
from __future__ import annotations

import numpy as np


def radial_bump(shape_zyx, center_xyz, radius, inner, outer, edge=1.5):
    """inner inside a sphere, outer outside, logistic edge; periodic distances."""
    nz, ny, nx = shape_zyx
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = []
    for c, L, a in ((center_xyz[0], nx, x), (center_xyz[1], ny, y), (center_xyz[2], nz, z)):
        t = np.abs(a - c)
        d.append(np.minimum(t, L - t))
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    s = 1.0 / (1.0 + np.exp((r - radius) / edge))
    return outer + (inner - outer) * s


def random_populations(shape_zyx, seed, inner=1.7, outer=0.25, radius=None, noise=0.05):
    """[19, z, y, x] positive populations whose sum is a radial bump times (1 + noise)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    radius = min(nx, ny, nz) / 4.0 if radius is None else radius
    n = radial_bump(shape_zyx, (nx // 2, ny // 2, nz // 2), radius, inner, outer)
    n = n * (1.0 + noise * rng.uniform(-1.0, 1.0, size=n.shape))
    frac = rng.uniform(0.5, 1.5, size=(19,) + tuple(shape_zyx))
    frac[0] *= 6.0                       # heavier rest population
    frac /= frac.sum(axis=0, keepdims=True)
    return frac * n[None]


def random_density(shape_zyx, seed, inner=1.7, outer=0.25, radius=None, noise=0.02):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    radius = min(nx, ny, nz) / 4.0 if radius is None else radius
    n = radial_bump(shape_zyx, (nx // 2, ny // 2, nz // 2), radius, inner, outer)
    return n * (1.0 + noise * rng.uniform(-1.0, 1.0, size=n.shape))
