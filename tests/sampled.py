"""One-step oracle values at sampled nodes of a large periodic box.

The update of Eqs. (3)-(8) at node c reads the populations of c's neighbours
(streaming) and the psi of their force-stencil neighbours: nothing farther than
R + 1 from c, R the stencil radius.  So the oracle's step on the periodic
window of half-width R + 2 around c gives c's post-step populations (up to the
rounding order of numpy's reductions), whatever the window's own wrap does at
its edges.  This lets boxes too large for
a whole-field oracle step be checked node by node.
"""
from __future__ import annotations

import numpy as np

from oracle import lbm3d


def window(f: np.ndarray, c_zyx, h: int) -> np.ndarray:
    """[19, 2h+1, 2h+1, 2h+1] periodic window of f[19, z, y, x] centred on c."""
    _, nz, ny, nx = f.shape
    iz = (np.arange(-h, h + 1) + c_zyx[0]) % nz
    iy = (np.arange(-h, h + 1) + c_zyx[1]) % ny
    ix = (np.arange(-h, h + 1) + c_zyx[2]) % nx
    return f[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]]


def step_at(f: np.ndarray, m: lbm3d.Model, c_zyx) -> np.ndarray:
    """Oracle post-step populations [19] at node c of f (one step of Eq. (3))."""
    R = max(int(np.max(np.abs(v))) for v in m.stencil_arrays()[0])
    h = R + 2
    return lbm3d.step(window(f, c_zyx, h), m)[:, h, h, h]


def sample_nodes(shape_zyx, count: int, seed: int) -> list[tuple[int, int, int]]:
    """count seeded random nodes plus the corners and the first/last row of a
    32 x 8 tile column (tile and wrap edges)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    out = {(0, 0, 0), (nz - 1, ny - 1, nx - 1), (0, ny - 1, 31 % nx), (nz // 2, 7 % ny, 32 % nx),
           (nz - 1, 8 % ny, nx - 1), (nz // 3, ny // 2, 0)}
    while len(out) < count:
        out.add((int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx))))
    return sorted(out)
