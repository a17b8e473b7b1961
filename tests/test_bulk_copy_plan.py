"""Host-side check of the row-bulk step kernel's copy plan (lbm_kernels_bulk.cuh).

A bulk copy with a misaligned address or size is a fault on the GPU, so the plan
is replayed here on the CPU for many box sizes and tiles: every copy must start
and end on 16-byte boundaries in global and shared memory, stay inside the
population buffer and its stage, the byte count posted to the stage's mbarrier
must equal the bytes copied, and every element the density and collision phases
read must hold the pulled population they expect.
"""
import itertools

import numpy as np
import pytest

from oracle import lattice as L

XI = L.D3Q19
Q = 19
APRON = 4


def wrap(g, n):
    return g + n if g < 0 else (g - n if g >= n else g)


def plan(nx, ny, nz, BX, BY, R, elem, x0, y0, z):
    """(copies, rows, stage_bytes) exactly as the kernel issues them for one plane."""
    XW = BX + 2 * APRON
    PY = BY + 2 * R
    N = nx * ny * nz
    h = min(BY, ny - y0)
    rows = h + 2 * R
    xa = x0 - APRON
    copies = []   # (smem_elem_offset, global_elem_offset, n_elems)
    for r in range(Q * rows):
        i, jy = divmod(r, rows)
        gy = wrap(wrap(y0 - R + jy, ny) - XI[i, 1], ny)
        gz = wrap(z - XI[i, 2], nz)
        row = i * N + (gz * ny + gy) * nx
        sp = (i * PY + jy) * XW
        if xa < 0:
            copies.append((sp, row + nx + xa, -xa))
            copies.append((sp - xa, row, XW + xa))
        elif xa + XW > nx:
            n1 = nx - xa
            copies.append((sp, row + xa, n1))
            copies.append((sp + n1, row, XW - n1))
        else:
            copies.append((sp, row + xa, XW))
    return copies, rows, Q * rows * XW * elem


CASES = [(nx, ny, nz, BX, BY, R, elem)
         for (nx, ny, nz) in [(128, 128, 128), (40, 12, 9), (72, 72, 72), (44, 20, 6), (160, 24, 7),
                              (48, 40, 36)]
         for (BX, BY) in [(32, 8), (32, 4), (64, 4)]
         for R in (1, 2)
         for elem in (4, 8)
         if nx % 4 == 0 and nx >= BX + 2 * APRON]


@pytest.mark.parametrize("nx,ny,nz,BX,BY,R,elem", CASES)
def test_bulk_copy_plan(nx, ny, nz, BX, BY, R, elem):
    N = nx * ny * nz
    XW = BX + 2 * APRON
    PY = BY + 2 * R
    stage_elems = Q * PY * XW
    rng = np.random.default_rng(nx * 7 + ny)
    src = np.arange(Q * N)           # element ids stand in for values
    for x0 in range(0, nx, BX):
        for y0 in range(0, ny, BY):
            z = int(rng.integers(nz))
            copies, rows, stage_bytes = plan(nx, ny, nz, BX, BY, R, elem, x0, y0, z)
            assert sum(n for _, _, n in copies) * elem == stage_bytes
            stage = np.full(stage_elems, -1)
            for sp, gp, n in copies:
                assert (sp * elem) % 16 == 0 and (gp * elem) % 16 == 0 and (n * elem) % 16 == 0
                assert n > 0 and 0 <= gp and gp + n <= Q * N
                assert 0 <= sp and sp + n <= stage_elems
                assert np.all(stage[sp:sp + n] == -1)      # no overlapping writes
                stage[sp:sp + n] = src[gp:gp + n]
            w = min(BX, nx - x0)
            for jy in range(rows):
                for jx in range(w + 2 * R):
                    for i in range(Q):
                        col = jx + APRON - R - XI[i, 0]
                        assert 0 <= col < XW
                        got = stage[(i * PY + jy) * XW + col]
                        gx = wrap(wrap(x0 - R + jx, nx) - XI[i, 0], nx)
                        gy = wrap(wrap(y0 - R + jy, ny) - XI[i, 1], ny)
                        gz = wrap(z - XI[i, 2], nz)
                        assert got == i * N + (gz * ny + gy) * nx + gx
