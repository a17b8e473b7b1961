"""Host-side replay of the TMA step kernel's copy plan (lbm_kernels_tma.cuh, kind 7).

For boxes with every kind of tile (the four periodic corners, edges, interior,
a ragged last column), one plane of one item is replayed on the CPU exactly as
the kernel computes it:
  * the tensor boxes (main XW x PY box per population, wrapped-row boxes of the
    first / last row of tiles): x origin on a 16-byte boundary, shared-memory
    destinations on 128-byte boundaries and inside their regions, wrapped-row
    boxes reading in-range rows only, no two boxes writing the same element, and
    the mbarrier's expected byte count equal to the bytes the boxes deliver
    (out-of-range elements of a box read as zero);
  * the fix-ups the threads write after the mbarrier wait (16-byte chunks from
    the wrapped-row buffer, x-wrapped cells from global memory): inside the
    stage, on disjoint cells;
  * every staged value the density pass reads (own node and halo ring) then
    holds the pulled population f_i(x - xi_i) of its padded node, with the
    periodic wrap in x, y and z.
A misaligned or out-of-range tensor copy faults the GPU, so these are checked
here before any launch.
"""
import numpy as np
import pytest

from oracle import lattice as L

XI = L.D3Q19
Q = 19
CX, CY, CZ = XI[:, 0], XI[:, 1], XI[:, 2]


def wrap(g, n):
    return g + n if g < 0 else (g - n if g >= n else g)


def align128(b):
    return (b + 127) // 128 * 128


def shape(BX, BY, R):
    PX, PY = BX + 2 * R, BY + 2 * R
    XW = BX + 8
    POP = (PY * XW + 31) // 32 * 32
    NT = BX * BY
    xpops = sum(1 for c in CX if R + int(c) > 0)
    return dict(PX=PX, PY=PY, NPAD=PX * PY, NT=NT, NH=PX * PY - NT, APRON=4, XW=XW, POP=POP,
                NR=2 * R + 2, LIST=Q * R, XPOPS=xpops, XSLOT=align128(4 * PY * 4))


def wrap_rows(R, side, i):
    return max(R + side * int(CY[i]), 0)


def wrap_cols(R, side, i):
    return max(R + side * int(CX[i]), 0)


def wrap_offset(R, XW, side, i):
    return sum(align128(wrap_rows(R, side, j) * XW * 4) for j in range(i))


def wrap_bytes(R, XW):
    return max(wrap_offset(R, XW, 1, Q), wrap_offset(R, XW, -1, Q))


def side_list(rows, side, R=1):
    """The kernel's packed list: (population, index) per wrapped row (rows) or x cell."""
    out = []
    for i in range(Q):
        for m in range(wrap_rows(R, side, i) if rows else wrap_cols(R, side, i)):
            out.append((i, m))
    return out


def corner_list(xside, yside, R=1):
    return [(i, v, m) for i in range(Q) for v in range(wrap_rows(R, yside, i))
            for m in range(wrap_cols(R, xside, i))]


def xslot(R, side, i, XSLOT):
    return XSLOT * sum(1 for j in range(i) if wrap_cols(R, side, j) > 0)


def halo_node_rows(h, BX, BY, R):
    PX, PY = BX + 2 * R, BY + 2 * R
    if h < 32:
        return h
    h -= 32
    if h < 32:
        return (PY - 1) * PX + h
    h -= 32
    if h < PX - 32:
        return 32 + h
    h -= PX - 32
    if h < PX - 32:
        return (PY - 1) * PX + 32 + h
    h -= PX - 32
    row, c = 1 + h // 2, h % 2
    return row * PX + (0 if c == 0 else PX - 1)


def value(nx, ny, nz, x, y, z, i):
    """Element (x, y, z) of population plane i as a unique positive id."""
    return 1 + i * nx * ny * nz + (z * ny + y) * nx + x


def replay(nx, ny, nz, BX, BY, R, x0, y0, z):
    sh = shape(BX, BY, R)
    PX, PY, XW, POP, APRON, NT = sh["PX"], sh["PY"], sh["XW"], sh["POP"], sh["APRON"], sh["NT"]
    w = min(BX, nx - x0)
    stage = np.zeros(Q * POP, dtype=np.int64)
    owner = np.full(Q * POP, -1, dtype=np.int64)          # which box wrote each element
    wbuf_bytes = wrap_bytes(R, XW)
    wbuf = np.zeros(wbuf_bytes // 4, dtype=np.int64)
    wowner = np.full(wbuf_bytes // 4, -1, dtype=np.int64)
    xbuf = np.zeros(sh["XPOPS"] * sh["XSLOT"] // 4, dtype=np.int64)
    xowner = np.full(xbuf.size, -1, dtype=np.int64)
    yside = 1 if y0 == 0 else (-1 if y0 + BY == ny else 0)
    xside = 1 if x0 < R + 1 else (-1 if x0 + w + R + 1 > nx else 0)
    delivered = 0
    nbox = 0

    def box(dst_arr, own, dst_off_bytes, region_end_bytes, bx_, by_, bw, h, zs, i, wrapped):
        nonlocal delivered, nbox
        assert (bx_ * 4) % 16 == 0, "tensor box x origin off a 16-byte boundary"
        assert (bw * 4) % 16 == 0, "box width not a multiple of 16 bytes"
        assert dst_off_bytes % 128 == 0, "shared destination off a 128-byte boundary"
        assert dst_off_bytes + h * bw * 4 <= region_end_bytes, "box overruns its region"
        if wrapped:
            assert 0 <= by_ and by_ + h <= ny, "wrapped-row box reads rows out of range"
        base = dst_off_bytes // 4
        for r in range(h):
            for c in range(bw):
                x, y = bx_ + c, by_ + r
                v = value(nx, ny, nz, x, y, zs, i) if (0 <= x < nx and 0 <= y < ny) else 0
                k = base + r * bw + c
                assert own[k] == -1, "two boxes write one element"
                own[k] = nbox
                dst_arr[k] = v
        delivered += h * bw * 4
        nbox += 1

    for i in range(Q):
        zs = wrap(z - int(CZ[i]), nz)
        yb = y0 - R - int(CY[i])
        box(stage, owner, i * POP * 4, (i + 1) * POP * 4, x0 - APRON, yb, XW, PY, zs, i, False)
        if yside != 0:
            k = wrap_rows(R, yside, i)
            if k > 0:
                off = wrap_offset(R, XW, yside, i)
                box(wbuf, wowner, off, off + align128(k * XW * 4), x0 - APRON, ny - k if yside > 0 else 0, XW, k,
                    zs, i, True)
        if xside != 0 and wrap_cols(R, xside, i) > 0:
            off = xslot(R, xside, i, sh["XSLOT"])
            xb = nx - 4 if xside > 0 else 0
            assert 0 <= xb and xb + 4 <= nx
            box(xbuf, xowner, off, off + sh["XSLOT"], xb, yb, 4, PY, zs, i, False)
    expect = 4 * (XW * (Q * PY + (sh["LIST"] if yside != 0 else 0)) + (4 * PY * sh["XPOPS"] if xside != 0 else 0))
    assert delivered == expect, (delivered, expect)
    assert wbuf_bytes % 128 == 0 and xbuf.size * 4 == sh["XPOPS"] * sh["XSLOT"]

    # thread fix-ups, after the mbarrier wait (fix_stage)
    written = np.zeros(Q * POP, dtype=bool)
    XC = XW // 4
    rows = side_list(True, yside) if yside else []
    cols = side_list(False, xside) if xside else []
    for tid in range(NT):
        if yside != 0 and tid < sh["LIST"] * XC:
            rho, c4 = tid // XC, tid % XC
            pop, v = rows[rho]
            xs = x0 - APRON + 4 * c4
            if xs >= 0 and xs + 4 <= nx:
                k = wrap_rows(R, yside, pop)
                frm = wrap_offset(R, XW, yside, pop) // 4 + v * XW + 4 * c4
                to = pop * POP + (v if yside > 0 else PY - k + v) * XW + 4 * c4
                assert frm % 4 == 0 and to % 4 == 0, "16-byte chunk copies"
                assert frm + 4 <= wbuf.size and to + 4 <= (pop + 1) * POP
                assert not written[to:to + 4].any(), "two fix-ups write one cell"
                written[to:to + 4] = True
                stage[to:to + 4] = wbuf[frm:frm + 4]
        if xside != 0 and tid < PY * sh["LIST"]:
            r, j = tid // sh["LIST"], tid % sh["LIST"]
            pop, m = cols[j]
            k = wrap_rows(R, yside, pop) if yside else 0
            row_wrapped = (r < k) if yside > 0 else ((r >= PY - k) if yside < 0 else False)
            if not row_wrapped:
                c = (APRON - R - int(CX[pop]) + m) if xside > 0 else (APRON + w + m)
                bc = c if xside > 0 else m
                x = x0 - APRON + c
                assert x < 0 or x >= nx, "x-apron copy onto an in-range cell"
                idx = pop * POP + r * XW + c
                src = xslot(R, xside, pop, sh["XSLOT"]) // 4 + r * 4 + bc
                assert 0 <= bc < 4 and idx < (pop + 1) * POP
                assert not written[idx], "two fix-ups write one cell"
                written[idx] = True
                stage[idx] = xbuf[src]
        if xside != 0 and yside != 0 and tid < len(corner_list(xside, yside)):
            pop, v, m = corner_list(xside, yside)[tid]
            k = wrap_rows(R, yside, pop)
            r = v if yside > 0 else PY - k + v
            c = (APRON - R - int(CX[pop]) + m) if xside > 0 else (APRON + w + m)
            idx = pop * POP + r * XW + c
            assert not written[idx], "two fix-ups write one cell"
            written[idx] = True
            yy = wrap(y0 - R - int(CY[pop]) + r, ny)
            xx = wrap(x0 - APRON + c, nx)
            stage[idx] = value(nx, ny, nz, xx, yy, wrap(z - int(CZ[pop]), nz), pop)

    # density-pass reads
    reads = 0
    NH, NHW = sh["NH"], (sh["NH"] + 31) // 32 * 32
    nodes = []
    for tid in range(NT):
        tx, ty = tid % BX, tid // BX
        if tx < w + R:
            nodes.append(((ty + R) * PX + tx + R, (ty + R) * XW + tx + APRON))
        hh = tid - (NT - NHW)
        if 0 <= hh < NH:
            jj = halo_node_rows(hh, BX, BY, R)
            if jj % PX < w + 2 * R:
                hx, hy = jj % PX, jj // PX
                nodes.append((jj, hy * XW + hx + APRON - R))
    covered = {j for j, _ in nodes}
    want_nodes = {py * PX + px for py in range(PY) for px in range(w + 2 * R)}
    assert covered == want_nodes, "density pass does not cover the padded tile exactly"
    assert len(nodes) == len(want_nodes)
    for j, base in nodes:
        px, py = j % PX, j // PX
        gx, gy = x0 + px - R, y0 + py - R
        for i in range(Q):
            k = i * POP + base - int(CX[i])
            want = value(nx, ny, nz, wrap(gx - int(CX[i]), nx), wrap(gy - int(CY[i]), ny),
                         wrap(z - int(CZ[i]), nz), i)
            assert stage[k] == want, (i, px, py, stage[k], want)
            reads += 1
    return reads


BOXES = [(64, 16, 5), (128, 128, 7), (72, 24, 4), (68, 32, 3), (96, 40, 6), (256, 16, 3)]


@pytest.mark.parametrize("nx,ny,nz", BOXES)
def test_tma_copy_plan(nx, ny, nz):
    BX, BY, R = 32, 8, 1
    xs = sorted({0, BX, (nx - 1) // BX * BX})
    ys = sorted({0, BY, ny - BY})
    for x0 in xs:
        for y0 in ys:
            for z in (0, nz - 1):
                assert replay(nx, ny, nz, BX, BY, R, x0, y0, z) > 0


def test_tma_shared_memory_budget():
    """Stages, psi ring, wrapped-row buffer, x-apron boxes and mbarriers of the 32 x 8 E4
    tile fit three CTAs per SM (228 KB, 1 KB reserved per CTA), every box region on a
    128-byte boundary; each fix-up list fits one entry per thread."""
    sh = shape(32, 8, 1)
    stage = 4 * Q * sh["POP"]
    ring_off = 2 * stage
    wrap_off = align128(ring_off + 4 * sh["NR"] * sh["NPAD"])
    xa_off = wrap_off + wrap_bytes(1, sh["XW"])
    bar_off = xa_off + sh["XPOPS"] * sh["XSLOT"]
    smem = bar_off + 16 + 128
    assert stage % 128 == 0 and wrap_off % 128 == 0 and xa_off % 128 == 0 and bar_off % 8 == 0
    assert 3 * (smem + 1024) <= 228 * 1024, smem
    assert sh["LIST"] * (sh["XW"] // 4) <= sh["NT"] and sh["PY"] * sh["LIST"] <= sh["NT"]
    assert all(len(corner_list(a, b)) == 19 for a in (1, -1) for b in (1, -1))
