"""Host-side replay of the unit-tau moment kernel's index arithmetic
(lbm_kernels_moment.cuh), for the row-chunk copies (kinds 5, FP16 stage) and
the element copies (kind 6).

For many boxes (ragged, narrow, odd) and every compiled tile shape, one plane of
one item is replayed thread by thread on the CPU:
  * every 16-byte chunk copy starts on a 16-byte boundary in global and shared
    memory, lies inside one row of the population buffer and inside its stage,
    and no two copies write the same staged element;
  * every staged value the density pass reads (own node and halo ring) holds
    the pulled population f_i(x - xi_i) of its padded node;
  * the own nodes and the halo-ring nodes dealt to the threads cover the padded
    tile (w + 2R) x (h + 2R) exactly once, and with the split roles the copy
    warps and the halo warps are disjoint;
  * the one-barrier-per-plane schedule never refills a stage or overwrites a
    psi plane that is still to be read, and the moments and psi kept in
    registers are those of the planes the collision needs.
A copy with a misaligned address is a fault on the GPU, so these are checked
here before any launch.
"""
import numpy as np
import pytest

from oracle import lattice as L

XI = L.D3Q19
Q = 19


def wrap(g, n):
    return g + n if g < 0 else (g - n if g >= n else g)


def ceil32(n):
    return (n + 31) // 32 * 32


def shape(BX, BY, R, S, ELEM):
    NT = BX * BY
    PX, PY = BX + 2 * R, BY + 2 * R
    NPAD = PX * PY
    NH = NPAD - NT
    VE = 16 // S
    APRON = max(VE, 4)
    XW = BX + 2 * APRON
    XWS = XW + 4 if (S == 4 and not ELEM and BX == 32 and BY == 8 and R == 1) else XW   # padded pitch
    NCH = XW // VE
    POS = PY * NCH
    HALO4 = (not ELEM) and BX == 32 and BY == 8 and R == 1 and ceil32(POS) + 128 <= NT
    NHW = 128 if HALO4 else ceil32(NH)
    SPLIT = (not ELEM) and ceil32(POS) + NHW <= NT
    NG = 1 if SPLIT else (2 if 2 * POS <= NT else 1)
    return dict(NT=NT, PX=PX, PY=PY, NPAD=NPAD, NH=NH, NHPER=(NH + NT - 1) // NT, VE=VE, APRON=APRON,
                XW=XW, XWS=XWS, NCH=NCH, POS=POS, POSW=ceil32(POS), NHW=NHW, HALO4=HALO4, SPLIT=SPLIT, NG=NG,
                NPP=1 if NG == 2 else (POS + NT - 1) // NT, ISPLIT=10 if NG == 2 else Q,
                NPER=(NPAD + NT - 1) // NT,
                stage_elems=Q * NPAD if ELEM else Q * PY * XWS)


def halo_node(h, R, PX, PY):
    if h < R * PX:
        return h
    h -= R * PX
    if h < R * PX:
        return (PY - R) * PX + h
    h -= R * PX
    row, c = R + h // (2 * R), h % (2 * R)
    return row * PX + (c if c < R else PX - 2 * R + c)


def halo_node_warps(h, BX, BY, R):
    """The four-warp order of the halo ring (32 x 8 tiles, R = 1): top row, bottom
    row, side columns, the four row ends; None for a lane without a node."""
    PX, PY = BX + 2 * R, BY + 2 * R
    if h < 0:
        return None
    if h < 32:
        return h
    if h < 64:
        return (PY - 1) * PX + (h - 32)
    if h < 80:
        return (1 + (h - 64) // 2) * PX + (PX - 1 if h % 2 else 0)
    if 96 <= h < 100:
        return (0 if h - 96 < 2 else (PY - 1) * PX) + 32 + h % 2
    return None


def replay_plane(nx, ny, nz, BX, BY, R, S, ELEM, x0, y0, z):
    """Stage contents (global element ids) after one plane's copies, and the
    padded nodes the density pass forms with the stage index of each read."""
    sh = shape(BX, BY, R, S, ELEM)
    N = nx * ny * nz
    w, h = min(BX, nx - x0), min(BY, ny - y0)
    rows = h + 2 * R
    xa = x0 - sh["APRON"]
    PX, PY, XW, VE, NPAD = sh["PX"], sh["PY"], sh["XWS"], sh["VE"], sh["NPAD"]
    zo = {c: wrap(z - c, nz) * ny * nx for c in (-1, 0, 1)}      # row of the pull in z
    stage = np.full(sh["stage_elems"], -1, dtype=np.int64)
    for tid in range(sh["NT"]):
        if not ELEM:
            grp = tid // sh["POS"] if sh["NG"] == 2 else 0
            for pp in range(sh["NPP"]):
                p = tid % sh["POS"] if sh["NG"] == 2 else tid + pp * sh["NT"]
                jy, k = divmod(p, sh["NCH"])
                ok = (grp < 2 if sh["NG"] == 2 else p < sh["POS"]) and jy < rows
                if not ok:
                    continue
                y = wrap(y0 - R + jy, ny)
                prow = {c: wrap(y - c, ny) * nx for c in (-1, 0, 1)}
                pgx = wrap(xa + k * VE, nx)
                psm = jy * XW + k * VE
                pops = range(sh["ISPLIT"]) if grp == 0 else range(sh["ISPLIT"], Q)
                for i in pops:
                    s_off = i * PY * XW + psm
                    g_off = i * N + zo[XI[i, 2]] + prow[XI[i, 1]] + pgx
                    assert (s_off * S) % 16 == 0 and (g_off * S) % 16 == 0
                    assert pgx + VE <= nx                     # one row of the buffer
                    assert 0 <= g_off and g_off + VE <= Q * N
                    assert 0 <= s_off and s_off + VE <= sh["stage_elems"]
                    assert np.all(stage[s_off:s_off + VE] == -1)
                    stage[s_off:s_off + VE] = np.arange(g_off, g_off + VE)
        else:
            for s in range(sh["NPER"]):
                j = tid + s * sh["NT"]
                jx, jy = j % PX, j // PX
                if not (j < NPAD and jx < w + 2 * R and jy < rows):
                    continue
                gx, gy = wrap(x0 + jx - R, nx), wrap(y0 + jy - R, ny)
                for i in range(Q):
                    s_off = i * NPAD + j
                    g_off = i * N + zo[XI[i, 2]] + wrap(gy - XI[i, 1], ny) * nx + wrap(gx - XI[i, 0], nx)
                    assert 0 <= g_off < Q * N and stage[s_off] == -1
                    stage[s_off] = g_off
    # density pass: own node of each thread, then the halo nodes dealt to it
    formed = {}
    for tid in range(sh["NT"]):
        tx, ty = tid % BX, tid // BX
        nodes = []
        if tx < w + R and ty < h + R:
            nodes.append((ty + R) * PX + (tx + R))
        for s in range(sh["NHPER"]):
            hh = (tid - (sh["NT"] - sh["NHW"]) if s == 0 else -1) if sh["SPLIT"] else tid + s * sh["NT"]
            if sh["HALO4"]:
                jh = halo_node_warps(hh, BX, BY, R)
            else:
                jh = halo_node(hh, R, PX, PY) if 0 <= hh < sh["NH"] else None
            if jh is not None and jh % PX < w + 2 * R and jh // PX < rows:
                nodes.append(jh)
        for jn in nodes:
            assert jn not in formed, "a padded node is formed twice"
            hx, hy = jn % PX, jn // PX
            if ELEM:
                formed[jn] = [i * NPAD + jn for i in range(Q)]
            else:
                formed[jn] = [i * PY * XW + hy * XW + hx + sh["APRON"] - R - XI[i, 0] for i in range(Q)]
    return stage, formed, w, h, rows


KINDS = [  # (BX, BY, R, S, ELEM): the compiled moment-kernel shapes
    (32, 8, 1, 4, False), (32, 4, 2, 4, False), (32, 8, 1, 8, False), (32, 4, 2, 8, False),
    (32, 8, 1, 2, False),                                   # FP16 stage
    (32, 8, 1, 4, True), (32, 4, 2, 4, True), (32, 8, 1, 8, True), (32, 4, 2, 8, True),
]
BOXES_CHUNK = [(40, 12, 9), (72, 20, 5), (44, 9, 7), (96, 8, 6), (48, 13, 5)]
BOXES_ELEM = [(37, 11, 7), (41, 9, 5), (16, 16, 6), (33, 5, 5), (7, 6, 5), (75, 14, 9)]


def cases():
    for BX, BY, R, S, ELEM in KINDS:
        boxes = BOXES_ELEM if ELEM else BOXES_CHUNK
        for nx, ny, nz in boxes:
            sh = shape(BX, BY, R, S, ELEM)
            # row chunks need nx % 4 == 0 (nx % 8 == 0 for the FP16 stage) and a
            # full staged row inside the box
            if not ELEM and (nx % max(4, sh["VE"]) or nx < BX + 2 * sh["APRON"]):
                continue
            if min(nx, ny, nz) < 2 * R + 1:
                continue
            yield nx, ny, nz, BX, BY, R, S, ELEM


@pytest.mark.parametrize("nx,ny,nz,BX,BY,R,S,ELEM", list(cases()))
def test_moment_copy_plan(nx, ny, nz, BX, BY, R, S, ELEM):
    N = nx * ny * nz
    rng = np.random.default_rng(nx * 31 + ny)
    for x0 in range(0, nx, BX):
        for y0 in range(0, ny, BY):
            z = int(rng.integers(nz))
            stage, formed, w, h, rows = replay_plane(nx, ny, nz, BX, BY, R, S, ELEM, x0, y0, z)
            PX = BX + 2 * R
            want = {jy * PX + jx for jy in range(rows) for jx in range(w + 2 * R)}
            assert set(formed) == want
            for jn, idx in formed.items():
                jx, jy = jn % PX, jn // PX
                gx, gy = wrap(x0 - R + jx, nx), wrap(y0 - R + jy, ny)
                for i in range(Q):
                    expect = (i * N + wrap(z - XI[i, 2], nz) * ny * nx
                              + wrap(gy - XI[i, 1], ny) * nx + wrap(gx - XI[i, 0], nx))
                    assert stage[idx[i]] == expect, (jn, i)


@pytest.mark.parametrize("BX,BY,R,S,ELEM", KINDS)
def test_split_roles_are_disjoint_whole_warps(BX, BY, R, S, ELEM):
    sh = shape(BX, BY, R, S, ELEM)
    if not sh["SPLIT"]:
        pytest.skip("this shape shares warps between copies and halo nodes")
    copy_threads = set(range(sh["POS"]))
    if sh["HALO4"]:
        halo_threads = {t for t in range(sh["NT"])
                        if halo_node_warps(t - (sh["NT"] - sh["NHW"]), BX, BY, R) is not None}
    else:
        halo_threads = {t for t in range(sh["NT"]) if 0 <= t - (sh["NT"] - sh["NHW"]) < sh["NH"]}
    assert not copy_threads & halo_threads
    assert max(copy_threads) // 32 < min(halo_threads) // 32      # different warps
    assert len(halo_threads) == sh["NH"]


@pytest.mark.parametrize("R", [1, 2])
@pytest.mark.parametrize("D", [1, 2])
@pytest.mark.parametrize("zc", [1, 2, 5, 19])
def test_one_barrier_schedule(R, D, zc):
    """Replays the loop of moment_process_item: stage slots q % (1 + D), psi slots
    q % (2R + 2), moments and psi registers shifted once per iteration."""
    NS, NR = 1 + D, 2 * R + 2
    nplanes = zc + 2 * R
    stage_plane = {}          # slot -> plane held
    ring_plane = {}           # slot -> plane whose psi it holds
    issued = set()

    def issue(q):
        if q < nplanes:
            slot = q % NS
            # the slot's previous plane must have had its densities formed already
            prev = stage_plane.get(slot)
            assert prev is None or prev in formed_planes
            stage_plane[slot] = q
            issued.add(q)

    formed_planes = set()
    m = [None] * (R + 1)      # moments: m[0] newest
    pz = [None] * (2 * R + 1) # psi of the own column: pz[2R] newest
    for q in range(D):
        issue(q)
    collided = []
    for qd in range(nplanes + 1):
        if qd < nplanes:
            assert qd in issued                                   # waited for before the barrier
        # --- barrier ---
        issue(qd + D)
        qc = qd - 1 - R
        if qc - R >= 0:
            need = [qc + dz for dz in range(-R, R + 1)]
            for p in need:
                assert ring_plane.get(p % NR) == p                # psi planes present
            assert m[R] == qc and pz == need                      # registers hold the right planes
            collided.append(qc)
        m = [None] + m[:-1]
        pz = pz[1:] + [None]
        if qd < nplanes:
            assert stage_plane[qd % NS] == qd                     # the stage read holds plane qd
            slot = qd % NR
            if qc - R >= 0:
                assert all(slot != (qc + dz) % NR for dz in range(-R, R + 1))
            ring_plane[slot] = qd
            formed_planes.add(qd)
            m[0] = qd
            pz[2 * R] = qd
    assert collided == list(range(R, R + zc))                     # every output plane, in order


def test_halo_warps_read_distinct_banks():
    """FP32 32 x 8 stage (rows XWS = 44 floats apart): every halo warp's 19 population
    reads hit 32 distinct banks (one wavefront each); the old three-warp order put the
    row ends and the side columns in one warp, 4 two-way conflicts per read."""
    sh = shape(32, 8, 1, 4, False)
    assert sh["HALO4"] and sh["XWS"] == 44
    PX, XWS, A = sh["PX"], sh["XWS"], sh["APRON"]
    nodes = sorted({halo_node_warps(h, 32, 8, 1) for h in range(128)} - {None})
    assert len(nodes) == sh["NH"]                        # the whole ring, once
    for warp in range(4):
        js = [halo_node_warps(h, 32, 8, 1) for h in range(32 * warp, 32 * warp + 32)]
        js = [j for j in js if j is not None]
        for i in range(Q):
            banks = [((j // PX) * XWS + j % PX + A - 1 - XI[i, 0] + i * sh["PY"] * XWS) % 32 for j in js]
            assert len(set(banks)) == len(banks), (warp, i)
