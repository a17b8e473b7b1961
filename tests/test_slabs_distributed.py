"""One lattice split into z-slabs (Sec. II: the update of Eq. (3) is local), on
the CPU: the partition and the ghost-plane populations come from liblbm's host
calls, each slab is stepped by the oracle as a periodic lattice of its owned plus
ghost planes, and the ghosts are refreshed through torch.distributed (gloo
ranks).  The owned planes must equal the whole lattice's, bit for bit, with
every ghost population outside the plan poisoned with NaN before each step.

The slabs hold the library's storage convention: slot i of node y is the
population leaving y along xi_i (the pre-collision f_i(x, t) of Eq. (3) is slot i
of node x - xi_i).  In that convention a step is collide-then-store, written
here from the oracle's collide-and-stream step and periodic shifts.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import lbm3d as O  # noqa: E402
from oracle.lattice import D3Q19 as XI  # noqa: E402
from tests.inputs import random_populations  # noqa: E402

SL = pytest.importorskip("paper_2105_08772_gb300.slabs")


def _shift_pops(a, sign):
    return np.stack([np.roll(a[i], shift=(sign * int(XI[i, 2]), sign * int(XI[i, 1]), sign * int(XI[i, 0])),
                             axis=(0, 1, 2)) for i in range(19)])


def stored_from_f(f):
    """slot i of node y = f_i(y + xi_i)"""
    return _shift_pops(f, -1)


def storage_step(g, m):
    """one step of Eq. (3) in the storage convention (periodic box)"""
    with np.errstate(invalid="ignore", over="ignore"):
        return stored_from_f(O.step(_shift_pops(g, +1), m))


def _model(stencil):
    return O.Model(tau=1.0, G=-5.0, stencil=stencil)


def _poison(g, p, rank):
    """NaN in every ghost population the plan does not refresh"""
    for dz, _, _, mask in p.ghost_sources(rank):
        for i in range(19):
            if not (mask >> i) & 1:
                g[i, dz] = np.nan


def _whole(shape, seed, stencil, steps):
    g = stored_from_f(random_populations(shape, seed))
    out = [g]
    for _ in range(steps):
        out.append(storage_step(out[-1], _model(stencil)))
    return out


def test_partition_and_ghost_masks_follow_the_stencil_radius():
    for stencil, R in (("E4", 1), ("E6", 2), ("E8", 2)):
        p = SL.plan(13, 3, stencil)
        assert p.z_begin == (0, 5, 9, 13) and p.H == R + 1
        cz = XI[:, 2]
        for side, masks in ((-1, p.mask_below), (+1, p.mask_above)):
            total = 0
            for k, m in enumerate(masks, start=1):
                pops = {i for i in range(19) if (m >> i) & 1}
                inward = {i for i in range(19) if cz[i] == -side}
                rest = {i for i in range(19) if cz[i] == 0}
                outward = {i for i in range(19) if cz[i] == side}
                want = (inward if k <= R + 1 else set()) | (rest if k <= R else set()) | \
                       (outward if k <= R - 1 else set())
                assert pops == want, (stencil, side, k)
                total += len(pops)
            assert total == 19 * R
    # a slab thinner than R + 1 planes is refused
    from paper_2105_08772_gb300._lib import LBMError
    with pytest.raises(LBMError):
        SL.plan(5, 3, "E4")
    with pytest.raises(LBMError):
        SL.plan(8, 3, "E8")


@pytest.mark.parametrize("stencil", ["E4", "E8"])
def test_every_ghost_population_of_the_plan_is_needed(stencil):
    """Poisoning any one (ghost plane, population) of the plan reaches an owned node
    within one step: the plan is minimal as well as sufficient."""
    shape = (14, 5, 6)
    p = SL.plan(shape[0], 2, stencil)
    g0 = _whole(shape, 7, stencil, 0)[0]
    r = 0
    loc = np.ascontiguousarray(g0[:, p.window(r)])
    H, n = p.H, p.n_owned(r)
    base = storage_step(loc, _model(stencil))[:, H:H + n]
    assert np.isfinite(base).all()
    for dz, _, _, mask in p.ghost_sources(r):
        for i in range(19):
            if not (mask >> i) & 1:
                continue
            bad = loc.copy()
            bad[i, dz] = np.nan
            out = storage_step(bad, _model(stencil))[:, H:H + n]
            assert not np.isfinite(out).all(), (dz, i)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir, shape, stencil, steps):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = SL.plan(shape[0], world, stencil)
        ref = _whole(shape, 11, stencil, steps)
        g = torch.from_numpy(np.ascontiguousarray(ref[0][:, p.window(rank)]))
        H, n = p.H, p.n_owned(rank)
        z0, z1 = p.owned(rank)
        ok = []
        for t in range(1, steps + 1):
            _poison(g.numpy(), p, rank)
            g = torch.from_numpy(storage_step(g.numpy(), _model(stencil)))
            SL.exchange_tensors(p, rank, g)
            ok.append(np.array_equal(g.numpy()[:, H:H + n], ref[t][:, z0:z1]))
            # ghosts now hold the neighbours' owned values for every population of the plan
            for dz, _, _, mask in p.ghost_sources(rank):
                zg = p.window(rank)[dz]
                for i in range(19):
                    if (mask >> i) & 1:
                        ok.append(np.array_equal(g.numpy()[i, dz], ref[t][i, zg]))
        # convergence-test style reduction: the mass over owned planes, summed over ranks
        mass = SL.allreduce_sum([g.numpy()[:, H:H + n].sum()])[0]
        whole = ref[steps].sum()
        ok.append(abs(mass - whole) <= 1e-12 * abs(whole))
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write("ok" if all(ok) else f"bad {ok}")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,shape,stencil", [
    (2, (11, 5, 6), "E4"),     # ragged: 6 + 5 planes
    (3, (13, 4, 5), "E4"),
    (2, (12, 5, 5), "E8"),     # R = 2: three ghost planes a side
])
def test_gloo_slabs_step_like_the_whole_lattice(tmp_path, world, shape, stencil):
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path), shape, stencil, 3), nprocs=world,
                       start_method="spawn", join=True)
    for r in range(world):
        assert (tmp_path / f"rank{r}.txt").read_text() == "ok"


def test_single_slab_wraps_onto_itself():
    """world = 1: the ghost planes come from the slab's own far planes."""
    shape = (9, 4, 5)
    p = SL.plan(shape[0], 1, "E4")
    ref = _whole(shape, 3, "E4", 2)
    g = torch.from_numpy(np.ascontiguousarray(ref[0][:, p.window(0)]))
    for t in (1, 2):
        _poison(g.numpy(), p, 0)
        g = torch.from_numpy(storage_step(g.numpy(), _model("E4")))
        SL.exchange_tensors(p, 0, g)
        assert np.array_equal(g.numpy()[:, p.H:p.H + 9], ref[t])


def test_slab_calls_reject_bad_arguments_on_the_host():
    import ctypes as C
    from paper_2105_08772_gb300 import _lib
    L = _lib.lib
    zb = (C.c_int * 4)()
    m = C.c_uint()
    assert L.lbm_slab_partition(12, 3, 4, None) == _lib.LBM_EINVAL
    assert L.lbm_slab_partition(12, 0, 4, zb) == _lib.LBM_EINVAL
    assert L.lbm_slab_partition(12, 3, 5, zb) == _lib.LBM_EINVAL          # no such stencil
    assert L.lbm_slab_partition(12, 1, 4, zb) == _lib.LBM_OK and list(zb)[:2] == [0, 12]
    assert L.lbm_slab_halo_mask(4, 0, 1, C.byref(m)) == _lib.LBM_EINVAL    # side must be +-1
    assert L.lbm_slab_halo_mask(4, 1, 3, C.byref(m)) == _lib.LBM_EINVAL    # E4: k = 1, 2 only
    assert L.lbm_slab_halo_mask(8, -1, 3, C.byref(m)) == _lib.LBM_OK and bin(m.value).count("1") == 5
    assert L.lbm_slab_halo_mask(4, 1, 1, None) == _lib.LBM_EINVAL
    assert L.lbm_halo_copy(None, 0, None, 0, 1) == _lib.LBM_EINVAL
    assert L.lbm_state_plane(None, 0, 0, None, None) == _lib.LBM_EINVAL
