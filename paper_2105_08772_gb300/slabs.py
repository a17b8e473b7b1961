"""Z-slab decomposition of one lattice over several processes or devices.

The update of Eq. (3) is local (Sec. II, below Eq. (3)): a node's new
populations depend only on the stored populations of the nodes within R + 1
planes (pull streaming, then the density of the force stencil's neighbours
within R; R = 1 for E4, 2 for E6 / E8).  A lattice too large for one GPU is
therefore cut along z into contiguous slabs.  Each slab is a lattice of its
owned planes plus H = R + 1 ghost planes on each side, stepped as an ordinary
periodic lattice by the single-GPU kernels: the wrap-around reaches only ghost
planes, whose results are discarded.  After every step the ghost planes'
needed populations (``lbm_slab_halo_mask``: 19 R population planes per side)
are copied from the neighbouring slabs.

Local plane indices of slab r with n_r owned planes: ghost plane k below the
owned planes (k = 1..H, counted outward) is local plane H - k; owned planes are
H .. H + n_r - 1; ghost plane k above is H + n_r - 1 + k.  Ghost k below comes
from the slab below's local plane H + n_{r-1} - k, ghost k above from the slab
above's local plane H + k - 1 (slabs periodic in r).

Two exchanges implement the same plan:

* ``exchange_local`` -- slabs held by one process (the same or peer devices):
  ``lbm_halo_copy`` device copies on the slabs' stream;
* ``exchange_tensors`` -- one slab per process: the rank's state as a
  [19, local_nz, ny, nx] tensor (a view of its population planes, or a host
  copy), exchanged with torch.distributed point-to-point messages (NCCL for
  device tensors, gloo for host tensors).

Reductions for the convergence test and the observables (Sec. IV) are sums
over owned planes (``allreduce_sum``, FP64) and point values read on the rank
that owns the point.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lbm as _lbm
from ._lib import STENCILS


@dataclass(frozen=True)
class SlabPlan:
    nz: int
    world: int
    stencil: str
    z_begin: tuple            # world + 1 global plane indices
    mask_below: tuple         # mask of ghost plane k = 1..H below the owned planes
    mask_above: tuple

    @property
    def H(self) -> int:
        return len(self.mask_below)

    def owned(self, r: int) -> tuple[int, int]:
        return self.z_begin[r], self.z_begin[r + 1]

    def n_owned(self, r: int) -> int:
        return self.z_begin[r + 1] - self.z_begin[r]

    def local_nz(self, r: int) -> int:
        return self.n_owned(r) + 2 * self.H

    def below(self, r: int) -> int:
        return (r - 1) % self.world

    def above(self, r: int) -> int:
        return (r + 1) % self.world

    def ghost_sources(self, r: int):
        """(local ghost plane, source slab, source local plane, mask) of every ghost
        plane of slab r, below (k = 1..H) then above."""
        H = self.H
        out = []
        b, a = self.below(r), self.above(r)
        for k in range(1, H + 1):
            out.append((H - k, b, H + self.n_owned(b) - k, self.mask_below[k - 1]))
        for k in range(1, H + 1):
            out.append((H + self.n_owned(r) - 1 + k, a, H + k - 1, self.mask_above[k - 1]))
        return out

    def window(self, r: int) -> np.ndarray:
        """Global plane of each local plane of slab r (periodic in z)."""
        z0, z1 = self.owned(r)
        return np.arange(z0 - self.H, z1 + self.H) % self.nz


def plan(nz: int, world: int, stencil: str = "E4") -> SlabPlan:
    st = STENCILS[stencil]
    zb = _lbm.lbm_slab_partition(nz, world, st)
    R = 1 if stencil == "E4" else 2
    below = tuple(_lbm.lbm_slab_halo_mask(st, -1, k) for k in range(1, R + 2))
    above = tuple(_lbm.lbm_slab_halo_mask(st, +1, k) for k in range(1, R + 2))
    return SlabPlan(nz, world, stencil, tuple(zb), below, above)


def _pops(mask: int):
    return [i for i in range(19) if (mask >> i) & 1]


def exchange_local(p: SlabPlan, ctxs) -> None:
    """Refresh every slab's ghost planes from its neighbours; ctxs[r] is slab r's
    context, all in this process (device copies, enqueued on the slabs' streams)."""
    for r in range(p.world):
        for dz, src, sz, mask in p.ghost_sources(r):
            _lbm.lbm_halo_copy(ctxs[r], dz, ctxs[src], sz, mask)


def _pack(state, planes):
    import torch
    return torch.cat([state[i, z].reshape(-1) for z, mask in planes for i in _pops(mask)])


def _unpack(state, planes, buf):
    o = 0
    for z, mask in planes:
        for i in _pops(mask):
            n = state[i, z].numel()
            state[i, z].copy_(buf[o:o + n].view_as(state[i, z]))
            o += n


def exchange_tensors(p: SlabPlan, rank: int, state, group=None) -> None:
    """Refresh this rank's ghost planes; state is its [19, local_nz, ny, nx] tensor,
    updated in place.  Every rank of the group calls this with its own slab."""
    import torch.distributed as dist
    H, n = p.H, p.n_owned(rank)
    # what this rank's neighbours need from it: the slab below's ghosts above, the
    # slab above's ghosts below
    to_below = [(H + k - 1, p.mask_above[k - 1]) for k in range(1, H + 1)]
    to_above = [(H + n - k, p.mask_below[k - 1]) for k in range(1, H + 1)]
    my_below = [(H - k, p.mask_below[k - 1]) for k in range(1, H + 1)]
    my_above = [(H + n - 1 + k, p.mask_above[k - 1]) for k in range(1, H + 1)]
    if p.world == 1:
        _unpack(state, my_below, _pack(state, to_above).clone())
        _unpack(state, my_above, _pack(state, to_below).clone())
        return
    send_down, send_up = _pack(state, to_below), _pack(state, to_above)
    recv_from_above = send_down.new_empty(send_down.numel())   # the slab above sends its to_below
    recv_from_below = send_up.new_empty(send_up.numel())
    b, a = p.below(rank), p.above(rank)
    reqs = [dist.isend(send_down, b, group=group, tag=1), dist.isend(send_up, a, group=group, tag=2),
            dist.irecv(recv_from_above, a, group=group, tag=1), dist.irecv(recv_from_below, b, group=group, tag=2)]
    for q in reqs:
        q.wait()
    _unpack(state, my_above, recv_from_above)
    _unpack(state, my_below, recv_from_below)


def allreduce_sum(values, group=None) -> np.ndarray:
    """FP64 sums over all ranks of per-rank partial sums (owned planes only)."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.asarray(values, dtype=np.float64))
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy()


class SlabLattice:
    """One lattice held as `world` z-slabs in this process (one device, or peer
    devices): each slab a Lattice of nx x ny x (owned + 2H), stepped by the
    single-GPU kernels one after another on one stream, ghost planes refreshed
    after every step."""

    def __init__(self, nx, ny, nz, world, tau=1.0, G=-5.0, psi="one_minus_exp", stencil="E4",
                 prec="f64", stream=None):
        self.plan = plan(nz, world, stencil)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.slabs = [_lbm.Lattice(nx, ny, self.plan.local_nz(r), tau=tau, G=G, psi=psi, stencil=stencil,
                                   prec=prec, stream=stream) for r in range(world)]

    def set_populations(self, f: np.ndarray, n0: float, scale: float = 1.0):
        """f: the whole lattice's pre-collision populations [19, nz, ny, nx]; every slab
        stores with the given shift and scale."""
        for r, lat in enumerate(self.slabs):
            _lbm.lbm_set_populations_storage(lat.ctx, np.ascontiguousarray(f[:, self.plan.window(r)]), n0, scale)

    def step(self, n: int = 1):
        ctxs = [lat.ctx for lat in self.slabs]
        for _ in range(n):
            for lat in self.slabs:
                lat.step(1)
            exchange_local(self.plan, ctxs)

    def populations(self) -> np.ndarray:
        """The owned planes of every slab, as the whole lattice's [19, nz, ny, nx]."""
        out = np.empty((19, self.nz, self.ny, self.nx))
        H = self.plan.H
        for r, lat in enumerate(self.slabs):
            z0, z1 = self.plan.owned(r)
            out[:, z0:z1] = lat.get_populations()[:, H:H + z1 - z0]
        return out

    def close(self):
        for lat in self.slabs:
            lat.close()
        self.slabs = []
