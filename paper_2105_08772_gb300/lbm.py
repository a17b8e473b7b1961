"""Python binding of the C ABI with the same names (argument marshalling only).

Device memory and streams come from PyTorch: ``Lattice`` allocates the
workspace as a uint8 CUDA tensor and passes its pointer and the current CUDA
stream to ``lbm_create``.  Host buffers are numpy float64 arrays.  All of the
method runs inside liblbm.so.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import (LBM_F16_SHIFTED, LBM_F32_SHIFTED, LBM_F64, PRECS, PSI_KINDS, STENCILS,
                   LBMError, check, lbm_box, lbm_eos, lbm_obs)

_lib_ = _lib.lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_box(nx: int, ny: int, nz: int) -> lbm_box:
    return lbm_box(int(nx), int(ny), int(nz))


def make_eos(kind: str | int = "one_minus_exp", a=1.0, b=4.0, Rgas=1.0, T=0.0) -> lbm_eos:
    k = PSI_KINDS[kind] if isinstance(kind, str) else int(kind)
    return lbm_eos(k, float(a), float(b), float(Rgas), float(T))


# ---------------------------------------------------------------- same-name wrappers

def lbm_workspace_bytes(box: lbm_box, stencil: int, prec: int) -> int:
    return int(_lib_.lbm_workspace_bytes(box, int(stencil), int(prec)))


def lbm_create(box, tau, G, eos, stencil, prec, dev_workspace: int, nbytes: int, stream: int):
    out = C.c_void_p()
    st = _lib_.lbm_create(box, float(tau), float(G), eos, int(stencil), int(prec),
                          C.c_void_p(dev_workspace), C.c_size_t(nbytes), C.c_void_p(stream),
                          C.byref(out))
    check(st, None)
    return out


def lbm_destroy(ctx) -> None:
    _lib_.lbm_destroy(ctx)


def lbm_init_drop(ctx, center, R, rho_in, rho_out, width=1.0):
    c = np.ascontiguousarray(center, dtype=np.float64)
    check(_lib_.lbm_init_drop(ctx, _dptr(c), float(R), float(rho_in), float(rho_out), float(width)), ctx)


def lbm_init_rho(ctx, host_rho: np.ndarray):
    r = np.ascontiguousarray(host_rho, dtype=np.float64)
    check(_lib_.lbm_init_rho(ctx, _dptr(r)), ctx)


def lbm_set_populations(ctx, host_f: np.ndarray):
    f = np.ascontiguousarray(host_f, dtype=np.float64)
    check(_lib_.lbm_set_populations(ctx, _dptr(f)), ctx)


def lbm_get_populations(ctx, out: np.ndarray):
    check(_lib_.lbm_get_populations(ctx, _dptr(out)), ctx)
    return out


def lbm_step(ctx, n: int):
    check(_lib_.lbm_step(ctx, int(n)), ctx)


def lbm_run_to_convergence(ctx, max_steps=50_000, check_every=2048, tol_dP_rel=1e-5, tol_du=1e-12):
    """Returns (status, steps_done, criterion); LBM_ENOTCONV and LBM_ECOLLAPSE are
    returned, not raised."""
    steps = C.c_longlong(0)
    crit = C.c_int(0)
    st = _lib_.lbm_run_to_convergence(ctx, int(max_steps), int(check_every), float(tol_dP_rel),
                                      float(tol_du), C.byref(steps), C.byref(crit))
    if st not in (_lib.LBM_OK, _lib.LBM_ENOTCONV, _lib.LBM_ECOLLAPSE):
        check(st, ctx)
    return st, steps.value, crit.value


def lbm_observables(ctx) -> lbm_obs:
    o = lbm_obs()
    check(_lib_.lbm_observables(ctx, C.byref(o)), ctx)
    return o


def lbm_rho_profile(ctx, length: int) -> np.ndarray:
    out = np.empty(length)
    check(_lib_.lbm_rho_profile(ctx, _dptr(out), length), ctx)
    return out


def lbm_pt_profile(ctx, length: int) -> np.ndarray:
    out = np.empty(length)
    check(_lib_.lbm_pt_profile(ctx, _dptr(out), length), ctx)
    return out


def lbm_sigma_of_R(ctx, R) -> tuple[np.ndarray, np.ndarray]:
    R = np.ascontiguousarray(R, dtype=np.float64)
    s = np.empty_like(R)
    ds = np.empty_like(R)
    check(_lib_.lbm_sigma_of_R(ctx, _dptr(R), _dptr(s), _dptr(ds), R.size), ctx)
    return s, ds


def lbm_copy_rho(ctx, out: np.ndarray) -> np.ndarray:
    check(_lib_.lbm_copy_rho(ctx, _dptr(out)), ctx)
    return out


def lbm_copy_velocity(ctx, out: np.ndarray) -> np.ndarray:
    check(_lib_.lbm_copy_velocity(ctx, _dptr(out)), ctx)
    return out


def lbm_save(ctx, path: str):
    check(_lib_.lbm_save(ctx, str(path).encode()), ctx)


def lbm_load(ctx, path: str):
    check(_lib_.lbm_load(ctx, str(path).encode()), ctx)


def lbm_autotune(ctx, reps: int = 8) -> int:
    ch = C.c_longlong(0)
    check(_lib_.lbm_autotune(ctx, int(reps), C.byref(ch)), ctx)
    return ch.value


def lbm_set_tile(ctx, code: int):
    check(_lib_.lbm_set_tile(ctx, int(code)), ctx)


def lbm_get_tile(ctx) -> int:
    code = C.c_longlong(0)
    check(_lib_.lbm_get_tile(ctx, C.byref(code)), ctx)
    return code.value


def lbm_default_tile(box: lbm_box, stencil: int, prec: int, tau: float = 1.0) -> int:
    """Tile code lbm_create starts from for these arguments (host only, no device)."""
    code = C.c_longlong(0)
    check(_lib_.lbm_default_tile(box, int(stencil), int(prec), float(tau), C.byref(code)), None)
    return code.value


def default_tile(nx: int, ny: int, nz: int, stencil="E4", prec="f32", tau=1.0) -> int:
    return lbm_default_tile(make_box(nx, ny, nz), STENCILS[stencil], PRECS[prec], tau)


def lbm_storage_params(ctx) -> tuple[float, float]:
    n0 = C.c_double()
    sc = C.c_double()
    check(_lib_.lbm_storage_params(ctx, C.byref(n0), C.byref(sc)), ctx)
    return n0.value, sc.value


def lbm_slab_partition(nz: int, world: int, stencil: int) -> list[int]:
    """First global plane of each of `world` z-slabs, and nz (world + 1 ints)."""
    out = (C.c_int * (world + 1))()
    check(_lib_.lbm_slab_partition(int(nz), int(world), int(stencil), out))
    return list(out)


def lbm_slab_halo_mask(stencil: int, side: int, k: int) -> int:
    """Bit mask of the populations ghost plane k (1..R+1) on side -1 / +1 must hold."""
    m = C.c_uint()
    check(_lib_.lbm_slab_halo_mask(int(stencil), int(side), int(k), C.byref(m)))
    return m.value


def lbm_set_populations_storage(ctx, host_f: np.ndarray, n0: float, scale: float):
    f = np.ascontiguousarray(host_f, dtype=np.float64)
    check(_lib_.lbm_set_populations_storage(ctx, _dptr(f), float(n0), float(scale)), ctx)


def lbm_state_plane(ctx, i: int, z: int) -> tuple[int, int]:
    """(device address, bytes) of population i's plane z of the current state."""
    p = C.c_void_p()
    nb = C.c_size_t()
    check(_lib_.lbm_state_plane(ctx, int(i), int(z), C.byref(p), C.byref(nb)), ctx)
    return p.value, nb.value


def lbm_halo_copy(dst, dst_z: int, src, src_z: int, mask: int):
    check(_lib_.lbm_halo_copy(dst, int(dst_z), src, int(src_z), int(mask)), dst)


def lbm_tolman_fit(R_s, sigma_s, is_bubble, quadratic=True) -> tuple[float, float, float]:
    R = np.ascontiguousarray(R_s, dtype=np.float64)
    s = np.ascontiguousarray(sigma_s, dtype=np.float64)
    b = np.ascontiguousarray(is_bubble, dtype=np.int32)
    s0, d, c = C.c_double(), C.c_double(), C.c_double()
    check(_lib_.lbm_tolman_fit(_dptr(R), _dptr(s), b.ctypes.data_as(C.POINTER(C.c_int)), R.size,
                               int(bool(quadratic)), C.byref(s0), C.byref(d), C.byref(c)), None)
    return s0.value, d.value, c.value


def lbm_density_moments_noalloc(dev_rho: int, nx: int, ny: int, nz: int, n_ref: float,
                                dev_out: int, stream: int = 0):
    """Mass and centre of mass of a device density field (device pointers as ints);
    allocates no device memory.  Writes {mass, com_x, com_y, com_z} to dev_out."""
    check(_lib_.lbm_density_moments_noalloc(C.c_void_p(dev_rho), int(nx), int(ny), int(nz),
                                            float(n_ref), C.c_void_p(dev_out), C.c_void_p(stream)),
          None)


def lbm_pn_profile(ctx, length: int) -> np.ndarray:
    out = np.empty(length)
    check(_lib_.lbm_pn_profile(ctx, _dptr(out), length), ctx)
    return out


def lbm_flat_workspace_bytes(Lx: int, stencil: int, prec: int) -> int:
    return int(_lib_.lbm_flat_workspace_bytes(int(Lx), int(stencil), int(prec)))


def lbm_flat_interface(tau, G, eos, stencil, prec, Lx, rho_l0, rho_g0, max_steps, tol_du,
                       dev_workspace: int, nbytes: int, stream: int):
    """(status, n_g, n_l, sigma0, steps); LBM_ENOTCONV is returned, not raised."""
    ng, nl, s0, steps = C.c_double(), C.c_double(), C.c_double(), C.c_longlong()
    st = _lib_.lbm_flat_interface(float(tau), float(G), eos, int(stencil), int(prec), int(Lx),
                                  float(rho_l0), float(rho_g0), int(max_steps), float(tol_du),
                                  C.c_void_p(dev_workspace), C.c_size_t(nbytes), C.c_void_p(stream),
                                  C.byref(ng), C.byref(nl), C.byref(s0), C.byref(steps))
    if st not in (_lib.LBM_OK, _lib.LBM_ENOTCONV):
        check(st, None)
    return st, ng.value, nl.value, s0.value, steps.value


def lbm_coexistence_estimate(eos, G) -> tuple[float, float, float]:
    """(n_g, n_l, p_0) of the continuum flat-interface construction (host only)."""
    ng, nl, p0 = C.c_double(), C.c_double(), C.c_double()
    check(_lib_.lbm_coexistence_estimate(eos, float(G), C.byref(ng), C.byref(nl), C.byref(p0)), None)
    return ng.value, nl.value, p0.value


def coexistence_estimate(G, psi="one_minus_exp", cs_T=0.0, a=1.0, b=4.0, Rgas=1.0):
    return lbm_coexistence_estimate(make_eos(psi, a=a, b=b, Rgas=Rgas, T=cs_T), G)


def flat_interface(G, psi="one_minus_exp", stencil="E4", prec="f64", tau=1.0, Lx=100, rho_l0=None,
                   rho_g0=None, max_steps=400_000, tol_du=1e-13, cs_T=0.0):
    """Flat-interface coexistence on the GPU with a torch-owned workspace.
    Returns (status, n_g, n_l, sigma0, steps)."""
    import torch
    st_, pr = STENCILS[stencil], PRECS[prec]
    nbytes = lbm_flat_workspace_bytes(Lx, st_, pr)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    ptr = ws.data_ptr() + (-ws.data_ptr()) % 256
    # both 0: the library starts from its continuum coexistence estimate
    rl = 0.0 if rho_l0 is None else rho_l0
    rg = 0.0 if rho_g0 is None else rho_g0
    return lbm_flat_interface(tau, G, make_eos(psi, T=cs_T), st_, pr, Lx, rl, rg, max_steps, tol_du, ptr,
                              nbytes, torch.cuda.current_stream().cuda_stream)


# ---------------------------------------------------------------- batches

def _bcheck(status: int, b) -> int:
    if status != _lib.LBM_OK:
        raise LBMError(status, _lib_.lbm_batch_last_error(b).decode())
    return status


def lbm_batch_workspace_bytes(slots: int, max_box: lbm_box, stencil: int, prec: int) -> int:
    return int(_lib_.lbm_batch_workspace_bytes(int(slots), max_box, int(stencil), int(prec)))


def lbm_batch_create(slots, max_box, stencil, prec, dev_workspace: int, nbytes: int, stream: int):
    out = C.c_void_p()
    _bcheck(_lib_.lbm_batch_create(int(slots), max_box, int(stencil), int(prec), C.c_void_p(dev_workspace),
                                   C.c_size_t(nbytes), C.c_void_p(stream), C.byref(out)), None)
    return out


def lbm_batch_enqueue(b, box, tau, G, eos, center, R, rho_in, rho_out, width=1.0) -> int:
    c = np.ascontiguousarray(center, dtype=np.float64)
    rid = C.c_int(-1)
    _bcheck(_lib_.lbm_batch_enqueue(b, box, float(tau), float(G), eos, _dptr(c), float(R), float(rho_in),
                                    float(rho_out), float(width), C.byref(rid)), b)
    return rid.value


def lbm_batch_run(b, max_steps=50_000, check_every=2048, tol_dP_rel=1e-5, tol_du=1e-12) -> int:
    lu = C.c_longlong(0)
    _bcheck(_lib_.lbm_batch_run(b, int(max_steps), int(check_every), float(tol_dP_rel), float(tol_du),
                                C.byref(lu)), b)
    return lu.value


def lbm_batch_autotune(b, reps: int = 8) -> int:
    """Time the batch step's kernel modes, z chunks and slot counts on the resident
    lattices and keep the fastest; returns the choice code (mode 10^6 + z chunk 10^3 +
    slots)."""
    code = C.c_longlong()
    _bcheck(_lib_.lbm_batch_autotune(b, int(reps), C.byref(code)), b)
    return code.value


def lbm_batch_result(b, rid: int):
    """(status, lbm_obs) of a finished run; the status is returned, not raised."""
    o = lbm_obs()
    st = _lib_.lbm_batch_result(b, int(rid), C.byref(o))
    if st == _lib.LBM_EINVAL:
        _bcheck(st, None)
    return st, o


def lbm_batch_destroy(b) -> None:
    _lib_.lbm_batch_destroy(b)


class Batch:
    """A batch of lattices on a torch-owned workspace (see lbm_batch_* in include/lbm.h).
    Stream rule as for Lattice: allocate under the stream the batch runs on, or
    synchronise that stream before the batch is closed."""

    def __init__(self, slots: int, max_box, stencil="E4", prec="f32", stream=None):
        import torch
        self.max_box = make_box(*max_box)
        st, pr = STENCILS[stencil], PRECS[prec]
        self.nbytes = lbm_batch_workspace_bytes(slots, self.max_box, st, pr)
        if self.nbytes == 0:
            raise LBMError(_lib.LBM_EINVAL, "invalid batch arguments")
        self.workspace = torch.empty(self.nbytes + 256, dtype=torch.uint8, device="cuda")
        ptr = self.workspace.data_ptr()
        ptr += (-ptr) % 256
        s = stream if stream is not None else torch.cuda.current_stream()
        self.b = lbm_batch_create(slots, self.max_box, st, pr, ptr, self.nbytes, s.cuda_stream)

    def enqueue(self, box, tau=1.0, G=-5.0, psi="one_minus_exp", center=None, R=8.0, rho_in=2.0,
                rho_out=0.15, width=1.0, cs_T=0.0) -> int:
        bx = make_box(*box)
        c = center if center is not None else (box[0] // 2, box[1] // 2, box[2] // 2)
        return lbm_batch_enqueue(self.b, bx, tau, G, make_eos(psi, T=cs_T), c, R, rho_in, rho_out, width)

    def run(self, **kw) -> int:
        return lbm_batch_run(self.b, **kw)

    def autotune(self, reps: int = 8) -> int:
        return lbm_batch_autotune(self.b, reps)

    def result(self, rid: int):
        return lbm_batch_result(self.b, rid)

    def close(self):
        if getattr(self, "b", None) is not None:
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _gcheck(status: int, g) -> int:
    if status != _lib.LBM_OK:
        raise LBMError(status, _lib_.lbm_group_last_error(g).decode())
    return status


def lbm_group_workspace_bytes(n: int) -> int:
    return int(_lib_.lbm_group_workspace_bytes(int(n)))


def lbm_group_create(ctxs, dev_workspace: int, nbytes: int, stream: int):
    arr = (C.c_void_p * len(ctxs))(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    out = C.c_void_p()
    _gcheck(_lib_.lbm_group_create(arr, len(ctxs), C.c_void_p(dev_workspace), C.c_size_t(nbytes),
                                   C.c_void_p(stream), C.byref(out)), None)
    return out


def lbm_group_step(g, n: int):
    _gcheck(_lib_.lbm_group_step(g, int(n)), g)


def lbm_group_destroy(g) -> None:
    _lib_.lbm_group_destroy(g)


class Group:
    """Several Lattice objects stepped together, one launch per time step (see
    lbm_group_* in include/lbm.h).  The lattices must outlive the group."""

    def __init__(self, lattices, stream=None):
        import torch
        self.lattices = list(lattices)
        self.nbytes = lbm_group_workspace_bytes(len(self.lattices))
        self.workspace = torch.empty(self.nbytes + 256, dtype=torch.uint8, device="cuda")
        ptr = self.workspace.data_ptr()
        ptr += (-ptr) % 256
        s = stream if stream is not None else torch.cuda.current_stream()
        self.g = lbm_group_create([lat.ctx for lat in self.lattices], ptr, self.nbytes, s.cuda_stream)

    def step(self, n: int):
        lbm_group_step(self.g, n)

    def close(self):
        if getattr(self, "g", None) is not None:
            lbm_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- convenience object

@dataclass
class Lattice:
    """One lattice: a torch-owned device workspace plus an lbm_ctx on a stream.

    The workspace is allocated on torch's current stream.  When `stream` is a
    different stream, create the lattice inside `with torch.cuda.stream(stream):`
    (as bench.py does), or synchronise `stream` before the lattice is closed or
    dropped: otherwise torch's caching allocator may hand the memory to other
    work while kernels queued on `stream` still use it."""
    nx: int
    ny: int
    nz: int
    tau: float = 1.0
    G: float = -5.0
    psi: str = "one_minus_exp"
    stencil: str = "E4"
    prec: str = "f64"
    cs_T: float = 0.0
    stream: object = None   # torch.cuda.Stream or None (current stream)

    def __post_init__(self):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Lattice needs a CUDA device (the library has no CPU path)")
        self.box = make_box(self.nx, self.ny, self.nz)
        self.eos = make_eos(self.psi, T=self.cs_T)
        st, pr = STENCILS[self.stencil], PRECS[self.prec]
        self.nbytes = lbm_workspace_bytes(self.box, st, pr)
        if self.nbytes == 0:
            raise LBMError(_lib.LBM_EINVAL, "invalid box/stencil/precision")
        self.workspace = torch.empty(self.nbytes + 256, dtype=torch.uint8, device="cuda")
        ptr = self.workspace.data_ptr()
        ptr += (-ptr) % 256
        s = self.stream if self.stream is not None else torch.cuda.current_stream()
        self.stream_handle = s.cuda_stream
        self.ctx = lbm_create(self.box, self.tau, self.G, self.eos, st, pr, ptr, self.nbytes,
                              self.stream_handle)
        self.N = self.nx * self.ny * self.nz

    def close(self):
        if getattr(self, "ctx", None) is not None:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # thin forwards
    def init_drop(self, center, R, rho_in, rho_out, width=1.0):
        lbm_init_drop(self.ctx, center, R, rho_in, rho_out, width)

    def init_rho(self, rho):
        lbm_init_rho(self.ctx, np.asarray(rho, dtype=np.float64).reshape(-1))

    def set_populations(self, f):
        lbm_set_populations(self.ctx, np.asarray(f, dtype=np.float64).reshape(-1))

    def get_populations(self) -> np.ndarray:
        out = np.empty((19, self.nz, self.ny, self.nx))
        return lbm_get_populations(self.ctx, out)

    def step(self, n: int):
        lbm_step(self.ctx, n)

    def run_to_convergence(self, **kw):
        return lbm_run_to_convergence(self.ctx, **kw)

    def observables(self) -> lbm_obs:
        return lbm_observables(self.ctx)

    def rho(self) -> np.ndarray:
        out = np.empty((self.nz, self.ny, self.nx))
        return lbm_copy_rho(self.ctx, out)

    def velocity(self) -> np.ndarray:
        out = np.empty((3, self.nz, self.ny, self.nx))
        return lbm_copy_velocity(self.ctx, out)

    def rho_profile(self) -> np.ndarray:
        return lbm_rho_profile(self.ctx, self.nx // 2 + 1)

    def pt_profile(self) -> np.ndarray:
        return lbm_pt_profile(self.ctx, self.nx // 2 + 1)

    def pn_profile(self) -> np.ndarray:
        return lbm_pn_profile(self.ctx, self.nx // 2 + 1)

    def sigma_of_R(self, R):
        return lbm_sigma_of_R(self.ctx, R)

    def autotune(self, reps=8) -> int:
        return lbm_autotune(self.ctx, reps)

    def set_tile(self, code: int):
        lbm_set_tile(self.ctx, code)

    def get_tile(self) -> int:
        return lbm_get_tile(self.ctx)

    def storage_params(self):
        return lbm_storage_params(self.ctx)

    def save(self, path):
        lbm_save(self.ctx, path)

    def load(self, path):
        lbm_load(self.ctx, path)
