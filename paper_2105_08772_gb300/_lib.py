"""ctypes binding of liblbm.so (argument marshalling only).

Every function here forwards to the C-ABI entry point of the same name
declared in include/lbm.h; no arithmetic of the method happens in Python.
The library is built in-tree by ``paper_2105_08772_gb300.build``; if it is
missing this module raises at import (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

_LIB_PATH = Path(__file__).resolve().parent / "liblbm.so"

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENUMERIC, LBM_ENOTCONV = 0, 1, 2, 3, 4, 5
LBM_ENOMIN, LBM_ECOLLAPSE, LBM_EOFFCENTER, LBM_ETIMEOUT = 6, 7, 8, 9
LBM_PSI_EXP_INV, LBM_PSI_ONE_MINUS_EXP, LBM_PSI_CS = 0, 1, 2
LBM_E4, LBM_E6, LBM_E8 = 4, 6, 8
LBM_F64, LBM_F32_SHIFTED, LBM_F16_SHIFTED = 0, 1, 2

PSI_KINDS = {"exp_inv": LBM_PSI_EXP_INV, "one_minus_exp": LBM_PSI_ONE_MINUS_EXP, "cs": LBM_PSI_CS}
STENCILS = {"E4": LBM_E4, "E6": LBM_E6, "E8": LBM_E8}
PRECS = {"f64": LBM_F64, "f32": LBM_F32_SHIFTED, "f16": LBM_F16_SHIFTED}

# exported symbols (must match include/lbm.h)
EXPORTS = (
    "lbm_workspace_bytes", "lbm_create", "lbm_destroy", "lbm_init_drop", "lbm_init_rho",
    "lbm_set_populations", "lbm_get_populations", "lbm_step", "lbm_run_to_convergence",
    "lbm_observables", "lbm_rho_profile", "lbm_pt_profile", "lbm_sigma_of_R", "lbm_copy_rho",
    "lbm_copy_velocity", "lbm_save", "lbm_load", "lbm_autotune", "lbm_set_tile", "lbm_get_tile",
    "lbm_default_tile",
    "lbm_storage_params", "lbm_density_moments_noalloc", "lbm_batch_workspace_bytes",
    "lbm_batch_create", "lbm_batch_enqueue", "lbm_batch_run", "lbm_batch_result", "lbm_batch_autotune",
    "lbm_batch_last_error", "lbm_batch_destroy", "lbm_pn_profile", "lbm_flat_workspace_bytes",
    "lbm_flat_interface", "lbm_coexistence_estimate", "lbm_group_workspace_bytes", "lbm_group_create",
    "lbm_group_step", "lbm_group_last_error", "lbm_group_destroy",
    "lbm_strerror", "lbm_last_error", "lbm_tolman_fit",
    "lbm_slab_partition", "lbm_slab_halo_mask", "lbm_set_populations_storage", "lbm_state_plane",
    "lbm_halo_copy",
)


class lbm_box(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)]


class lbm_eos(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.c_double), ("b", C.c_double), ("Rgas", C.c_double),
                ("T", C.c_double)]


class lbm_obs(C.Structure):
    _fields_ = [("n_in", C.c_double), ("n_out", C.c_double), ("P_in", C.c_double),
                ("P_out", C.c_double), ("dP", C.c_double), ("mass", C.c_double),
                ("com", C.c_double * 3), ("R_e", C.c_double), ("C", C.c_double), ("D", C.c_double),
                ("R_s", C.c_double), ("sigma_s", C.c_double), ("max_u", C.c_double),
                ("du", C.c_double), ("dP_rel_change", C.c_double), ("steps", C.c_longlong),
                ("status_bits", C.c_uint), ("criterion", C.c_int)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if name == "com" else v
        return out


_P = C.c_void_p
_D = C.POINTER(C.c_double)


def _load():
    if not _LIB_PATH.exists():
        raise ImportError(f"{_LIB_PATH} is missing: build it with "
                          "`python paper_2105_08772_gb300/build.py` (there is no CPU fallback)")
    lib = C.CDLL(str(_LIB_PATH))
    sig = {
        "lbm_workspace_bytes": (C.c_size_t, [lbm_box, C.c_int, C.c_int]),
        "lbm_create": (C.c_int, [lbm_box, C.c_double, C.c_double, lbm_eos, C.c_int, C.c_int, _P,
                                 C.c_size_t, _P, C.POINTER(_P)]),
        "lbm_destroy": (None, [_P]),
        "lbm_init_drop": (C.c_int, [_P, _D, C.c_double, C.c_double, C.c_double, C.c_double]),
        "lbm_init_rho": (C.c_int, [_P, _D]),
        "lbm_set_populations": (C.c_int, [_P, _D]),
        "lbm_get_populations": (C.c_int, [_P, _D]),
        "lbm_step": (C.c_int, [_P, C.c_longlong]),
        "lbm_run_to_convergence": (C.c_int, [_P, C.c_longlong, C.c_longlong, C.c_double, C.c_double,
                                             C.POINTER(C.c_longlong), C.POINTER(C.c_int)]),
        "lbm_observables": (C.c_int, [_P, C.POINTER(lbm_obs)]),
        "lbm_rho_profile": (C.c_int, [_P, _D, C.c_longlong]),
        "lbm_pt_profile": (C.c_int, [_P, _D, C.c_longlong]),
        "lbm_sigma_of_R": (C.c_int, [_P, _D, _D, _D, C.c_longlong]),
        "lbm_copy_rho": (C.c_int, [_P, _D]),
        "lbm_copy_velocity": (C.c_int, [_P, _D]),
        "lbm_save": (C.c_int, [_P, C.c_char_p]),
        "lbm_load": (C.c_int, [_P, C.c_char_p]),
        "lbm_autotune": (C.c_int, [_P, C.c_int, C.POINTER(C.c_longlong)]),
        "lbm_set_tile": (C.c_int, [_P, C.c_longlong]),
        "lbm_get_tile": (C.c_int, [_P, C.POINTER(C.c_longlong)]),
        "lbm_default_tile": (C.c_int, [lbm_box, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_longlong)]),
        "lbm_storage_params": (C.c_int, [_P, _D, _D]),
        "lbm_strerror": (C.c_char_p, [C.c_int]),
        "lbm_last_error": (C.c_char_p, [_P]),
        "lbm_tolman_fit": (C.c_int, [_D, _D, C.POINTER(C.c_int), C.c_longlong, C.c_int, _D, _D, _D]),
        "lbm_density_moments_noalloc": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, _P, _P]),
        "lbm_batch_workspace_bytes": (C.c_size_t, [C.c_int, lbm_box, C.c_int, C.c_int]),
        "lbm_batch_create": (C.c_int, [C.c_int, lbm_box, C.c_int, C.c_int, _P, C.c_size_t, _P, C.POINTER(_P)]),
        "lbm_batch_enqueue": (C.c_int, [_P, lbm_box, C.c_double, C.c_double, lbm_eos, _D, C.c_double,
                                        C.c_double, C.c_double, C.c_double, C.POINTER(C.c_int)]),
        "lbm_batch_run": (C.c_int, [_P, C.c_longlong, C.c_longlong, C.c_double, C.c_double,
                                    C.POINTER(C.c_longlong)]),
        "lbm_batch_result": (C.c_int, [_P, C.c_int, C.POINTER(lbm_obs)]),
        "lbm_batch_autotune": (C.c_int, [_P, C.c_int, C.POINTER(C.c_longlong)]),
        "lbm_batch_last_error": (C.c_char_p, [_P]),
        "lbm_batch_destroy": (None, [_P]),
        "lbm_pn_profile": (C.c_int, [_P, _D, C.c_longlong]),
        "lbm_flat_workspace_bytes": (C.c_size_t, [C.c_int, C.c_int, C.c_int]),
        "lbm_coexistence_estimate": (C.c_int, [lbm_eos, C.c_double, _D, _D, _D]),
        "lbm_group_workspace_bytes": (C.c_size_t, [C.c_int]),
        "lbm_group_create": (C.c_int, [C.POINTER(_P), C.c_int, _P, C.c_size_t, _P, C.POINTER(_P)]),
        "lbm_group_step": (C.c_int, [_P, C.c_longlong]),
        "lbm_group_last_error": (C.c_char_p, [_P]),
        "lbm_group_destroy": (None, [_P]),
        "lbm_slab_partition": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]),
        "lbm_slab_halo_mask": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_uint)]),
        "lbm_set_populations_storage": (C.c_int, [_P, _D, C.c_double, C.c_double]),
        "lbm_state_plane": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(_P), C.POINTER(C.c_size_t)]),
        "lbm_halo_copy": (C.c_int, [_P, C.c_int, _P, C.c_int, C.c_uint]),
        "lbm_flat_interface": (C.c_int, [C.c_double, C.c_double, lbm_eos, C.c_int, C.c_int, C.c_int,
                                         C.c_double, C.c_double, C.c_longlong, C.c_double, _P,
                                         C.c_size_t, _P, _D, _D, _D, C.POINTER(C.c_longlong)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{lib.lbm_strerror(status).decode()} ({status}): {message}")
        self.status = status


def check(status: int, ctx=None) -> int:
    """Raise LBMError for a non-zero status, with the library's last message."""
    if status != LBM_OK:
        raise LBMError(status, lib.lbm_last_error(ctx).decode())
    return status
