"""Host-side checks of the C ABI: the library loads, exports every declared symbol, and
rejects bad arguments before touching a GPU."""
import ctypes as C
import re
import subprocess
from pathlib import Path

import numpy as np
import pytest

import paper_2105_08772_gb300 as P
from paper_2105_08772_gb300 import _lib
from oracle import observables as O

ROOT = Path(__file__).resolve().parent.parent
HEADER = ROOT / "include" / "lbm.h"


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-zA-Z0-9_]+)\s*\(", text)))


def test_header_declares_what_the_binding_knows():
    assert declared_functions() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol():
    for name in declared_functions():
        assert hasattr(_lib.lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", str(_lib._LIB_PATH)], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lbm_\w+)", out))
    assert set(declared_functions()) <= exported


def test_struct_layout_matches_header(tmp_path):
    """ctypes mirrors of the header structs have the C compiler's sizes and offsets."""
    fields = [f for f, _ in _lib.lbm_obs._fields_]
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbm.h"', "int main(void) {",
           'printf("%zu %zu %zu\\n", sizeof(lbm_box), sizeof(lbm_eos), sizeof(lbm_obs));']
    src += [f'printf("%zu\\n", offsetof(lbm_obs, {f}));' for f in fields]
    src += ["return 0; }"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", str(ROOT / "include"), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out[:3]] == [C.sizeof(_lib.lbm_box), C.sizeof(_lib.lbm_eos),
                                         C.sizeof(_lib.lbm_obs)]
    assert [int(v) for v in out[3:]] == [getattr(_lib.lbm_obs, f).offset for f in fields]


def test_workspace_bytes():
    b = P.make_box(128, 128, 128)
    n = 128 ** 3
    got = P.lbm_workspace_bytes(b, 4, 1)
    assert got >= 2 * 19 * n * 4 + 3 * n * 4
    assert P.lbm_workspace_bytes(b, 4, 0) >= 2 * 19 * n * 8
    assert P.lbm_workspace_bytes(P.make_box(2, 8, 8), 4, 0) == 0     # too small for E4
    assert P.lbm_workspace_bytes(P.make_box(4, 8, 8), 6, 0) == 0     # too small for E6
    assert P.lbm_workspace_bytes(b, 5, 0) == 0                       # no such stencil
    assert P.lbm_workspace_bytes(b, 4, 7) == 0                       # no such precision
    assert P.lbm_workspace_bytes(P.make_box(1300, 1300, 1300), 4, 1) == 0   # >= 2^31 nodes
    assert P.lbm_workspace_bytes(P.make_box(1290, 1290, 1290), 4, 1) > 0


def _create(**kw):
    args = dict(box=P.make_box(16, 16, 16), tau=1.0, G=-5.0, eos=P.make_eos("one_minus_exp"),
                stencil=4, prec=0, ws=256 * 1024, nbytes=1 << 40, stream=0)
    args.update(kw)
    out = C.c_void_p()
    st = _lib.lib.lbm_create(args["box"], args["tau"], args["G"], args["eos"], args["stencil"],
                             args["prec"], C.c_void_p(args["ws"]), C.c_size_t(args["nbytes"]),
                             C.c_void_p(args["stream"]), C.byref(out))
    return st, _lib.lib.lbm_last_error(None).decode(), out


@pytest.mark.parametrize("kw,status,msg", [
    (dict(G=-3.9), _lib.LBM_EINVAL, "G_c = -4"),
    (dict(G=-7.0, eos=P.make_eos("exp_inv")), _lib.LBM_EINVAL, "exp(-1/n)"),
    (dict(tau=0.5), _lib.LBM_EINVAL, "tau"),
    (dict(box=P.make_box(2, 16, 16)), _lib.LBM_EINVAL, "sides >= 3"),
    (dict(box=P.make_box(4, 16, 16), stencil=8), _lib.LBM_EINVAL, "sides >= 5"),
    # node offsets inside a population plane are 32-bit in the kernels
    (dict(box=P.make_box(1300, 1300, 1300)), _lib.LBM_EINVAL, "below 2^31 nodes"),
    (dict(stencil=5), _lib.LBM_EINVAL, "stencil"),
    (dict(prec=3), _lib.LBM_EINVAL, "prec"),
    (dict(ws=0), _lib.LBM_EINVAL, "null"),
    (dict(ws=256 * 1024 + 8), _lib.LBM_EINVAL, "aligned"),
    (dict(nbytes=1000), _lib.LBM_ENOMEM, "needs"),
    (dict(eos=P.make_eos("cs", T=0.0), G=-1.0), _lib.LBM_EINVAL, "Carnahan"),
    (dict(eos=P.make_eos(9)), _lib.LBM_EINVAL, "kind"),
])
def test_create_rejects_bad_arguments_before_any_gpu_work(kw, status, msg):
    st, err, out = _create(**kw)
    assert st == status and msg in err and not out.value


def test_null_context_calls_fail_cleanly():
    assert _lib.lib.lbm_step(None, 1) == _lib.LBM_EINVAL
    assert _lib.lib.lbm_batch_autotune(None, 4, None) == _lib.LBM_EINVAL
    assert _lib.lib.lbm_observables(None, None) == _lib.LBM_EINVAL
    _lib.lib.lbm_destroy(None)
    assert _lib.lib.lbm_strerror(_lib.LBM_ENOTCONV) == b"not converged"


def test_tolman_fit_matches_oracle():
    rng = np.random.default_rng(5)
    Rs = rng.uniform(5, 40, size=30)
    bub = (rng.uniform(size=30) < 0.5).astype(np.int32)
    x = np.where(bub == 1, -1.0, 1.0) / Rs
    sig = 0.036 * (1 - 2 * 1.3 * x + 2.0 * x * x) + 1e-6 * rng.normal(size=30)
    for quad in (True, False):
        got = P.lbm_tolman_fit(Rs, sig, bub, quadratic=quad)
        ref = O.tolman_fit(Rs, sig, bub, quadratic=quad)
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-12)


def test_tolman_fit_skips_points_without_a_minimum():
    Rs = np.array([6.0, np.nan, 10.0, 14.0, 20.0])
    sig = np.array([0.03, np.nan, 0.032, 0.033, 0.034])
    s0, d, c = P.lbm_tolman_fit(Rs, sig, np.zeros(5, dtype=np.int32), quadratic=False)
    s0r, dr, _ = O.tolman_fit(Rs[np.isfinite(Rs)], sig[np.isfinite(sig)], np.zeros(4), quadratic=False)
    assert abs(s0 - s0r) < 1e-14 and abs(d - dr) < 1e-12
    with pytest.raises(P.LBMError):
        P.lbm_tolman_fit(Rs[:1], sig[:1], np.zeros(1, dtype=np.int32), quadratic=False)


@pytest.mark.parametrize("kind,G,tfrac", [("one_minus_exp", -4.2, 0), ("one_minus_exp", -5.0, 0),
                                          ("one_minus_exp", -6.0, 0), ("exp_inv", -np.e ** 2 * 1.1, 0),
                                          ("exp_inv", -np.e ** 2 * 1.293, 0), ("cs", -1.0, 0.8),
                                          ("cs", -1.0, 0.9)])
def test_coexistence_estimate_matches_oracle(kind, G, tfrac):
    """lbm_coexistence_estimate (bisection on n_g, Gauss-Legendre in log n) against the
    oracle's construction (bisection on p_0, adaptive quadrature): the same equal-area
    condition solved two independent ways."""
    from oracle import eos as E
    T = tfrac * E.cs_critical_temperature(E.EOS("cs"))[1] if kind == "cs" else 0.0
    ng, nl, p0 = P.coexistence_estimate(G, psi=kind, cs_T=T)
    lo = 0.02 if kind == "exp_inv" else 1e-3
    rg, rl, rp = E.coexistence(E.EOS(kind, T=T), G, lo=lo, hi=4.0 if kind != "cs" else 1.1 * nl)
    assert abs(ng - rg) < 1e-11 * rg and abs(nl - rl) < 1e-11 * rl and abs(p0 - rp) < 1e-11 * abs(rp)


def test_coexistence_estimate_rejects_no_loop():
    with pytest.raises(P.LBMError):
        P.coexistence_estimate(-3.9)             # above G_c = -4: no van der Waals loop
    with pytest.raises(P.LBMError):
        P.coexistence_estimate(-7.0)             # the construction's gas density has reached 0


@pytest.mark.parametrize("box,stencil,prec,tau,code", [
    # row chunks (nx % 4 == 0, nx >= 40): the moment kernel, 32 x 8 for E4 ...
    ((128, 128, 128), "E4", "f32", 1.0, 532080001),
    ((156, 156, 156), "E4", "f32", 1.0, 532080001),    # 3.8M nodes: prefetch depth 1
    ((160, 160, 160), "E4", "f32", 1.0, 532080002),    # 4.1M nodes: depth 2 in FP32
    ((160, 160, 160), "E4", "f64", 1.0, 532080001),
    ((128, 128, 128), "E4", "f32", 0.8, 532080001),    # same code; tau != 1 runs the chunked kernel
    ((256, 256, 256), "E6", "f32", 1.0, 532040001),    # ... 32 x 4 for the wider stencils
    # odd or narrow rows: the moment kernel with element copies
    ((127, 127, 127), "E4", "f32", 1.0, 632080001),
    ((158, 158, 158), "E4", "f32", 1.0, 632080001),
    ((36, 36, 36), "E4", "f32", 1.0, 632080001),
    ((16, 16, 16), "E4", "f64", 1.0, 632080001),
    ((255, 255, 255), "E8", "f64", 1.0, 632040001),
    # FP16: the moment kernel with an FP16 stage (E4, tau = 1, nx % 8 == 0, nx >= 48),
    # else the register-load kernel (kind 0, z chunk 16)
    ((128, 128, 128), "E4", "f16", 1.0, 532080002),
    ((128, 128, 128), "E4", "f16", 0.8, 32080016),
    ((40, 40, 40), "E4", "f16", 1.0, 32080016),
])
def test_default_tile_policy(box, stencil, prec, tau, code):
    """The kernel choice lbm_create starts from, queried on the host."""
    assert P.default_tile(*box, stencil=stencil, prec=prec, tau=tau) == code


@pytest.mark.parametrize("args", [
    ((64, 64, 64), 5, _lib.LBM_F32_SHIFTED, 1.0),
    ((64, 64, 64), _lib.LBM_E4, 3, 1.0),
    ((64, 64, 64), _lib.LBM_E4, _lib.LBM_F32_SHIFTED, 0.5),
    ((2, 64, 64), _lib.LBM_E4, _lib.LBM_F32_SHIFTED, 1.0),
    ((64, 64, 4), _lib.LBM_E6, _lib.LBM_F32_SHIFTED, 1.0),
])
def test_default_tile_rejects_what_create_rejects(args):
    box, stencil, prec, tau = args
    with pytest.raises(_lib.LBMError) as e:
        P.lbm_default_tile(P.make_box(*box), stencil, prec, tau)
    assert e.value.status == _lib.LBM_EINVAL


def test_batch_workspace_sizes_by_storage():
    """FP16 batches exist for the E4 stencil only (the FP16 moment kernel)."""
    box = P.make_box(64, 64, 64)
    f16 = _lib.PRECS["f16"]
    assert _lib.lib.lbm_batch_workspace_bytes(4, box, 4, f16) > 0
    assert _lib.lib.lbm_batch_workspace_bytes(4, box, 6, f16) == 0
    assert _lib.lib.lbm_batch_workspace_bytes(4, box, 4, _lib.PRECS["f32"]) > \
        _lib.lib.lbm_batch_workspace_bytes(4, box, 4, f16)
