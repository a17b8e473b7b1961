"""Flat-interface coexistence on the GPU (lbm_flat_interface) against the oracle.

Sec. IV: the bulk densities of a flat interface (strip of Eq. (24)) initialise
the droplets and bubbles, and sigma_0 follows from Eq. (25).  The GPU runs the
strip on a thin periodic D3Q19 box; a field uniform in y and z makes that run
the oracle's exact D1Q3 reduction, so after the same number of steps the two
agree to rounding.
"""
import numpy as np
import pytest

from oracle import eos as E
from oracle import flat

P = pytest.importorskip("paper_2105_08772_gb300")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("psi,G,stencil", [("one_minus_exp", -5.0, "E4"),
                                           ("exp_inv", -np.e ** 2 * 1.25, "E4"),
                                           ("one_minus_exp", -5.5, "E6"),
                                           ("one_minus_exp", -4.6, "E8")])
def test_flat_fixed_steps_match_oracle(psi, G, stencil):
    """Same start (Eq. (24)), same 8192 steps: n_g, n_l and sigma_0 to FP64 rounding."""
    Lx, steps, nl0, ng0 = 64, 8192, 1.9, 0.15
    ref = flat.run_flat(G, E.EOS(psi), stencil=stencil, Lx=Lx, n_l0=nl0, n_g0=ng0,
                        max_steps=steps, tol_n=-1.0)
    assert ref.steps == steps
    st, ng, nl, s0, done = P.flat_interface(G, psi=psi, stencil=stencil, prec="f64", Lx=Lx,
                                            rho_l0=nl0, rho_g0=ng0, max_steps=steps, tol_du=-1.0)
    assert done == steps and st == P.LBM_ENOTCONV
    assert abs(ng - ref.n_g) < 1e-11 and abs(nl - ref.n_l) < 1e-11
    assert abs(s0 - ref.sigma0) < 1e-11 * max(1.0, abs(ref.sigma0))


@pytest.mark.parametrize("G", [-4.6, -5.0, -5.5, -6.0])
def test_flat_converged_coexistence_matches_oracle(G):
    """Run to rest (delta u < 1e-13): the oracle's converged coexistence, and P_N flat."""
    eos = E.EOS("one_minus_exp")
    ng0, nl0, _ = E.coexistence(eos, G)
    ref = flat.run_flat(G, eos, Lx=100)
    assert ref.converged
    st, ng, nl, s0, done = P.flat_interface(G, Lx=100, rho_l0=nl0, rho_g0=ng0, tol_du=1e-13)
    assert st == P.LBM_OK and done < 400_000
    assert abs(ng - ref.n_g) < 1e-10 * ref.n_g and abs(nl - ref.n_l) < 1e-10 * ref.n_l
    assert abs(s0 - ref.sigma0) < 1e-9 * ref.sigma0


def test_flat_f32_storage_close_to_f64():
    """FP32 storage (shifted populations) run for the steps FP64 needed to reach rest
    (~4e4) lands on the FP64 coexistence: n_l to 1e-5, n_g to 3e-4 (its FP32 rounding
    relative to the storage shift n0 ~ 1 is ~8x larger than relative to n_g), sigma_0
    to 1e-3."""
    st64, ng64, nl64, s64, done = P.flat_interface(-5.0, Lx=100, prec="f64", tol_du=1e-13)
    st32, ng32, nl32, s32, _ = P.flat_interface(-5.0, Lx=100, prec="f32", max_steps=done,
                                                tol_du=-1.0)
    assert st64 == P.LBM_OK and st32 == P.LBM_ENOTCONV
    assert abs(ng32 - ng64) < 3e-4 * ng64 and abs(nl32 - nl64) < 1e-5 * nl64, (ng32, ng64, nl32, nl64)
    assert abs(s32 - s64) < 1e-3 * s64, (s32, s64)


def test_flat_rejects_bad_arguments():
    with pytest.raises(P.LBMError):
        P.flat_interface(-5.0, Lx=4)
    with pytest.raises(P.LBMError):
        P.flat_interface(-5.0, rho_l0=0.1, rho_g0=1.9)
