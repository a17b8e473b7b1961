"""Pins of the oracle's flat-interface run (Sec. IV, Eqs. (24), (25))."""
import numpy as np
import pytest

from oracle import eos as E
from oracle import flat


@pytest.fixture(scope="module")
def flat_runs():
    out = {}
    # psi = 1 - exp(-n), G = -5 (eps = 0.25); psi = exp(-1/n), G = -e^2 (1 + 0.25)
    out["one_minus_exp"] = (-5.0, flat.run_flat(-5.0, E.EOS("one_minus_exp"), Lx=100))
    Gx = -np.e ** 2 * 1.25
    out["exp_inv"] = (Gx, flat.run_flat(Gx, E.EOS("exp_inv"), Lx=100))
    return out


@pytest.mark.parametrize("kind", ["one_minus_exp", "exp_inv"])
def test_flat_normal_pressure_constant_to_machine_precision(flat_runs, kind):
    """Sec. II below Eq. (9): on the lattice, P_N is constant through a flat interface."""
    G, r = flat_runs[kind]
    assert r.converged
    assert r.pn_spread < 1e-13


@pytest.mark.parametrize("kind", ["one_minus_exp", "exp_inv"])
def test_flat_equilibrium_is_at_rest(flat_runs, kind):
    G, r = flat_runs[kind]
    assert r.max_u < 1e-12


@pytest.mark.parametrize("kind", ["one_minus_exp", "exp_inv"])
def test_flat_coexistence_matches_mechanical_stability_construction(flat_runs, kind):
    """Lattice bulk densities vs the psi'/psi construction (continuum limit of Eq. (9) at
    constant P_N): agreement to the size of the neglected higher-order terms, 1e-3."""
    G, r = flat_runs[kind]
    ng, nl, p0 = E.coexistence(E.EOS(kind), G, lo=0.02 if kind == "exp_inv" else 1e-3)
    assert abs(r.n_g - ng) / ng < 1e-3
    assert abs(r.n_l - nl) / nl < 1e-3


@pytest.mark.parametrize("kind", ["one_minus_exp", "exp_inv"])
def test_flat_sigma0_positive_and_both_interfaces_equal(flat_runs, kind):
    """Eq. (25) over the right half; the left interface carries the same tension."""
    G, r = flat_runs[kind]
    assert r.sigma0 > 0
    vecs, w = flat._lat.stencil("E4")
    psi = E.psi(r.n, E.EOS(kind), G)
    PN, PT = flat.pressure_NT(r.n, psi, G, vecs, w)
    Lx = len(r.n)
    left = np.trapezoid((PN - PT)[: Lx // 2 + 1], dx=1.0)
    assert abs(left - r.sigma0) / r.sigma0 < 1e-10


def test_flat_bulk_pressures_equal_bulk_eos(flat_runs):
    """Far from the interfaces P_N = P_T = P(n) (Eq. (10)) at both bulk densities."""
    G, r = flat_runs["one_minus_exp"]
    eos = E.EOS("one_minus_exp")
    assert abs(E.bulk_pressure(r.n_g, eos, G) - E.bulk_pressure(r.n_l, eos, G)) < 1e-12


def test_strip_profile_shape():
    """Eq. (24): liquid outside, gas inside a strip of width Lx/2 centred at Lx/2."""
    n = flat.strip_density(100, 1.9, 0.1)
    assert abs(n[0] - 1.9) < 1e-9 and abs(n[50] - 0.1) < 1e-9 and abs(n[99] - 1.9) < 1e-9
    assert abs(n[25] - 1.0) < 1e-9 and abs(n[75] - 1.0) < 1e-9
