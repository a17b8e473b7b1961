"""Pins of the oracle's pseudopotentials, bulk pressure and critical couplings."""
import numpy as np
import pytest

from oracle import eos as E
from oracle import lattice as L
from oracle import lbm3d
from oracle import observables as O


@pytest.mark.parametrize("kind", ["exp_inv", "one_minus_exp"])
def test_critical_coupling_matches_paper(kind, paper):
    n_c, G_c = E.critical_point(E.EOS(kind))
    printed = paper["G_c_cs2"][kind]
    assert round(G_c / 3.0, 3) == printed
    # closed forms: psi'^2 + psi psi'' = 0 at n_c = 1 (exp(-1/n)) and ln 2 (1 - exp(-n))
    exact = {"exp_inv": (1.0, -np.e ** 2), "one_minus_exp": (np.log(2.0), -4.0)}[kind]
    assert abs(n_c - exact[0]) < 1e-7 and abs(G_c - exact[1]) < 1e-7


def test_bulk_pressure_has_inflection_at_critical_point():
    for kind in ("exp_inv", "one_minus_exp"):
        eos = E.EOS(kind)
        n_c, G_c = E.critical_point(eos)
        h = 1e-3
        P = lambda n: E.bulk_pressure(n, eos, G_c)
        assert abs((P(n_c + h) - P(n_c - h)) / (2 * h)) < 1e-6
        assert abs((P(n_c + h) - 2 * P(n_c) + P(n_c - h)) / h ** 2) < 1e-4


@pytest.mark.parametrize("kind,G", [("one_minus_exp", -5.0), ("exp_inv", -9.2), ("cs", -1.0)])
def test_uniform_field_pressure_tensor_is_bulk_pressure(kind, G):
    """Eq. (9) on a uniform field equals P(n) delta (Eq. (10), e_2 = 1) -- brute force."""
    eos = E.EOS(kind, T=0.085) if kind == "cs" else E.EOS(kind)
    for stencil in ("E4", "E6", "E8"):
        vecs, w = L.stencil(stencil)
        for n0 in (0.1, 0.3, 1.7):
            if kind == "cs" and n0 > 0.4:
                continue
            n = np.full((5, 6, 7), n0)
            psi = E.psi(n, eos, G)
            P = O.pressure_tensor(n, psi, G, vecs, w)
            Pb = E.bulk_pressure(n0, eos, G)
            for a in range(3):
                for b in range(3):
                    expect = Pb if a == b else 0.0
                    assert np.max(np.abs(P[a, b] - expect)) < 1e-15


def test_cs_mapping_reproduces_carnahan_starling():
    eos = E.EOS("cs", T=0.08)
    n = np.linspace(0.01, 0.4, 50)
    assert np.max(np.abs(E.bulk_pressure(n, eos, -1.0) - E.p_cs(n, eos))) < 1e-15


def test_cs_critical_point_textbook():
    """Carnahan-Starling with a = 1, b = 4, R = 1: b n_c = 0.5218, b R T_c / a = 0.3773."""
    n_c, T_c = E.cs_critical_temperature(E.EOS("cs"))
    assert abs(4 * n_c - 0.5218) < 2e-4
    assert abs(4 * T_c - 0.3773) < 2e-4


def test_coexistence_construction_is_consistent():
    eos = E.EOS("one_minus_exp")
    ng, nl, p0 = E.coexistence(eos, -5.0)
    assert abs(E.bulk_pressure(ng, eos, -5.0) - p0) < 1e-14
    assert abs(E.bulk_pressure(nl, eos, -5.0) - p0) < 1e-14
    # coexistence widens with |G|, and closes towards n_c as G -> G_c
    ng2, nl2, _ = E.coexistence(eos, -6.0)
    assert ng2 < ng and nl2 > nl
    ng3, nl3, _ = E.coexistence(eos, -4.05)
    assert abs(ng3 - np.log(2)) < 0.25 and abs(nl3 - np.log(2)) < 0.25


def test_psi_rejects_unknown_kind():
    with pytest.raises(ValueError):
        E.psi(1.0, E.EOS("nope"), -5.0)
