"""Pins of the oracle's observables (Eq. (9), Sec. III Eqs. (11), (12), (21), (22), Sec. IV)."""
import numpy as np
import pytest

import inputs
from oracle import eos as E
from oracle import lbm3d
from oracle import observables as O


def synthetic_line(rmax=30, R0=9.0, P_in=0.045, P_out=0.03, dip=0.03, width=1.3):
    """A droplet-like P_T(r): P_in inside, P_out outside and a tension dip at the interface
    sized so that Laplace holds roughly (dP ~ 2 sigma / R)."""
    r = np.arange(rmax + 1, dtype=np.float64)
    step = P_out + (P_in - P_out) / (1 + np.exp((r - R0) / width))
    return step - dip * np.exp(-((r - R0) / width) ** 2), P_in, P_out


def test_sigma_closed_form_identities():
    """Universal curve sigma[R]/sigma_s (Sec. III below Eq. (22)), sigma_s = dP R_s/2 (Eq. (12)),
    and the generalised Laplace law Eq. (11) with the closed-form derivative."""
    PT, P_in, P_out = synthetic_line()
    dP = P_in - P_out
    C, D = O.line_integrals(PT, P_out)
    Rs = O.surface_of_tension(dP, C)
    assert np.isfinite(Rs) and Rs > 0
    R = np.linspace(0.3 * Rs, 3 * Rs, 101)
    sig, _ = O.sigma_of_R(R, dP, C, D)
    sig_s = O.sigma_of_R(Rs, dP, C, D)[0]
    assert abs(sig_s - 0.5 * dP * Rs) < 1e-15
    assert np.max(np.abs(sig / sig_s - ((Rs / R) ** 2 / 3 + 2 * R / (3 * Rs)))) < 1e-12
    # sigma'[R] of Eq. (22) = d sigma/dR (closed form) + 2 D / R^2
    dclosed = dP / 3 - 2 * C / R ** 3
    _, dsig = O.sigma_of_R(R, dP, C, D)
    assert np.max(np.abs(dsig - dclosed - 2 * D / R ** 2)) < 1e-15
    assert np.max(np.abs(2 * sig / R + dclosed - dP)) < 1e-15
    assert sig.min() >= sig_s - 1e-15


def test_sigma_integrals_by_brute_force_quadrature():
    """Eq. (21) by brute force: the step part int (r/R)^2 (P_J - P_out) dr by a fine midpoint
    sum must equal dP R / 3 exactly (to the sum's error); with the node trapezoid for the P_T
    part it reproduces sigma[R].  A fine sum with P_T interpolated linearly between nodes agrees
    to the trapezoid's O(h^2) error."""
    PT, P_in, P_out = synthetic_line()
    dP = P_in - P_out
    C, D = O.line_integrals(PT, P_out)
    rr = np.linspace(0, len(PT) - 1, 600001)
    mid = 0.5 * (rr[1:] + rr[:-1])
    dr = rr[1] - rr[0]
    PTm = np.interp(mid, np.arange(len(PT)), PT)
    for R in (5.0, 8.3, 12.0):
        PJ = np.where(mid < R, P_in, P_out)
        step_part = np.sum((mid / R) ** 2 * (PJ - P_out)) * dr
        closed = O.sigma_of_R(R, dP, C, D)[0]
        assert abs(step_part + C / R ** 2 - closed) < 1e-9
        brute = np.sum((mid / R) ** 2 * (PJ - PTm)) * dr
        assert abs(brute - closed) / abs(closed) < 1e-2


def test_paper_grid_minimum_agrees_with_closed_form():
    """The paper's route (grid + parabola): the minimum value sigma[R_s] matches dP R_s / 2
    well inside the 1e-3 the Sec. IV footnote reports, and R_s agrees with the closed form to
    the difference of the two P_T quadratures (below 1%)."""
    PT, P_in, P_out = synthetic_line()
    dP = P_in - P_out
    C, D = O.line_integrals(PT, P_out)
    Rs = O.surface_of_tension(dP, C)
    Rg, sg = O.sigma_min_by_grid(PT, P_in, P_out, 0.5 * Rs, 1.5 * Rs, m=2001, sub=512)
    assert abs(sg - 0.5 * dP * Rg) / (0.5 * dP * Rg) < 1e-5
    assert abs(Rg - Rs) / Rs < 1e-2


def test_no_minimum_when_C_has_the_wrong_sign():
    assert np.isnan(O.surface_of_tension(0.01, -0.5))
    assert np.isnan(O.surface_of_tension(-0.01, 0.5))


def test_equimolar_radius_of_a_sharp_sphere():
    """Sec. IV: M = 4 pi R_e^3 n_in/3 + (V - 4 pi R_e^3/3) n_out -- exact for a mass built
    from a sphere of known volume."""
    V, n_in, n_out, R = 50.0 ** 3, 1.9, 0.12, 11.3
    M = 4 * np.pi * R ** 3 * n_in / 3 + (V - 4 * np.pi * R ** 3 / 3) * n_out
    assert abs(O.equimolar_radius(M, V, n_in, n_out) - R) < 1e-12
    # bubble: n_in < n_out
    M = 4 * np.pi * R ** 3 * n_out / 3 + (V - 4 * np.pi * R ** 3 / 3) * n_in
    assert abs(O.equimolar_radius(M, V, n_out, n_in) - R) < 1e-12


def test_lattice_sphere_equimolar_radius_close_to_geometric():
    n = lbm3d.drop_density((40, 40, 40), (20, 20, 20), 10.0, 1.9, 0.12, width=0.3)
    R_e = O.equimolar_radius(n.sum(), n.size, 1.9, 0.12)
    assert abs(R_e - 10.0) < 0.05


@pytest.mark.parametrize("L", [15, 16])
def test_centre_of_mass_of_centred_field_is_centre(L):
    n = lbm3d.drop_density((L, L, L), (L // 2,) * 3, L / 4, 1.9, 0.12)
    com = O.centre_of_mass(n, n[0, 0, 0])
    assert np.max(np.abs(com - L // 2)) < 1e-12
    # shifted by one node in x: the centre of mass follows
    com2 = O.centre_of_mass(np.roll(n, 1, axis=2), n[0, 0, 0])
    assert abs(com2[0] - (L // 2 + 1)) < 1e-2


def test_far_node_is_paper_corner_for_odd_sizes():
    assert O.far_node((41, 41, 41)) == (40, 40, 40)
    assert O.centre_node((41, 41, 41)) == (20, 20, 20)
    assert O.far_node((16, 17, 18)) == (0, 16, 0)


def test_tolman_fit_recovers_known_coefficients():
    s0, d, c = 0.0364, 1.7, 3.0
    Rs = np.array([6, 8, 10, 14, 20, 30, 6, 9, 12, 25.0])
    bub = np.array([0] * 6 + [1] * 4)
    x = np.where(bub == 1, -1.0, 1.0) / Rs
    sig = s0 * (1 - 2 * d * x + c * x * x)
    got = O.tolman_fit(Rs, sig, bub, quadratic=True)
    assert np.allclose(got, (s0, d, c), rtol=1e-10)
    s0l, dl, _ = O.tolman_fit(Rs, s0 * (1 - 2 * d * x), bub, quadratic=False)
    assert abs(s0l - s0) < 1e-14 and abs(dl - d) < 1e-12


@pytest.fixture(scope="module")
def converged_small_droplet():
    m = lbm3d.Model(tau=1.0, G=-6.0, eos=E.EOS("one_minus_exp"))
    ng, nl, _ = E.coexistence(m.eos, m.G)
    n = lbm3d.drop_density((16, 16, 16), (8, 8, 8), 4.0, nl, ng)
    res = O.run_to_convergence(lbm3d.init_from_density(n), m, max_steps=12288)
    return m, res, nl - ng


def test_small_droplet_converges_by_a_paper_criterion(converged_small_droplet):
    m, res, contrast = converged_small_droplet
    assert res.criterion in ("dP", "du")
    ob = O.observe(res.f, m, contrast0=contrast)
    assert not (ob.status & O.ST_OFF_CENTER)
    assert not (ob.status & O.ST_COLLAPSED)
    assert ob.dP > 0 and ob.R_e > 0


def test_converged_droplet_satisfies_mechanical_equilibrium_moment(converged_small_droplet):
    """The n = d - 1 identity of Eq. (17): int 2 r (P_T - P_out) dr = 0 at equilibrium."""
    m, res, _ = converged_small_droplet
    ob = O.observe(res.f, m)
    r = np.arange(len(ob.PT_line))
    scale = np.trapezoid(2 * r * np.abs(ob.PT_line - ob.P_out), r)
    assert abs(2 * ob.D) < 0.05 * scale


def test_delta_hat_signs_and_flat_limit():
    """hat-delta_+- = +-(R_e - R_s) (Sec. IV).  With R_e - R_s = delta + k/R_s for droplets
    and R_s - R_e = delta - k/R_s for bubbles -- one line delta + k x in the signed
    curvature -- the flat limit is delta exactly; two runs fix it by hand."""
    assert O.delta_hat(10.4, 10.0, False) == pytest.approx(0.4)
    assert O.delta_hat(9.7, 10.0, True) == pytest.approx(0.3)
    delta, k = 0.57, -1.9
    Rs = np.array([8.0, 12.0, 17.0, 25.0, 9.0, 14.0, 21.0, 33.0])
    bub = np.array([False] * 4 + [True] * 4)
    x = np.where(bub, -1.0, 1.0) / Rs
    Re = Rs + np.where(bub, -1.0, 1.0) * (delta + k * x)
    assert O.delta_hat_flat_limit(Re, Rs, bub) == pytest.approx(delta, rel=1e-12)
    # a droplet at R_s = 10 and a bubble at R_s = 20: the line through (0.1, h1) and
    # (-0.05, h2) meets x = 0 at h2 + (h1 - h2) / 3
    h1, h2 = 0.9, 0.6
    got = O.delta_hat_flat_limit([10.0 + h1, 20.0 - h2], [10.0, 20.0], [False, True])
    assert got == pytest.approx(h2 + (h1 - h2) / 3.0, rel=1e-12)
    # the bubble sign matters: treating bubbles like droplets moves the limit
    assert abs(O.delta_hat_flat_limit(Re, Rs, np.zeros(8, dtype=bool)) - delta) > 0.1
