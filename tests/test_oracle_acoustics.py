"""Pins on the oracle's 3-D transient: linear acoustics of a uniform phase.

A small standing density wave n = n_bar + A sin(k x) on a periodic box evolves,
to leading order in k, by the linearised continuity and momentum equations of
Eqs. (3)-(8) (Sec. II):
    d_t n' = -div j',   d_t j' = -grad(dP/dn n') + viscous terms,
with P the bulk pressure of Eq. (10), P = n c_s^2 + (G c_s^2 / 2) psi(n)^2
(the force of Eq. (8) is -grad of its non-ideal part, since sum_a W_a xi_a xi_a
= identity for every forcing stencil).  So the wave oscillates at
    omega = c k,   c^2 = dP/dn = c_s^2 + G c_s^2 psi(n_bar) psi'(n_bar),
and its amplitude decays as exp(-Gamma k^2 t) with Gamma = nu = c_s^2 (tau - 1/2),
the lattice kinematic viscosity of the BGK collision (Chapman-Enskog expansion
of Eqs. (3)-(6); the D3Q19 bulk viscosity 2 nu / 3 makes (4 nu / 3 + 2 nu / 3) / 2
= nu).  Both are closed forms independent of the oracle's code; the lattice
corrections are O(k^2) (0.1% at L = 64).  The force lowers c by 25% at
n_bar = 0.1 and G = -5, so a dropped, mis-signed or mis-weighted force term, a
wrong c_s^2 or a wrong relaxation rate fails these tests.
"""
import math

import numpy as np
import pytest

from oracle import eos as E
from oracle import lbm3d


def _wave(G, n_bar, L, axis, tau=1.0, stencil="E4", periods=2.2, A=1e-5):
    """Projection a(t) of n - n_bar on the initial mode for each step, and the
    closed-form c^2 (psi = 1 - exp(-n))."""
    m = lbm3d.Model(tau=tau, G=G, eos=E.EOS("one_minus_exp"), stencil=stencil)
    shape = [1, 1, 1]
    shape[2 - axis] = L                       # fields are [z, y, x]
    k = 2 * math.pi / L
    mode = np.sin(k * np.arange(L)).reshape(shape)
    f = lbm3d.init_from_density(n_bar + A * mode)
    psi, dpsi = 1 - math.exp(-n_bar), math.exp(-n_bar)
    c2 = 1.0 / 3.0 + G / 3.0 * psi * dpsi
    steps = int(periods * 2 * math.pi / (math.sqrt(c2) * k)) + 2
    a = np.empty(steps)
    for t in range(steps):
        a[t] = np.sum((lbm3d.density(f) - n_bar) * mode)
        f = lbm3d.step(f, m)
    return a, k, c2


@pytest.mark.parametrize("stencil", ["E4", "E6"])
@pytest.mark.parametrize("axis", [0, 2])
@pytest.mark.parametrize("G,n_bar", [(0.0, 1.0), (-5.0, 0.1), (-5.0, 2.2)])
def test_sound_speed_is_the_slope_of_the_bulk_pressure(G, n_bar, axis, stencil):
    a, k, c2 = _wave(G, n_bar, 64, axis, stencil=stencil)
    # zero crossings of A cos(omega t) e^{-Gamma k^2 t} are pi / omega apart
    z = [t + a[t] / (a[t] - a[t + 1]) for t in range(len(a) - 1) if a[t] * a[t + 1] < 0]
    assert len(z) >= 4
    omega = math.pi / np.mean(np.diff(z))
    assert abs(omega / (math.sqrt(c2) * k) - 1) < 3e-3, (omega, math.sqrt(c2) * k)


@pytest.mark.parametrize("tau", [0.8, 1.0, 1.3])
@pytest.mark.parametrize("G,n_bar", [(0.0, 1.0), (-5.0, 0.1)])
def test_sound_damping_is_the_lattice_viscosity(G, n_bar, tau):
    a, k, c2 = _wave(G, n_bar, 64, 0, tau=tau, periods=3.0)
    half = math.pi / (math.sqrt(c2) * k)      # extrema of the cosine, half a period apart
    ext = []
    for j in range(6):
        i = int(round(j * half))
        if i >= len(a):
            break
        lo, hi = max(0, i - 3), min(len(a), i + 4)
        t = lo + int(np.argmax(np.abs(a[lo:hi])))
        ext.append((t, abs(a[t])))
    t, amp = np.array(ext).T
    gamma = -np.polyfit(t, np.log(amp), 1)[0] / k ** 2
    nu = (tau - 0.5) / 3.0
    assert abs(gamma / nu - 1) < 1e-2, (gamma, nu)


def test_planted_force_scale_error_changes_the_sound_speed(monkeypatch):
    """A force off by a factor (here 1.5, as if the second shell's weight were
    doubled) moves omega far outside the bound the tests above use."""
    orig = lbm3d.sc_force
    monkeypatch.setattr(lbm3d, "sc_force", lambda *args: 1.5 * orig(*args))
    a, k, c2 = _wave(-5.0, 0.1, 64, 0)
    z = [t + a[t] / (a[t] - a[t + 1]) for t in range(len(a) - 1) if a[t] * a[t + 1] < 0]
    omega = math.pi / np.mean(np.diff(z))
    assert abs(omega / (math.sqrt(c2) * k) - 1) > 0.05
