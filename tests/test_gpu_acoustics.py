"""Linear acoustics of a uniform phase on the GPU path, at a box the oracle's
acoustics pins do not reach (256 x 8 x 8, k = 2 pi / 256).

A standing wave n = n_bar + A sin(k x) started at rest oscillates at omega = c k,
c^2 = dP/dn of the bulk pressure of Eq. (10), and decays at the lattice
viscosity c_s^2 (tau - 1/2) (Secs. II, linearised Eqs. (3)-(8)); the lattice
corrections are O(k^2), 1e-5 here.  Holds for FP64 and shifted FP32 storage.
"""
import math

import numpy as np
import pytest

import paper_2105_08772_gb300 as P

pytestmark = pytest.mark.gpu

L, NY, NZ = 256, 8, 8


def _run(G, n_bar, prec, tau=1.0, periods=2.3, every=2):
    lat = P.Lattice(L, NY, NZ, tau=tau, G=G, psi="one_minus_exp", stencil="E4", prec=prec)
    k = 2 * math.pi / L
    mode = np.broadcast_to(np.sin(k * np.arange(L)), (NZ, NY, L))
    A = 1e-4
    lat.init_rho(n_bar + A * mode)
    psi, dpsi = 1 - math.exp(-n_bar), math.exp(-n_bar)
    c2 = 1.0 / 3.0 + G / 3.0 * psi * dpsi
    steps = int(periods * 2 * math.pi / (math.sqrt(c2) * k))
    t, a = [], []
    for s in range(0, steps, every):
        t.append(s)
        a.append(float(np.sum((lat.rho() - n_bar) * mode)))
        lat.step(every)
    lat.close()
    return np.array(t, dtype=float), np.array(a), k, c2


@pytest.mark.parametrize("prec", ["f64", "f32"])
# (the library takes only couplings below G_c = -4, where the phases coexist)
@pytest.mark.parametrize("G,n_bar", [(-4.5, 0.1), (-5.0, 0.1), (-5.0, 2.2)])
def test_gpu_sound_speed_and_damping(G, n_bar, prec):
    t, a, k, c2 = _run(G, n_bar, prec)
    i = [j for j in range(len(a) - 1) if a[j] * a[j + 1] < 0]
    z = [t[j] + (t[j + 1] - t[j]) * a[j] / (a[j] - a[j + 1]) for j in i]
    assert len(z) >= 4
    omega = math.pi / np.mean(np.diff(z))
    assert abs(omega / (math.sqrt(c2) * k) - 1) < 1e-3, (omega, math.sqrt(c2) * k)
    # envelope at the cosine's extrema, half a period apart
    half = math.pi / omega
    ext = []
    for m in range(5):
        j = int(np.argmin(np.abs(t - m * half)))
        lo, hi = max(0, j - 2), min(len(a), j + 3)
        jj = lo + int(np.argmax(np.abs(a[lo:hi])))
        ext.append((t[jj], abs(a[jj])))
    tt, amp = np.array(ext).T
    gamma = -np.polyfit(tt, np.log(amp), 1)[0] / k ** 2
    nu = (1.0 - 0.5) / 3.0
    assert abs(gamma / nu - 1) < 0.05, (gamma, nu)
