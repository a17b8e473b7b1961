"""Pins of the oracle's D3Q19 Shan-Chen step (Sec. II, Eqs. (3)-(8))."""
import numpy as np
import pytest

import inputs
from oracle import eos as E
from oracle import flat
from oracle import lattice as L
from oracle import lbm3d

XI = lbm3d.XI.astype(np.float64)


def model(G=-5.0, tau=1.0, kind="one_minus_exp", stencil="E4", T=0.0):
    return lbm3d.Model(tau=tau, G=G, eos=E.EOS(kind, T=T), stencil=stencil)


def test_equilibrium_moments():
    """Eq. (6) (with the Hermite 1/2): sum f = n, sum xi f = n u, sum xi xi f = n cs2 d + n u u."""
    rng = np.random.default_rng(1)
    n = rng.uniform(0.1, 2.0, size=(4, 5, 6))
    u = rng.uniform(-0.1, 0.1, size=(3, 4, 5, 6))
    feq = lbm3d.equilibrium(n, u)
    assert np.max(np.abs(feq.sum(0) - n)) < 1e-14
    assert np.max(np.abs(np.einsum("ia,i...->a...", XI, feq) - n * u)) < 1e-14
    P = np.einsum("ia,ib,i...->ab...", XI, XI, feq)
    for a in range(3):
        for b in range(3):
            expect = n * u[a] * u[b] + (n / 3.0 if a == b else 0.0)
            assert np.max(np.abs(P[a, b] - expect)) < 1e-14


def test_guo_source_moments():
    """Eq. (5): sum F_i = 0, sum xi F_i = (1 - 1/2tau) F, sum xi xi F_i = (1 - 1/2tau)(uF + Fu)."""
    rng = np.random.default_rng(2)
    u = rng.uniform(-0.1, 0.1, size=(3, 3, 4, 5))
    F = rng.uniform(-0.01, 0.01, size=(3, 3, 4, 5))
    tau = 0.8
    Fi = lbm3d.guo_source(u, F, tau)
    k = 1 - 0.5 / tau
    assert np.max(np.abs(Fi.sum(0))) < 1e-16
    assert np.max(np.abs(np.einsum("ia,i...->a...", XI, Fi) - k * F)) < 1e-16
    M = np.einsum("ia,ib,i...->ab...", XI, XI, Fi)
    for a in range(3):
        for b in range(3):
            assert np.max(np.abs(M[a, b] - k * (u[a] * F[b] + F[a] * u[b]))) < 1e-16


def test_uniform_field_is_a_fixed_point():
    m = model()
    f = lbm3d.init_from_density(np.full((4, 5, 6), 0.8))
    g = lbm3d.run(f, m, 5)
    assert np.max(np.abs(g - f)) < 1e-15


@pytest.mark.parametrize("stencil", ["E4", "E6"])
def test_mass_and_momentum_conservation(stencil):
    """BGK + Guo conserve mass (Sec. II, sum Omega = 0, sum F_i = 0) and the total force of
    Eq. (8) vanishes on a periodic box, so total momentum is conserved too."""
    m = model(tau=0.8, stencil=stencil)
    f = inputs.random_populations((8, 7, 10), seed=3)
    M0 = f.sum()
    J0 = np.einsum("ia,izyx->a", XI, f)
    g = lbm3d.run(f, m, 60)
    assert abs(g.sum() - M0) / M0 < 1e-13
    J = np.einsum("ia,izyx->a", XI, g)
    assert np.max(np.abs(J - J0)) < 1e-12 * M0
    n, psi, F, u = lbm3d.macroscopic(g, m)
    assert np.max(np.abs(F.reshape(3, -1).sum(1))) < 1e-13


def test_total_momentum_changes_by_total_force():
    """One collision moves the momentum of every node by exactly F (Guo), so sum j changes by
    sum F = 0; checked node-wise: j_post = j + F."""
    m = model(tau=0.9)
    f = inputs.random_populations((6, 6, 6), seed=4)
    n, psi, F, u = lbm3d.macroscopic(f, m)
    feq = lbm3d.equilibrium(n, u)
    post = f - (f - feq) / m.tau + lbm3d.guo_source(u, F, m.tau)
    assert np.max(np.abs(np.einsum("ia,i...->a...", XI, post) - lbm3d.momentum(f) - F)) < 1e-15


def test_streaming_moves_each_population_along_its_velocity():
    m = model()
    f = lbm3d.init_from_density(np.full((5, 5, 5), 1.0))
    spike = np.zeros_like(f)
    spike[:, 2, 2, 2] = 1e-3      # tiny perturbation at one node
    g = lbm3d.step(f + spike, m) - lbm3d.step(f, m)
    for i in range(19):
        dst = ((2 + L.D3Q19[i, 2]) % 5, (2 + L.D3Q19[i, 1]) % 5, (2 + L.D3Q19[i, 0]) % 5)
        assert abs(g[i][dst]) > 0


def test_cubic_symmetry_of_a_centred_droplet():
    m = model()
    n = lbm3d.drop_density((11, 11, 11), (5, 5, 5), 3.0, 1.9, 0.12)
    f = lbm3d.run(lbm3d.init_from_density(n), m, 80)
    rho = lbm3d.density(f)
    for perm in ((0, 2, 1), (1, 0, 2), (2, 1, 0)):
        assert np.max(np.abs(rho - rho.transpose(perm))) < 1e-13
    for ax in range(3):
        assert np.max(np.abs(rho - np.flip(rho, axis=ax))) < 1e-13


def test_d3q19_on_flat_field_equals_d1q3_run():
    """A field uniform in y, z: the 3-D step reduces exactly to the D1Q3 flat run."""
    G, eos = -5.0, E.EOS("one_minus_exp")
    Lx = 40
    n1 = flat.strip_density(Lx, 1.88, 0.12)
    f1 = np.stack([flat.W1[i] * n1 for i in range(3)])
    vecs, w = L.stencil("E4")
    n3 = np.broadcast_to(n1, (3, 3, Lx)).copy()
    f3 = lbm3d.init_from_density(n3)
    m = model(G=G)
    for _ in range(300):
        f1 = flat.step(f1, G, 1.0, eos, vecs, w)
        f3 = lbm3d.step(f3, m)
    rho3 = lbm3d.density(f3)
    assert np.max(np.abs(rho3 - f1.sum(0)[None, None, :])) < 1e-13


def test_planted_mistake_in_equilibrium_is_caught(monkeypatch):
    """Dropping the 1/2 of Eq. (6) (the printed form) breaks the second-moment pin."""
    def bad_eq(n, u):
        uu = (u * u).sum(axis=0)
        out = np.empty((19,) + n.shape)
        for i in range(19):
            eu = sum(lbm3d.XI[i, a] * u[a] for a in range(3))
            out[i] = lbm3d.W[i] * n * (1 + eu * 3 + eu * eu * 9 - uu * 1.5)
        return out
    monkeypatch.setattr(lbm3d, "equilibrium", bad_eq)
    with pytest.raises(AssertionError):
        test_equilibrium_moments()


def test_planted_sign_error_in_force_is_caught(monkeypatch):
    """A sign slip in Eq. (8) destroys the droplet (it diffuses or blows up)."""
    m = model()
    n = lbm3d.drop_density((12, 12, 12), (6, 6, 6), 3.5, 1.9, 0.12)
    good = lbm3d.density(lbm3d.run(lbm3d.init_from_density(n), m, 150))
    orig = lbm3d.sc_force
    monkeypatch.setattr(lbm3d, "sc_force", lambda *a: -orig(*a))
    with np.errstate(all="ignore"):
        bad = lbm3d.density(lbm3d.run(lbm3d.init_from_density(n), m, 150))
    assert np.ptp(good) > 1.5
    assert not (np.isfinite(bad).all() and np.ptp(bad) > 1.5)


@pytest.mark.parametrize("stencil,tau", [("E4", 1.0), ("E4", 0.7), ("E6", 1.3)])
def test_step_equals_brute_force_node_loop(stencil, tau):
    """Brute force on a tiny box: Eqs. (3)-(8) evaluated node by node and population
    by population with explicit periodic indexing (no array shifts, scalar
    arithmetic), against the vectorised oracle step."""
    import math
    from oracle import eos as E
    from oracle import lattice as Lt
    rng = np.random.default_rng(5)
    nz, ny, nx = 5, 6, 7
    f = rng.uniform(0.02, 0.2, size=(19, nz, ny, nx))
    m = lbm3d.Model(tau=tau, G=-5.0, eos=E.EOS("one_minus_exp"), stencil=stencil)
    vecs, wts = Lt.stencil(stencil)
    xi = Lt.D3Q19
    w = Lt.d3q19_weights()
    cs2 = 1.0 / 3.0

    def n_at(z, y, x):
        return sum(f[i, z % nz, y % ny, x % nx] for i in range(19))

    def psi(n):
        return 1.0 - math.exp(-n)

    out = np.zeros_like(f)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                n = n_at(z, y, x)
                j = [sum(f[i, z, y, x] * xi[i][a] for i in range(19)) for a in range(3)]
                F = [0.0, 0.0, 0.0]
                for v, wv in zip(vecs, wts):
                    p = psi(n_at(z + int(v[2]), y + int(v[1]), x + int(v[0])))
                    for a in range(3):
                        F[a] += -m.G * cs2 * psi(n) * wv * p * v[a]
                u = [(j[a] + 0.5 * F[a]) / n for a in range(3)]
                uu = sum(ua * ua for ua in u)
                uF = sum(u[a] * F[a] for a in range(3))
                for i in range(19):
                    eu = sum(xi[i][a] * u[a] for a in range(3))
                    eF = sum(xi[i][a] * F[a] for a in range(3))
                    feq = w[i] * n * (1 + eu / cs2 + eu * eu / (2 * cs2 * cs2) - uu / (2 * cs2))
                    Fi = (1 - 0.5 / tau) * w[i] * (eF / cs2 + (eu * eF - cs2 * uF) / (cs2 * cs2))
                    post = f[i, z, y, x] - (f[i, z, y, x] - feq) / tau + Fi
                    out[i, (z + xi[i][2]) % nz, (y + xi[i][1]) % ny, (x + xi[i][0]) % nx] = post
    ref = lbm3d.step(f, m)
    assert np.max(np.abs(out - ref)) < 1e-14
