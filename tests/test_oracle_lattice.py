"""Pins of the oracle's velocity sets and weights (Sec. II; Sec. IV flat runs)."""
import itertools
from fractions import Fraction
from math import prod

import numpy as np
import pytest

from oracle import lattice as L


def test_d3q19_is_rest_plus_first_two_shells():
    vecs = {tuple(v) for v in L.D3Q19}
    expect = {(0, 0, 0)} | set(L.integer_shell(3, 1)) | set(L.integer_shell(3, 2))
    assert len(L.D3Q19) == 19 and vecs == expect
    # opposite pairs sit at (2k-1, 2k): the layout the C ABI documents
    for i in range(1, 19, 2):
        assert tuple(-L.D3Q19[i]) == tuple(L.D3Q19[i + 1])


def test_d3q19_weights_reproduce_maxwellian_moments_by_brute_force():
    w = L.lattice_weights(L.D3Q19)
    cs2 = Fraction(1, 3)
    vecs = [tuple(int(c) for c in v) for v in L.D3Q19]
    assert sum(w) == 1
    for a in range(3):
        assert sum(wi * v[a] for wi, v in zip(w, vecs)) == 0
    for a, b in itertools.product(range(3), repeat=2):
        assert sum(wi * v[a] * v[b] for wi, v in zip(w, vecs)) == (cs2 if a == b else 0)
    for a, b, c in itertools.product(range(3), repeat=3):
        assert sum(wi * v[a] * v[b] * v[c] for wi, v in zip(w, vecs)) == 0
    d = lambda i, j: 1 if i == j else 0
    for a, b, c, e in itertools.product(range(3), repeat=4):
        iso = cs2 * cs2 * (d(a, b) * d(c, e) + d(a, c) * d(b, e) + d(a, e) * d(b, c))
        assert sum(wi * v[a] * v[b] * v[c] * v[e] for wi, v in zip(w, vecs)) == iso
    assert [w[0], w[1], w[7]] == [Fraction(1, 3), Fraction(1, 18), Fraction(1, 36)]


def test_d1q3_weights():
    assert L.lattice_weights(L.D1Q3) == [Fraction(2, 3), Fraction(1, 6), Fraction(1, 6)]


def test_e4_weights_match_paper(paper):
    got = L.forcing_weights(L.STENCIL_SHELLS["E4"], 4)
    assert got == [Fraction(s) for s in paper["W_E4"]["values"]]


def test_d2q9_projection_matches_paper(paper):
    got = L.forcing_weights((1, 2), 4, dim=2)
    assert got == [Fraction(s) for s in paper["W_D2Q9"]["values"]]


def _double_fact(k):
    return prod(range(k - 1, 0, -2)) if k > 1 else 1


@pytest.mark.parametrize("name", ["E4", "E6", "E8"])
def test_forcing_stencils_are_isotropic_in_every_direction(name):
    """sum_a W_a (xi_a . n)^2k = e_2k (2k-1)!! for random unit n up to the stencil's order,
    and e_2 = 1 (Sec. II); the next order is NOT isotropic (the check has teeth)."""
    vecs, w = L.stencil(name)
    order = L.STENCIL_ORDER[name]
    rng = np.random.default_rng(0)
    dirs = rng.normal(size=(25, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    for k in range(1, order // 2 + 2):
        vals = np.array([(w * (vecs @ n) ** (2 * k)).sum() for n in dirs]) / _double_fact(2 * k)
        spread = np.ptp(vals) / abs(vals.mean())
        if 2 * k <= order:
            assert spread < 1e-12, (name, 2 * k, spread)
            if k == 1:
                assert abs(vals.mean() - 1.0) < 1e-13       # e_2 = 1
        else:
            assert spread > 1e-3, (name, 2 * k, spread)
    # odd moments vanish
    for n in dirs[:5]:
        assert abs((w * (vecs @ n)).sum()) < 1e-13
        assert abs((w * (vecs @ n) ** 3).sum()) < 1e-13


def test_stencil_sizes():
    assert [len(L.stencil(s)[0]) for s in ("E4", "E6", "E8")] == [18, 32, 92]
    v, _ = L.stencil("E4")
    assert np.array_equal(v, L.D3Q19[1:])


def test_lumped_e4_x_weight_equals_paper_2d_projection():
    """Flat fields: the x-neighbour weight of E4 lumps to W(1) + 4 W(2) = 1/2, the same as
    the paper's D2Q9 projection W(1) + 2 W(2) (the exact 1-D reduction the flat run uses)."""
    v, w = L.stencil("E4")
    lump = w[v[:, 0] == 1].sum()
    W2d = L.forcing_weights((1, 2), 4, dim=2)
    assert abs(lump - 0.5) < 1e-15
    assert W2d[0] + 2 * W2d[1] == Fraction(1, 2)
    wq = L.d3q19_weights()
    assert abs(wq[L.D3Q19[:, 0] == 0].sum() - 2 / 3) < 1e-15
    assert abs(wq[L.D3Q19[:, 0] == 1].sum() - 1 / 6) < 1e-15
