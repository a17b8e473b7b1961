"""Exact mirror symmetry of the GPU step.

A drop centred on the centre node of a periodic box is symmetric under the three
reflections about that node, and so is the method's exact dynamics.  The kernels
sum the populations, the momentum and the force in mirror-exact orders
(lbm_kernels.cuh, sum19 / sc_force_pairs), so the stored field stays bitwise
symmetric in every storage precision and kernel kind; the centre of mass cannot
leave the centre node (the paper's centring test, Sec. IV).  Rounding of shifted
FP16 storage used to break this symmetry and let drops drift.
"""
import numpy as np
import pytest

import paper_2105_08772_gb300 as P

pytestmark = pytest.mark.gpu


def mirrored(a, axis, c):
    n = a.shape[axis]
    idx = (2 * c - np.arange(n)) % n
    return np.take(a, idx, axis=axis)


@pytest.mark.parametrize("L,prec,bubble,tile", [
    (64, "f32", False, 732080001),   # the TMA kernel (kind 7)
    (64, "f32", True, 0),            # row chunks (kind 5)
    (41, "f32", False, 0),           # odd box: element copies (kind 6)
    (48, "f16", False, 0),           # FP16 stage (kind 5)
    (40, "f16", True, 0),            # FP16 register-load kernel (kind 0)
    (36, "f64", False, 0),
])
def test_drop_stays_bitwise_mirror_symmetric(L, prec, bubble, tile):
    c = L // 2 if L % 2 == 0 else (L - 1) // 2
    lat = P.Lattice(L, L, L, G=-5.0, prec=prec)
    try:
        if tile:
            lat.set_tile(tile)
        a, b = (0.12, 1.89) if bubble else (1.89, 0.12)
        lat.init_drop((c, c, c), L / 4.0, a, b)
        lat.step(400)
        rho = lat.rho()                          # [z, y, x]
        for axis in range(3):
            assert np.array_equal(rho, mirrored(rho, axis, c)), (axis, lat.get_tile())
        ob = lat.observables()
        assert np.allclose(list(ob.com), [c, c, c], rtol=0, atol=1e-9), list(ob.com)
        assert not (ob.status_bits & 4), ob.status_bits          # not off-centre
    finally:
        lat.close()
