"""1000-step density parity with the FP64 oracle at the sizes where the library's
default kernels run several z chunks (64^3: row-chunk moment kernel) and take
element copies (41^3, odd: kind 6), on the paper's droplet workload (Sec. IV,
Eq. (23), at the flat-interface densities).  Bounds: 1e-4 relative on the
FP32-shifted path, 1e-11 absolute on the FP64 path.  The oracle runs start in
the background when these tests are selected (tests/long_oracle.py)."""
import numpy as np
import pytest

import long_oracle as LO
import paper_2105_08772_gb300 as P

pytestmark = pytest.mark.gpu


def _droplet(name, prec, code=None):
    L, R, steps = LO.JOBS[name]
    c = LO.centre(L)
    lat = P.Lattice(L, L, L, G=-5.0, prec=prec)
    try:
        if code is not None:
            lat.set_tile(code)
        lat.init_drop((c, c, c), R, LO.N_L, LO.N_G, 1.0)
        lat.step(steps)
        return lat.rho(), lat.get_tile()
    finally:
        lat.close()


@pytest.mark.long_oracle("droplet64")
def test_f32_64_box_several_z_chunks_1000_steps():
    ref = LO.result("droplet64")
    rhos = []
    # kind 5, 32 x 8 tiles, depth 1: the launcher's z chunk, then chunks of 8 and 21 planes
    for code in (None, 532080081, 532080211):
        rho, tile = _droplet("droplet64", "f32", code)
        assert tile // 100000000 == 5, tile
        rel = float(np.max(np.abs(rho - ref) / ref))
        print(f"f32 64^3 tile {tile}: max relative density error after 1000 steps {rel:.3e}")
        assert rel < 1e-4, (tile, rel)
        rhos.append(rho)
    assert all(np.array_equal(rhos[0], r) for r in rhos[1:])   # the z chunk changes no bit


@pytest.mark.long_oracle("droplet64")
def test_f64_64_box_1000_steps():
    ref = LO.result("droplet64")
    rho, _ = _droplet("droplet64", "f64")
    assert float(np.max(np.abs(rho - ref))) < 1e-11


@pytest.mark.long_oracle("droplet41")
def test_f32_odd_41_box_element_copies_1000_steps():
    ref = LO.result("droplet41")
    rho, tile = _droplet("droplet41", "f32")
    assert tile // 100000000 == 6, tile
    rel = float(np.max(np.abs(rho - ref) / ref))
    print(f"f32 41^3 tile {tile}: max relative density error after 1000 steps {rel:.3e}")
    assert rel < 1e-4, rel
