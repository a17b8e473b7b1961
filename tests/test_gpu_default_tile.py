"""A lattice starts from the kernel configuration that lbm_default_tile reports
for its arguments (the host-side query and lbm_create share the policy)."""
import pytest

import paper_2105_08772_gb300 as P

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("box,stencil,prec,tau", [
    ((128, 128, 128), "E4", "f32", 1.0),
    ((156, 156, 156), "E4", "f32", 1.0),
    ((127, 127, 127), "E4", "f32", 1.0),
    ((40, 40, 40), "E4", "f64", 1.0),
    ((16, 16, 16), "E4", "f64", 0.8),
    ((48, 48, 48), "E4", "f16", 1.0),
    ((36, 36, 36), "E6", "f32", 1.0),
    ((41, 43, 47), "E8", "f32", 1.3),
])
def test_lattice_starts_from_the_default_tile(box, stencil, prec, tau):
    lat = P.Lattice(*box, tau=tau, G=-5.0, stencil=stencil, prec=prec)
    try:
        assert lat.get_tile() == P.default_tile(*box, stencil=stencil, prec=prec, tau=tau)
    finally:
        lat.close()
