"""Failure detection without a GPU fault: fields that the step cannot carry are
reported as LBM_ENUMERIC (status bit 3) at the next convergence check, and the
context stays usable.  The inputs are finite (set_populations rejects anything
else); the library has no data-dependent addressing, so non-finite values are
harmless to the device."""
import numpy as np
import pytest

import inputs
import paper_2105_08772_gb300 as P
from oracle import lattice as Lt

pytestmark = pytest.mark.gpu

SHAPE = (12, 16, 20)     # z, y, x


def _lattice(prec):
    nz, ny, nx = SHAPE
    return P.Lattice(nx, ny, nz, tau=1.0, G=-5.0, stencil="E4", prec=prec)


def _expect_enumeric(lat):
    with pytest.raises(P.LBMError) as e:
        lat.run_to_convergence(max_steps=1024, check_every=64)
    assert e.value.status == P.LBM_ENUMERIC
    assert lat.observables().status_bits & 8


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_non_positive_density_is_reported(prec):
    """A uniform field of density -1 is a fixed point of the step (no force, no
    flow), so the check finds a non-positive density whatever the step does."""
    w = Lt.d3q19_weights()
    lat = _lattice(prec)
    lat.set_populations(-w[:, None, None, None] * np.ones(SHAPE))
    _expect_enumeric(lat)
    # the context stays usable: a valid field runs normally afterwards
    lat.set_populations(inputs.random_populations(SHAPE, seed=42))
    lat.step(16)
    assert np.all(np.isfinite(lat.rho())) and np.all(lat.rho() > 0)
    lat.close()


def test_overflowing_population_is_reported():
    """FP64 populations of 1e308 at one node: their sum overflows, the node's
    velocity is NaN and the field turns non-finite."""
    f = inputs.random_populations(SHAPE, seed=43)
    f[:, 6, 8, 10] = 1e308
    lat = _lattice("f64")
    lat.set_populations(f)
    _expect_enumeric(lat)
    lat.close()
