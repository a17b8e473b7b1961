"""The windowed one-node oracle step used by the full-size sampled GPU tests
equals the whole-field oracle step at every sampled node, up to the rounding
order of numpy's reductions (which depends on the array's shape): 1e-15."""
import numpy as np
import pytest

import inputs
import sampled
from oracle import eos as E
from oracle import lbm3d


@pytest.mark.parametrize("stencil,kind,G,T,inner,outer", [
    ("E4", "one_minus_exp", -5.0, 0.0, 1.89, 0.15),
    ("E6", "cs", -1.0, 0.0755, 0.3, 0.02),
    ("E8", "exp_inv", -9.2, 0.0, 2.3, 0.45),
])
def test_windowed_step_equals_whole_field_step(stencil, kind, G, T, inner, outer):
    shape = (13, 17, 22)
    f = inputs.random_populations(shape, seed=21, inner=inner, outer=outer)
    m = lbm3d.Model(tau=1.0, G=G, eos=E.EOS(kind, T=T), stencil=stencil)
    full = lbm3d.step(f, m)
    for c in sampled.sample_nodes(shape, 40, seed=3):
        assert np.max(np.abs(sampled.step_at(f, m, c) - full[(slice(None),) + c])) < 1e-15, c


def test_sample_nodes_are_in_range_and_include_corners():
    shape = (9, 10, 40)
    nodes = sampled.sample_nodes(shape, 30, seed=1)
    assert len(nodes) == 30 and (0, 0, 0) in nodes and (8, 9, 39) in nodes
    assert all(0 <= z < 9 and 0 <= y < 10 and 0 <= x < 40 for z, y, x in nodes)
