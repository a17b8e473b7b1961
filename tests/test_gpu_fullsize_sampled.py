"""Parity at the full sizes of the measured configurations, in the kernel
configuration the library starts from for them (the one the benchmark times):
one step from a seeded state far from equilibrium, and the post-step
populations at sampled nodes (corners, tile and wrap edges, random nodes)
against the oracle's step evaluated node by node on a periodic window
(tests/sampled.py).  The whole-field comparison at 128^3 is in test_gpu_parity.

Sizes: 192^3 (precision study, FP64 and shifted FP32), 256^3 (the roofline
box, shifted FP32), 256^3 with the Carnahan-Starling psi at 0.8 T_c and the E6
stencil (equation-of-state study), and 213^3 (an odd box of the paper's sweep,
element-copy kernel).

Bounds: FP64 1e-14 absolute per population (populations <= 1); shifted FP32
2e-6 of the node's density (FP32 arithmetic on the stored values, the
oracle's input being the device's own rounded populations).
"""
import numpy as np
import pytest

import inputs
import paper_2105_08772_gb300 as P
import sampled
from oracle import eos as E
from oracle import lbm3d

pytestmark = pytest.mark.gpu

T_C = 0.0943287031337238      # Carnahan-Starling (a = 1, b = 4, R = 1) critical temperature


@pytest.mark.parametrize("L,prec,stencil,kind,G,T", [
    (192, "f64", "E4", "one_minus_exp", -5.0, 0.0),
    (192, "f32", "E4", "one_minus_exp", -5.0, 0.0),
    (256, "f32", "E4", "one_minus_exp", -5.0, 0.0),
    (256, "f32", "E6", "cs", -1.0, 0.8 * T_C),
    (213, "f32", "E4", "one_minus_exp", -5.0, 0.0),
])
def test_full_size_one_step_at_sampled_nodes(L, prec, stencil, kind, G, T):
    shape = (L, L, L)
    if kind == "cs":
        f0 = inputs.random_populations(shape, seed=31, inner=0.3, outer=0.02, radius=L / 5.3)
    else:
        f0 = inputs.random_populations(shape, seed=31, inner=1.89, outer=0.15, radius=L / 4.0)
    lat = P.Lattice(L, L, L, tau=1.0, G=G, psi=kind, stencil=stencil, prec=prec, cs_T=T)
    try:
        assert lat.get_tile() == P.default_tile(L, L, L, stencil=stencil, prec=prec, tau=1.0)
        lat.set_populations(f0)
        del f0
        f_in = lat.get_populations()          # the device's (rounded) state
        lat.step(1)
        f_out = lat.get_populations()
    finally:
        lat.close()
    m = lbm3d.Model(tau=1.0, G=G, eos=E.EOS(kind, T=T), stencil=stencil)
    worst = 0.0
    for c in sampled.sample_nodes(shape, 160, seed=L):
        ref = sampled.step_at(f_in, m, c)
        got = f_out[(slice(None),) + c]
        err = np.max(np.abs(got - ref))
        worst = max(worst, err if prec == "f64" else err / ref.sum())
    assert worst < (1e-14 if prec == "f64" else 2e-6), worst
