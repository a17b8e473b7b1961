"""Groups of lattices (lbm_group_*): several existing lattices stepped by one launch
per time step evolve bitwise as they do under lbm_step, through graph replays, odd
step counts and lattices stepped on their own in between."""
import numpy as np
import pytest

import paper_2105_08772_gb300 as P

pytestmark = pytest.mark.gpu


def _make(box, tau=1.0, G=-5.0, prec="f32", R=6.0, bubble=False):
    lat = P.Lattice(*box, tau=tau, G=G, prec=prec)
    c = (box[0] // 2, box[1] // 2, box[2] // 2)
    lat.init_drop(c, R, 0.12 if bubble else 1.89, 1.89 if bubble else 0.12)
    return lat


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("boxes,taus", [
    ([(48, 40, 36), (64, 32, 20)], [1.0, 1.0]),            # moment kernel
    ([(48, 40, 36), (37, 29, 23), (40, 24, 16)], [1.0, 1.0, 1.0]),   # odd box: pipelined kernel
    ([(48, 40, 36), (40, 32, 28)], [1.0, 0.8]),            # mixed tau
])
def test_group_equals_separate_steps(prec, boxes, taus):
    grouped = [_make(b, tau=t, prec=prec, bubble=(k % 2 == 1)) for k, (b, t) in enumerate(zip(boxes, taus))]
    alone = [_make(b, tau=t, prec=prec, bubble=(k % 2 == 1)) for k, (b, t) in enumerate(zip(boxes, taus))]
    g = P.Group(grouped)
    plan = [131, 128, 5]                 # graph replay + odd remainder, then more
    for n in plan:
        g.step(n)
        for lat in alone:
            lat.step(n)
    grouped[0].step(3)                   # one lattice on its own: parities now differ
    alone[0].step(3)
    g.step(130)
    for lat in alone:
        lat.step(130)
    for a, b in zip(grouped, alone):
        assert a.observables().steps == b.observables().steps
        assert np.array_equal(a.get_populations(), b.get_populations())
    g.close()


def test_group_rejects_mixed_storage():
    a = _make((40, 24, 16), prec="f32")
    b = _make((40, 24, 16), prec="f64")
    with pytest.raises(P.LBMError):
        P.Group([a, b])
    with pytest.raises(P.LBMError):
        P.Group([a, a])
