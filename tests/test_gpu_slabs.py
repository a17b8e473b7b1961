"""z-slabs of one lattice held in one process on one GPU: each slab is a lattice
of its owned planes plus R + 1 ghost planes a side, stepped by the library's
kernels one slab after another on one stream (no kernel waits on another), the
ghost planes refreshed by lbm_halo_copy after every step.  The owned planes
must equal the whole lattice's run bit for bit (Sec. II: the update of Eq. (3)
is local), in every storage precision, when all slabs store with the whole
lattice's shift and scale."""
import numpy as np
import pytest

import paper_2105_08772_gb300 as P
from paper_2105_08772_gb300 import lbm as L
from paper_2105_08772_gb300 import slabs as SL
from tests.inputs import random_populations

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,world,stencil,prec", [
    ((40, 24, 32), 2, "E4", "f64"),
    ((40, 24, 37), 3, "E4", "f32"),     # ragged slabs, row-chunk kernel
    ((41, 20, 30), 2, "E4", "f32"),     # odd nx: element-copy kernel
    ((40, 16, 24), 2, "E8", "f32"),     # R = 2: three ghost planes a side
    ((48, 16, 32), 2, "E4", "f16"),
])
def test_slabs_step_like_the_whole_lattice(shape, world, stencil, prec):
    nx, ny, nz = shape
    f = random_populations((nz, ny, nx), seed=5, inner=1.8, outer=0.2)
    whole = P.Lattice(nx, ny, nz, G=-5.0, stencil=stencil, prec=prec)
    sl = SL.SlabLattice(nx, ny, nz, world, G=-5.0, stencil=stencil, prec=prec)
    try:
        whole.set_populations(f)
        n0, scale = L.lbm_storage_params(whole.ctx)
        sl.set_populations(f, n0, scale)
        whole.step(7)
        sl.step(7)
        a, b = whole.get_populations(), sl.populations()
        assert np.array_equal(a, b), float(np.max(np.abs(a - b)))
    finally:
        sl.close()
        whole.close()


def test_halo_copy_rejects_mismatched_slabs():
    a = P.Lattice(32, 16, 12, G=-5.0, prec="f32")
    b = P.Lattice(32, 8, 12, G=-5.0, prec="f32")
    try:
        a.init_drop((16, 8, 6), 4.0, 1.8, 0.2)
        b.init_drop((16, 4, 6), 3.0, 1.8, 0.2)
        with pytest.raises(P.LBMError):
            L.lbm_halo_copy(a.ctx, 0, b.ctx, 1, 1)      # plane sizes differ
        with pytest.raises(P.LBMError):
            L.lbm_halo_copy(a.ctx, 12, a.ctx, 1, 1)     # plane out of range
        with pytest.raises(P.LBMError):
            L.lbm_halo_copy(a.ctx, 0, a.ctx, 1, 1 << 19)  # no population 19
        ptr, nb = L.lbm_state_plane(a.ctx, 3, 5)
        assert nb == 32 * 16 * 4 and ptr != 0
    finally:
        a.close()
        b.close()
