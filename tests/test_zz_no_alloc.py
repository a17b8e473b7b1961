"""The no-allocation entry point against lbm_observables.

lbm_density_moments_noalloc serves callers that cannot allocate device memory:
its scratch is a fixed array inside the library.  It must give the mass and
centre of mass that lbm_observables reports for the same field, on repeated
calls that reuse the same scratch.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import paper_2105_08772_gb300 as P

pytestmark = pytest.mark.gpu


def test_noalloc_moments_match_observables_on_two_calls():
    import torch
    nx, ny, nz = 48, 40, 36
    lat = P.Lattice(nx, ny, nz, G=-5.0, prec="f64")
    lat.init_drop((nx // 2, ny // 2, nz // 2), 9.0, 1.89, 0.12)
    lat.step(200)
    ob = lat.observables()
    rho = torch.from_numpy(lat.rho()).to("cuda").contiguous()
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    results = []
    for _ in range(2):
        out.fill_(np.nan)
        P.lbm_density_moments_noalloc(rho.data_ptr(), nx, ny, nz, ob.n_out, out.data_ptr(), stream)
        torch.cuda.synchronize()
        mass, cx, cy, cz = out.cpu().numpy()
        assert abs(mass - ob.mass) <= 1e-12 * ob.mass
        assert np.allclose([cx, cy, cz], list(ob.com), rtol=0, atol=1e-9)
        results.append((mass, cx, cy, cz))
    assert results[0] == results[1]


def test_noalloc_rejects_fields_beyond_its_scratch():
    with pytest.raises(P.LBMError, match="33554432"):
        P.lbm_density_moments_noalloc(256, 512, 256, 257, 0.1, 256, 0)
    with pytest.raises(P.LBMError):
        P.lbm_density_moments_noalloc(0, 8, 8, 8, 0.1, 256, 0)
