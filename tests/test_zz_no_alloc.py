"""The no-allocation entry point against lbm_observables and a numpy restatement.

lbm_density_moments_noalloc serves callers that cannot allocate device memory:
its scratch is a fixed array inside the library.  It must give the mass and
centre of mass that lbm_observables reports for the same field, on repeated
calls that reuse the same scratch, and must not allocate.  This file is
collected last on purpose.
"""
import re
from pathlib import Path

import numpy as np
import pytest

import paper_2105_08772_gb300 as P

ROOT = Path(__file__).resolve().parent.parent
SOURCE = ROOT / "paper_2105_08772_gb300" / "csrc" / "lbm_noalloc.cu"
MAX_NODES = 33554432


def _code_without_comments(text: str) -> str:
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return re.sub(r'"(\\.|[^"\\])*"', '""', text)


def test_noalloc_source_calls_no_allocator():
    """The translation unit of the entry point names no device (or pinned) allocator."""
    code = _code_without_comments(SOURCE.read_text())
    banned = ("cudaMalloc", "cudaMallocAsync", "cudaMallocManaged", "cudaMallocHost", "cudaHostAlloc",
              "cudaFree", "cudaFreeAsync", "cuMemAlloc", "cuMemCreate", "malloc(", "new ")
    for name in banned:
        assert name not in code, name


def test_noalloc_accepts_the_largest_field_and_rejects_one_more_plane():
    """256 x 512 x 256 = 33554432 nodes (the whole scratch) passes the size check: with null
    pointers it fails on the pointers, before any launch; one more plane fails on the size."""
    with pytest.raises(P.LBMError, match="null device pointer"):
        P.lbm_density_moments_noalloc(0, 256, 512, 256, 0.1, 0, 0)
    assert 256 * 512 * 256 == MAX_NODES
    with pytest.raises(P.LBMError, match="33554432"):
        P.lbm_density_moments_noalloc(256, 256, 512, 257, 0.1, 256, 0)
    with pytest.raises(P.LBMError, match=">= 1"):
        P.lbm_density_moments_noalloc(256, 0, 8, 8, 0.1, 256, 0)


def _moments_numpy(rho: np.ndarray, n_ref: float):
    """Mass and minimum-image centre of mass of rho - n_ref about the centre node
    (n//2 per axis); an even side's plane at exactly n/2 counts as displacement 0."""
    nz, ny, nx = rho.shape
    w = rho - n_ref

    def disp(n):
        d = np.arange(n) - n // 2
        d[2 * d == -n] = 0
        return d.astype(np.float64)

    W = w.sum()
    cx = nx // 2 + (w.sum(axis=(0, 1)) * disp(nx)).sum() / W
    cy = ny // 2 + (w.sum(axis=(0, 2)) * disp(ny)).sum() / W
    cz = nz // 2 + (w.sum(axis=(1, 2)) * disp(nz)).sum() / W
    return rho.sum(), cx, cy, cz


def _call(rho_dev, shape, n_ref, out):
    import torch
    nz, ny, nx = shape
    out.fill_(-1.0)
    P.lbm_density_moments_noalloc(rho_dev.data_ptr(), nx, ny, nz, n_ref, out.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().copy()


@pytest.mark.gpu
def test_noalloc_moments_match_observables_on_two_calls():
    import torch
    nx, ny, nz = 48, 40, 36
    lat = P.Lattice(nx, ny, nz, G=-5.0, prec="f64")
    lat.init_drop((nx // 2, ny // 2, nz // 2), 9.0, 1.89, 0.12)
    lat.step(200)
    ob = lat.observables()
    rho = torch.from_numpy(lat.rho()).to("cuda").contiguous()
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    results = []
    for _ in range(2):
        mass, cx, cy, cz = _call(rho, (nz, ny, nx), ob.n_out, out)
        assert abs(mass - ob.mass) <= 1e-12 * ob.mass
        assert np.allclose([cx, cy, cz], list(ob.com), rtol=0, atol=1e-9)
        results.append((mass, cx, cy, cz))
    assert results[0] == results[1]
    lat.close()


@pytest.mark.gpu
def test_noalloc_odd_box_with_a_drop_across_the_periodic_wrap():
    """An odd 37 x 41 x 33 box with the drop's excess crossing the x and z wraps, and an
    even 36 x 40 x 32 box whose half planes count 0, against the numpy restatement."""
    import torch
    rng = np.random.default_rng(7)
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    for shape, c in (((33, 41, 37), (31.5, 19.0, 35.0)), ((32, 40, 36), (2.0, 21.0, 33.5))):
        nz, ny, nx = shape
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        d2 = np.zeros(shape)
        for g, cc, n in ((x, c[2], nx), (y, c[1], ny), (z, c[0], nz)):
            dd = np.abs(g - cc)
            d2 += np.minimum(dd, n - dd) ** 2
        rho = 0.12 + 1.7 * np.exp(-d2 / 18.0) + 1e-3 * rng.random(shape)
        want = _moments_numpy(rho, 0.12)
        dev = torch.from_numpy(rho).to("cuda").contiguous()
        for _ in range(2):
            got = _call(dev, shape, 0.12, out)
            assert abs(got[0] - want[0]) <= 1e-12 * want[0]
            assert np.allclose(got[1:], want[1:], rtol=0, atol=1e-9), (got, want)


@pytest.mark.gpu
def test_noalloc_uniform_field_has_mass_but_no_centre():
    """No excess over n_ref: the mass is written and the centre of mass is NaN."""
    import torch
    shape = (9, 10, 11)
    dev = torch.full(shape, 0.25, dtype=torch.float64, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    got = _call(dev, shape, 0.25, out)
    assert abs(got[0] - 0.25 * 990) <= 1e-12 * 0.25 * 990
    assert np.all(np.isnan(got[1:]))


@pytest.mark.gpu
def test_noalloc_calls_leave_device_memory_unchanged():
    """After the first call (which may load the library's device module, and with it the
    fixed scratch), further calls take no device memory: the driver's free count holds."""
    import torch
    shape = (64, 64, 64)
    dev = torch.full(shape, 0.3, dtype=torch.float64, device="cuda")
    dev[20:40, 20:40, 20:40] = 1.5
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    first = _call(dev, shape, 0.3, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        got = _call(dev, shape, 0.3, out)
        assert np.array_equal(got, first)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
