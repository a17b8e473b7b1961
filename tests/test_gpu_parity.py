"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: density max-abs 1e-11 on the FP64 path and 1e-4 relative on the
FP32-shifted path after 1000 steps.  FP16-shifted storage is bounded by twice the
error of the same storage in an FP64 model of the oracle (f16_storage_model).
"""
import numpy as np
import pytest

import inputs
import paper_2105_08772_gb300 as P
from oracle import eos as E
from oracle import lbm3d
from oracle import observables as O

pytestmark = pytest.mark.gpu

G = -5.0


def oracle_model(G=G, kind="one_minus_exp", stencil="E4", tau=1.0, T=0.0):
    return lbm3d.Model(tau=tau, G=G, eos=E.EOS(kind, T=T), stencil=stencil)


def lattice(shape_zyx, prec="f64", stencil="E4", kind="one_minus_exp", G=G, tau=1.0, T=0.0):
    nz, ny, nx = shape_zyx
    return P.Lattice(nx, ny, nz, tau=tau, G=G, psi=kind, stencil=stencil, prec=prec, cs_T=T)


SHAPE = (12, 20, 40)          # z, y, x: 2 x-tiles (one ragged), ragged y tiles, one z chunk
RAGGED = (23, 29, 37)


@pytest.fixture(scope="module")
def random_state():
    f0 = inputs.random_populations(SHAPE, seed=11)
    ref = lbm3d.run(f0, oracle_model(), 1000)
    return f0, ref


def test_population_roundtrip_is_exact():
    f0 = inputs.random_populations((7, 9, 11), seed=1)
    lat = lattice((7, 9, 11))
    lat.set_populations(f0)
    assert np.array_equal(lat.get_populations(), f0)


def test_single_step_matches_oracle_f64():
    f0 = inputs.random_populations(RAGGED, seed=2)
    lat = lattice(RAGGED)
    lat.set_populations(f0)
    lat.step(1)
    ref = lbm3d.step(f0, oracle_model())
    assert np.max(np.abs(lat.get_populations() - ref)) < 1e-14


def test_parity_f64_1000_steps(random_state):
    f0, ref = random_state
    lat = lattice(SHAPE)
    lat.set_populations(f0)
    lat.step(1000)
    rho, rho_ref = lat.rho(), lbm3d.density(ref)
    assert np.max(np.abs(rho - rho_ref)) < 1e-11
    assert np.max(np.abs(lat.get_populations() - ref)) < 1e-11


@pytest.fixture(scope="module")
def droplet_state():
    """The paper's workload: a tanh droplet at the flat-interface densities (Eq. (23))."""
    shape, c = (16, 24, 32), (16, 12, 8)
    n = lbm3d.drop_density(shape, c, 6.0, 1.8883, 0.1193)
    f0 = lbm3d.init_from_density(n)
    return shape, c, f0, lbm3d.run(f0, oracle_model(), 1000)


def test_parity_f32_shifted_1000_steps_droplet(droplet_state):
    shape, c, f0, ref = droplet_state
    lat = lattice(shape, prec="f32")
    lat.init_drop(c, 6.0, 1.8883, 0.1193, 1.0)
    lat.step(1000)
    rho_ref = lbm3d.density(ref)
    rel = np.max(np.abs(lat.rho() - rho_ref) / rho_ref)
    print(f"f32 shifted droplet: max relative density error after 1000 steps {rel:.3e}")
    assert rel < 1e-4, rel


def test_parity_f32_shifted_1000_steps_random_state(random_state):
    """A noisy far-from-equilibrium state: FP32 rounding is amplified while it separates."""
    f0, ref = random_state
    lat = lattice(SHAPE, prec="f32")
    lat.set_populations(f0)
    lat.step(1000)
    rho_ref = lbm3d.density(ref)
    rel = np.max(np.abs(lat.rho() - rho_ref) / rho_ref)
    print(f"f32 shifted random state: max relative density error after 1000 steps {rel:.3e}")
    assert rel < 1e-4, rel


def f16_storage_model(f0, steps, m):
    """The oracle's step with FP16 storage emulated: after every step each population is
    stored as (f_i - w_i n0) 2^k rounded to half precision (n0 the field's mean density,
    2^k putting the largest deviation near 2^13, as the library chooses), in FP64
    arithmetic otherwise.  The error of this model against the exact oracle is the
    error FP16 storage itself makes."""
    w = lbm3d.W[:, None, None, None]
    n0 = float(lbm3d.density(f0).mean())
    k = int(np.floor(np.log2(8192.0 / np.max(np.abs(f0 - w * n0)))))
    q = lambda f: ((f - w * n0) * 2.0 ** k).astype(np.float16).astype(np.float64) / 2.0 ** k + w * n0  # noqa: E731
    f = q(f0)
    for _ in range(steps):
        f = q(lbm3d.step(f, m))
    return f


@pytest.fixture(scope="module")
def f16_model_error(droplet_state):
    shape, c, f0, ref = droplet_state
    rho_ref = lbm3d.density(ref)
    emu = lbm3d.density(f16_storage_model(f0, 1000, oracle_model()))
    return float(np.max(np.abs(emu - rho_ref) / rho_ref))


def test_parity_f16_shifted_1000_steps_droplet(droplet_state, f16_model_error):
    """FP16 storage against the FP64 oracle after 1000 steps, bounded by the error of the
    same storage in an FP64 model (f16_storage_model): the kernels differ from that
    model only by FP32 instead of FP64 arithmetic, 2^-24 against FP16's 2^-11 per
    rounding, which can flip single roundings but not change the error's size.
    Bound: twice the model's error."""
    shape, c, f0, ref = droplet_state
    lat = lattice(shape, prec="f16")
    lat.init_drop(c, 6.0, 1.8883, 0.1193, 1.0)
    lat.step(1000)
    rho_ref = lbm3d.density(ref)
    rel = np.max(np.abs(lat.rho() - rho_ref) / rho_ref)
    print(f"f16 shifted droplet: max relative density error after 1000 steps {rel:.3e} "
          f"(FP16 storage model {f16_model_error:.3e})")
    assert np.isfinite(rel) and rel < 2.0 * f16_model_error


def test_droplet_init_matches_oracle():
    shape = (16, 24, 32)
    lat = lattice(shape)
    c = (16, 12, 8)
    lat.init_drop(c, 6.0, 1.89, 0.12, 1.0)
    f = lbm3d.init_from_density(lbm3d.drop_density(shape, c, 6.0, 1.89, 0.12))
    assert np.max(np.abs(lat.get_populations() - f)) < 1e-14
    lat.step(300)
    ref = lbm3d.run(f, oracle_model(), 300)
    assert np.max(np.abs(lat.rho() - lbm3d.density(ref))) < 1e-11


def test_init_rho_matches_init_from_density():
    shape = (10, 12, 14)
    n = inputs.random_density(shape, seed=3)
    lat = lattice(shape)
    lat.init_rho(n)
    assert np.max(np.abs(lat.get_populations() - lbm3d.init_from_density(n))) < 1e-15


@pytest.mark.parametrize("stencil", ["E6", "E8"])
def test_parity_wide_stencils_f64(stencil):
    shape = (10, 14, 20)
    f0 = inputs.random_populations(shape, seed=4)
    lat = lattice(shape, stencil=stencil)
    lat.set_populations(f0)
    lat.step(200)
    ref = lbm3d.run(f0, oracle_model(stencil=stencil), 200)
    assert np.max(np.abs(lat.get_populations() - ref)) < 1e-11


@pytest.mark.parametrize("kind,Gk,T", [("exp_inv", -9.2, 0.0), ("cs", -1.0, 0.085)])
def test_parity_other_pseudopotentials_f64(kind, Gk, T):
    shape = (10, 12, 18)
    if kind == "cs":
        f0 = inputs.random_populations(shape, seed=5, inner=0.3, outer=0.05)
    else:
        f0 = inputs.random_populations(shape, seed=5, inner=2.3, outer=0.45)
    lat = lattice(shape, kind=kind, G=Gk, T=T)
    lat.set_populations(f0)
    lat.step(200)
    ref = lbm3d.run(f0, oracle_model(G=Gk, kind=kind, T=T), 200)
    assert np.max(np.abs(lat.get_populations() - ref)) < 1e-11


@pytest.mark.parametrize("shape,stencil", [((3, 3, 3), "E4"), ((5, 5, 5), "E6"), ((4, 3, 7), "E4"),
                                           ((5, 6, 5), "E8")])
def test_minimum_boxes(shape, stencil):
    f0 = inputs.random_populations(shape, seed=6)
    lat = lattice(shape, stencil=stencil)
    lat.set_populations(f0)
    lat.step(50)
    ref = lbm3d.run(f0, oracle_model(stencil=stencil), 50)
    assert np.max(np.abs(lat.get_populations() - ref)) < 1e-12


def test_tau_other_than_one():
    f0 = inputs.random_populations((8, 10, 12), seed=7)
    lat = lattice((8, 10, 12), tau=0.7)
    lat.set_populations(f0)
    lat.step(100)
    ref = lbm3d.run(f0, oracle_model(tau=0.7), 100)
    assert np.max(np.abs(lat.get_populations() - ref)) < 1e-11


def test_graph_replay_equals_eager_steps():
    f0 = inputs.random_populations((12, 16, 20), seed=8)
    a = lattice((12, 16, 20))
    a.set_populations(f0)
    a.step(300)                 # graph replays + eager remainder
    b = lattice((12, 16, 20))
    b.set_populations(f0)
    for _ in range(300):
        b.step(1)
    assert np.array_equal(a.get_populations(), b.get_populations())


def test_every_tile_shape_gives_identical_results():
    """The per-node arithmetic does not depend on the tiling: bitwise-equal fields."""
    f0 = inputs.random_populations(RAGGED, seed=9)
    lat = lattice(RAGGED)
    lat.set_populations(f0)
    choice = lat.autotune(reps=2)
    assert choice > 0
    steps_done = lat.observables().steps
    ref = lbm3d.run(f0, oracle_model(), steps_done)
    assert np.max(np.abs(lat.get_populations() - ref)) < 1e-12


def test_observables_match_oracle():
    shape = (24, 26, 28)
    f0 = inputs.random_populations(shape, seed=10, inner=1.85, outer=0.13, noise=0.0)
    lat = lattice(shape)
    lat.set_populations(f0)
    lat.step(200)
    ob = lat.observables()
    fr = lbm3d.run(f0, oracle_model(), 200)
    ref = O.observe(fr, oracle_model(), contrast0=None)
    for k in ("n_in", "n_out", "P_in", "P_out", "dP", "mass", "R_e", "C", "D", "max_u"):
        a, b = getattr(ob, k), getattr(ref, k)
        assert abs(a - b) <= 1e-10 * max(1.0, abs(b)), (k, a, b)
    assert np.allclose(list(ob.com), ref.com, atol=1e-9)
    if np.isfinite(ref.R_s):
        assert abs(ob.R_s - ref.R_s) < 1e-9 * ref.R_s
    else:
        assert np.isnan(ob.R_s) and (ob.status_bits & 1)
    assert np.max(np.abs(lat.pt_profile() - ref.PT_line)) < 1e-12
    assert np.max(np.abs(lat.rho_profile() - ref.n_line)) < 1e-12
    u = lat.velocity()
    assert np.max(np.abs(u - O.velocity(fr, oracle_model()))) < 1e-12


def test_delta_u_matches_oracle():
    shape = (10, 12, 14)
    f0 = inputs.random_populations(shape, seed=12)
    lat = lattice(shape)
    lat.set_populations(f0)
    lat.observables()                 # snapshot u(t)
    lat.step(40)
    ob = lat.observables()
    m = oracle_model()
    u0 = O.velocity(f0, m)
    u1 = O.velocity(lbm3d.run(f0, m, 40), m)
    assert abs(ob.du - O.delta_u(u1, u0)) < 1e-12


def test_sigma_of_R_uses_the_measured_integrals():
    shape = (24, 26, 28)
    f0 = inputs.random_populations(shape, seed=10, inner=1.85, outer=0.13, noise=0.0)
    lat = lattice(shape)
    lat.set_populations(f0)
    ob = lat.observables()
    R = np.array([2.0, 5.0, 9.5])
    s, ds = lat.sigma_of_R(R)
    s_ref, ds_ref = O.sigma_of_R(R, ob.dP, ob.C, ob.D)
    assert np.allclose(s, s_ref, rtol=1e-14) and np.allclose(ds, ds_ref, rtol=1e-14)


def test_save_load_resumes_bitwise(tmp_path):
    f0 = inputs.random_populations((8, 9, 10), seed=13)
    a = lattice((8, 9, 10), prec="f32")
    a.set_populations(f0)
    a.step(50)
    a.save(tmp_path / "ck.bin")
    a.step(77)
    b = lattice((8, 9, 10), prec="f32")
    b.load(tmp_path / "ck.bin")
    b.step(77)
    assert np.array_equal(a.get_populations(), b.get_populations())
    assert b.observables().steps == 127


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_full_size_steps_in_bench_configuration(prec):
    """128^3 (the benchmark box) in the benchmark's tiling: two steps (both buffer parities)
    against the oracle on the whole field."""
    shape = (128, 128, 128)
    f0 = inputs.random_populations(shape, seed=14, inner=1.89, outer=0.15, radius=32.0)
    lat = lattice(shape, prec=prec)
    lat.set_populations(f0)
    m = oracle_model()
    ref = f0
    for k in range(2):
        lat.step(1)
        ref = lbm3d.step(ref, m)
        rho_ref = lbm3d.density(ref)
        err = np.max(np.abs(lat.rho() - rho_ref) / rho_ref)
        assert err < (1e-14 if prec == "f64" else 2e-6), (k, err)


@pytest.mark.parametrize("prec,code", [(p, c) for p in ("f64", "f32")
                                       for c in (432080001, 432040001, 464040001, 432080081)]
                         + [("f32", 432080002), ("f32", 432040002)])
def test_chunked_kernel_matches_pipelined_kernel_and_oracle(prec, code):
    """The chunked kernel (kind 4: 16-byte row chunks) stages the same values as the
    pipelined kernel: bitwise-equal fields, and the oracle's.  nx = 72 with 32-wide
    tiles has a ragged last column whose staged rows wrap at the right end; ny and
    nz are ragged too."""
    shape = (13, 22, 72)
    f0 = inputs.random_populations(shape, seed=25)
    a = lattice(shape, prec=prec)
    a.set_populations(f0)
    a.set_tile(code)
    a.step(130)
    b = lattice(shape, prec=prec)
    b.set_populations(f0)
    b.set_tile(132080001)
    b.step(130)
    assert np.array_equal(a.get_populations(), b.get_populations())
    if prec == "f64":
        ref = lbm3d.run(f0, oracle_model(), 130)
        assert np.max(np.abs(a.get_populations() - ref)) < 1e-12


def test_chunked_kernel_wide_stencil_and_tau():
    shape = (9, 10, 40)
    f0 = inputs.random_populations(shape, seed=26)
    a = lattice(shape, stencil="E6", tau=0.8)
    a.set_populations(f0)
    a.set_tile(432040001)
    a.step(40)
    ref = lbm3d.run(f0, oracle_model(stencil="E6", tau=0.8), 40)
    assert np.max(np.abs(a.get_populations() - ref)) < 1e-12


@pytest.mark.parametrize("prec,code,tau", [(p, c, 1.0) for p in ("f64", "f32")
                                           for c in (532080001, 532040001, 564040001, 532080081)]
                         + [("f32", 532080002, 1.0), ("f32", 532040002, 1.0),
                            ("f64", 532080001, 0.8), ("f32", 532040002, 0.8)])
def test_moment_kernel_matches_pipelined_kernel_and_oracle(prec, code, tau):
    """The unit-tau moment kernel (kind 5) keeps only n and j of a node between its
    density pass and its collision; for tau = 1 that is all the collision uses, so
    fields are bitwise equal to the pipelined kernel's, and to the oracle's.  For
    tau != 1 the same tile code runs the chunked kernel.  Ragged x, y and z."""
    shape = (13, 22, 72)
    f0 = inputs.random_populations(shape, seed=27)
    a = lattice(shape, prec=prec, tau=tau)
    a.set_populations(f0)
    a.set_tile(code)
    a.step(130)
    b = lattice(shape, prec=prec, tau=tau)
    b.set_populations(f0)
    b.set_tile(132080001)
    b.step(130)
    assert np.array_equal(a.get_populations(), b.get_populations())
    if prec == "f64":
        ref = lbm3d.run(f0, oracle_model(tau=tau), 130)
        assert np.max(np.abs(a.get_populations() - ref)) < 1e-12


@pytest.mark.parametrize("shape", [(13, 16, 64), (9, 24, 72), (5, 32, 68), (7, 40, 128), (3, 16, 96)])
def test_tma_kernel_matches_moment_kernel_and_oracle(shape):
    """The moment kernel fed by TMA tensor-tile copies (kind 7) stages the same values as
    the row-chunk kernel (kind 5): bitwise-equal fields after 130 steps, both buffer
    parities.  The boxes cover every periodic case the tensor boxes and the fix-ups
    handle: tiles wrapping in x on the left and on the right, in y at the top and the
    bottom, the four corners, a ragged last column (nx = 72, and nx = 68 with a 4-wide
    column), the minimum z (nz = 3)."""
    f0 = inputs.random_populations(shape, seed=31)
    a = lattice(shape, prec="f32")
    a.set_tile(732080001)
    a.set_populations(f0)
    a.step(130)
    b = lattice(shape, prec="f32")
    b.set_populations(f0)
    b.set_tile(532080001)
    b.step(130)
    assert np.array_equal(a.get_populations(), b.get_populations())
    c = lattice(shape, prec="f32")
    c.set_tile(732080001)
    c.set_populations(f0)
    c.step(3)
    ref = lbm3d.run(f0, oracle_model(), 3)
    rho_ref = lbm3d.density(ref)
    assert np.max(np.abs(c.rho() - rho_ref) / rho_ref) < 2e-6


def test_tma_kernel_is_offered_only_where_it_applies():
    """Kind 7 needs tau = 1, FP32 storage and the box rules; elsewhere its tile code is
    refused and the lattice keeps its kernel."""
    for kw in ({"tau": 0.8}, {"prec": "f64"}):
        lat = lattice((8, 16, 64), **kw)
        before = lat.get_tile()
        with pytest.raises(P.LBMError):
            lat.set_tile(732080001)
        assert lat.get_tile() == before
    lat = lattice((8, 20, 64), prec="f32")            # ny % 8 != 0
    with pytest.raises(P.LBMError):
        lat.set_tile(732080001)


@pytest.mark.parametrize("stencil", ["E6", "E8"])
def test_moment_kernel_wide_stencils(stencil):
    shape = (9, 10, 40)
    f0 = inputs.random_populations(shape, seed=28)
    a = lattice(shape, stencil=stencil)
    a.set_populations(f0)
    a.set_tile(532040001)
    a.step(40)
    ref = lbm3d.run(f0, oracle_model(stencil=stencil), 40)
    assert np.max(np.abs(a.get_populations() - ref)) < 1e-12


@pytest.fixture(scope="module")
def droplet_state_48():
    """The droplet workload in a box wide enough for the FP16 moment kernel (nx = 48)."""
    shape, c = (16, 24, 48), (24, 12, 8)
    n = lbm3d.drop_density(shape, c, 6.0, 1.8883, 0.1193)
    f0 = lbm3d.init_from_density(n)
    return shape, c, f0, lbm3d.run(f0, oracle_model(), 1000)


def test_f16_moment_kernel_parity(droplet_state_48):
    """FP16 storage through the moment kernel (its default at tau = 1, nx % 8 == 0):
    within twice the FP16 storage model's error of the oracle after 1000 steps (see
    test_parity_f16_shifted_1000_steps_droplet), and as close to the register-load
    FP16 kernel."""
    shape, c, f0, ref = droplet_state_48
    rho_ref = lbm3d.density(ref)
    bound = 2.0 * float(np.max(np.abs(lbm3d.density(f16_storage_model(f0, 1000, oracle_model())) - rho_ref)
                               / rho_ref))
    a = lattice(shape, prec="f16")
    assert a.get_tile() // 100000000 == 5
    a.init_drop(c, 6.0, 1.8883, 0.1193, 1.0)
    a.step(1000)
    b = lattice(shape, prec="f16")
    b.set_tile(32080016)                  # register-load kernel, 32 x 8, z chunk 16
    b.init_drop(c, 6.0, 1.8883, 0.1193, 1.0)
    b.step(1000)
    ra, rb = a.rho(), b.rho()
    rel = np.max(np.abs(ra - rho_ref) / rho_ref)
    ab = np.max(np.abs(ra - rb) / rho_ref)
    print(f"f16 moment kernel: max relative density error {rel:.3e}; vs register-load kernel {ab:.3e}; "
          f"bound {bound:.3e}")
    assert np.isfinite(rel) and rel < bound and ab < bound


@pytest.mark.parametrize("prec,code,tau,shape", [(p, c, 1.0, sh) for p in ("f64", "f32")
                                                 for c in (632080001, 632080002)
                                                 for sh in ((13, 22, 72), (11, 21, 37))
                                                 if not (p == "f64" and c == 632080002)]
                         + [("f32", 632080001, 0.8, (11, 21, 37))])
def test_moment_elem_kernel_matches_pipelined_kernel_and_oracle(prec, code, tau, shape):
    """Kind 6: the moment kernel with element copies (any nx, here also odd, as the
    paper's boxes are).  Bitwise equal to the pipelined kernel, and to the oracle;
    tau != 1 runs the pipelined kernel under the same code.  (FP64 with prefetch
    depth 2 does not fit two CTAs per SM and is not offered.)"""
    f0 = inputs.random_populations(shape, seed=29)
    a = lattice(shape, prec=prec, tau=tau)
    a.set_populations(f0)
    a.set_tile(code)
    a.step(130)
    b = lattice(shape, prec=prec, tau=tau)
    b.set_populations(f0)
    b.set_tile(132080001)
    b.step(130)
    assert np.array_equal(a.get_populations(), b.get_populations())
    if prec == "f64":
        ref = lbm3d.run(f0, oracle_model(tau=tau), 130)
        assert np.max(np.abs(a.get_populations() - ref)) < 1e-12


def test_moment_elem_kernel_wide_stencil():
    shape = (9, 10, 37)
    f0 = inputs.random_populations(shape, seed=30)
    a = lattice(shape, stencil="E6")
    a.set_populations(f0)
    a.set_tile(632040001)
    a.step(40)
    ref = lbm3d.run(f0, oracle_model(stencil="E6"), 40)
    assert np.max(np.abs(a.get_populations() - ref)) < 1e-12
