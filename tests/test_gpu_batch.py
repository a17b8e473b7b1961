"""Batches of lattices (lbm_batch_*): every lattice of a batch evolves exactly as the
same lattice run alone with the batch's tile, slots are refilled from the queue, and
small droplets converge by one of the Sec. IV criteria."""
import numpy as np
import pytest

import paper_2105_08772_gb300 as P

pytestmark = pytest.mark.gpu

STATE_KEYS = ("n_in", "n_out", "P_in", "P_out", "dP", "mass", "R_e", "C", "D", "R_s", "max_u")

RUNS = [  # box, tau, G, R, rho_in, rho_out
    ((24, 24, 24), 1.0, -5.0, 6.0, 1.89, 0.12),
    ((40, 32, 28), 1.0, -5.5, 7.0, 0.12, 1.89),     # bubble
    ((33, 27, 35), 1.3, -5.5, 6.5, 1.90, 0.12),     # odd sizes, tau != 1
    ((48, 48, 48), 1.0, -4.6, 11.0, 1.70, 0.25),
    ((16, 20, 12), 1.0, -5.0, 4.0, 1.89, 0.12),
]


@pytest.mark.parametrize("prec,tile", [("f32", 132080161), ("f64", 132040161)])
def test_batch_equals_single_lattice_runs(prec, tile):
    steps, check = 512, 256
    b = P.Batch(2, (48, 48, 48), prec=prec)
    ids = [b.enqueue(box, tau=tau, G=G, R=R, rho_in=ri, rho_out=ro) for box, tau, G, R, ri, ro in RUNS]
    b.run(max_steps=steps, check_every=check, tol_dP_rel=-1.0, tol_du=-1.0)
    for rid, (box, tau, G, R, ri, ro) in zip(ids, RUNS):
        st, ob = b.result(rid)
        assert st == P._lib.LBM_ENOTCONV and ob.steps == steps, (rid, st, ob.steps)
        lat = P.Lattice(*box, tau=tau, G=G, prec=prec)
        lat.set_tile(tile - 160 + 10 * min(16, box[2]))   # the batch's z chunk: min(16, nz)
        lat.init_drop((box[0] // 2, box[1] // 2, box[2] // 2), R, ri, ro)
        lat.step(steps)
        ref = lat.observables()
        for k in STATE_KEYS:
            a, r = getattr(ob, k), getattr(ref, k)
            assert (a == r) or (np.isnan(a) and np.isnan(r)), (rid, k, a, r)
        assert list(ob.com) == list(ref.com)


RUNS_UNIT_TAU = [  # tau = 1 and nx % 4 == 0, nx >= 40: the batch takes the moment kernel
    ((40, 32, 28), 1.0, -5.5, 7.0, 0.12, 1.89),
    ((48, 40, 36), 1.0, -5.0, 9.0, 1.89, 0.12),
    ((44, 20, 13), 1.0, -4.6, 5.0, 1.70, 0.25),
]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_moment_batch_equals_single_lattice_runs(prec):
    """All-tau-1 batches run the moment kernel; each lattice still evolves bitwise as
    it does alone (default tile)."""
    steps, check = 384, 128
    b = P.Batch(2, (48, 40, 36), prec=prec)
    ids = [b.enqueue(box, tau=tau, G=G, R=R, rho_in=ri, rho_out=ro)
           for box, tau, G, R, ri, ro in RUNS_UNIT_TAU]
    b.run(max_steps=steps, check_every=check, tol_dP_rel=-1.0, tol_du=-1.0)
    for rid, (box, tau, G, R, ri, ro) in zip(ids, RUNS_UNIT_TAU):
        st, ob = b.result(rid)
        assert st == P._lib.LBM_ENOTCONV and ob.steps == steps, (rid, st, ob.steps)
        lat = P.Lattice(*box, tau=tau, G=G, prec=prec)
        lat.init_drop((box[0] // 2, box[1] // 2, box[2] // 2), R, ri, ro)
        lat.step(steps)
        ref = lat.observables()
        for k in STATE_KEYS:
            a, r = getattr(ob, k), getattr(ref, k)
            assert (a == r) or (np.isnan(a) and np.isnan(r)), (rid, k, a, r)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_moment_elem_batch_equals_single_lattice_runs(prec):
    """All-tau-1 batches with an odd box (the paper's sizes) run the moment kernel with
    element copies; each lattice still evolves bitwise as it does alone."""
    runs = [((41, 41, 41), 1.0, -5.0, 10.25, 1.89, 0.12), ((37, 29, 23), 1.0, -5.5, 6.0, 0.12, 1.89)]
    steps, check = 256, 128
    b = P.Batch(2, (41, 41, 41), prec=prec)
    ids = [b.enqueue(box, tau=tau, G=G, R=R, rho_in=ri, rho_out=ro) for box, tau, G, R, ri, ro in runs]
    b.run(max_steps=steps, check_every=check, tol_dP_rel=-1.0, tol_du=-1.0)
    for rid, (box, tau, G, R, ri, ro) in zip(ids, runs):
        st, ob = b.result(rid)
        assert st == P._lib.LBM_ENOTCONV and ob.steps == steps, (rid, st, ob.steps)
        lat = P.Lattice(*box, tau=tau, G=G, prec=prec)
        lat.init_drop((box[0] // 2, box[1] // 2, box[2] // 2), R, ri, ro)
        lat.step(steps)
        ref = lat.observables()
        for k in STATE_KEYS:
            a, r = getattr(ob, k), getattr(ref, k)
            assert (a == r) or (np.isnan(a) and np.isnan(r)), (rid, k, a, r)


def test_batch_droplets_converge_and_small_bubbles_collapse():
    """32^3 droplets of R = 8 converge to a centred droplet; bubbles that small dissolve
    into the liquid, which the runs must report as COLLAPSED (status bit 1)."""
    from oracle import eos as E
    coex = {G: E.coexistence(E.EOS("one_minus_exp"), G)[:2] for G in (-5.0, -5.5, -6.0)}
    b = P.Batch(3, (32, 32, 32), prec="f32")
    # Sec. IV: start from the flat-interface coexistence densities of each G
    drops = [b.enqueue((32, 32, 32), G=G, R=8.0, rho_in=coex[G][1], rho_out=coex[G][0]) for G in coex]
    bubbles = {G: b.enqueue((32, 32, 32), G=G, R=8.0, rho_in=coex[G][0], rho_out=coex[G][1])
               for G in (-5.0, -5.5)}
    lu = b.run(max_steps=30_000, check_every=2048)
    assert lu > 0
    for rid in drops:
        st, ob = b.result(rid)
        assert st == 0 and ob.criterion in (1, 2), (rid, st, ob.criterion, ob.steps)
        assert not (ob.status_bits & (2 | 4 | 8 | 16)), ob.status_bits
        assert ob.dP > 0
    for G, rid in bubbles.items():
        st, ob = b.result(rid)
        assert st in (0, P._lib.LBM_ENOTCONV, P._lib.LBM_ECOLLAPSE), st
        collapsed = abs(ob.n_in - ob.n_out) < 1e-2 * (coex[G][1] - coex[G][0])
        assert bool(ob.status_bits & 2) == collapsed
        # a bubble gone for good ends its run early, at the second collapsed check
        if st == P._lib.LBM_ECOLLAPSE:
            assert collapsed and ob.steps < 30_000


def test_batch_rejects_boxes_larger_than_its_slots():
    b = P.Batch(1, (16, 16, 16), prec="f32")
    with pytest.raises(P.LBMError):
        b.enqueue((17, 16, 16))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_autotuned_batch_equals_single_lattice_runs(prec):
    """lbm_batch_autotune times kernel modes, z chunks and slot counts on the resident
    lattices, then starts them again from their drops: the tuned batch still gives each
    lattice bitwise what it gives alone (every kernel kind and z chunk computes the same
    values)."""
    steps, check = 256, 128
    runs = RUNS_UNIT_TAU + [((40, 40, 40), 1.0, -5.0, 9.0, 1.89, 0.12)]
    b = P.Batch(4, (48, 40, 40), prec=prec)
    ids = [b.enqueue(box, tau=tau, G=G, R=R, rho_in=ri, rho_out=ro) for box, tau, G, R, ri, ro in runs]
    code = b.autotune(reps=4)
    mode, zc, slots = code // 1000000, code // 1000 % 1000, code % 1000
    assert mode in (1, 2, 3) and zc in (8, 16, 32) and slots in (2, 4), code
    b.run(max_steps=steps, check_every=check, tol_dP_rel=-1.0, tol_du=-1.0)
    for rid, (box, tau, G, R, ri, ro) in zip(ids, runs):
        st, ob = b.result(rid)
        assert st == P._lib.LBM_ENOTCONV and ob.steps == steps, (rid, st, ob.steps)
        lat = P.Lattice(*box, tau=tau, G=G, prec=prec)
        lat.init_drop((box[0] // 2, box[1] // 2, box[2] // 2), R, ri, ro)
        lat.step(steps)
        ref = lat.observables()
        for k in STATE_KEYS:
            a, r = getattr(ob, k), getattr(ref, k)
            assert (a == r) or (np.isnan(a) and np.isnan(r)), (rid, k, a, r)
        lat.close()


RUNS_F16 = [  # FP16 batches: tau = 1, nx % 8 == 0, nx >= 48
    ((48, 40, 36), 1.0, -5.0, 9.0, 1.89, 0.12),
    ((56, 24, 20), 1.0, -5.5, 5.0, 0.12, 1.89),     # bubble
    ((64, 32, 16), 1.0, -4.6, 6.0, 1.70, 0.25),
]


def test_f16_batch_equals_single_lattice_runs():
    """FP16-shifted batches run the FP16 moment kernel; each lattice keeps its own shift
    and power-of-two scale and evolves bitwise as it does alone (kind 5, the batch's z
    chunk)."""
    steps, check = 384, 128
    b = P.Batch(2, (64, 40, 36), prec="f16")
    ids = [b.enqueue(box, tau=tau, G=G, R=R, rho_in=ri, rho_out=ro) for box, tau, G, R, ri, ro in RUNS_F16]
    with pytest.raises(P.LBMError):
        b.enqueue((40, 40, 40), tau=1.0, G=-5.0, R=8.0, rho_in=1.89, rho_out=0.12)   # nx < 48
    with pytest.raises(P.LBMError):
        b.enqueue((48, 40, 36), tau=0.8, G=-5.0, R=8.0, rho_in=1.89, rho_out=0.12)   # tau != 1
    b.run(max_steps=steps, check_every=check, tol_dP_rel=-1.0, tol_du=-1.0)
    for rid, (box, tau, G, R, ri, ro) in zip(ids, RUNS_F16):
        st, ob = b.result(rid)
        assert st == P._lib.LBM_ENOTCONV and ob.steps == steps, (rid, st, ob.steps)
        lat = P.Lattice(*box, tau=tau, G=G, prec="f16")
        lat.set_tile(532080001 + 10 * min(16, box[2]))
        lat.init_drop((box[0] // 2, box[1] // 2, box[2] // 2), R, ri, ro)
        lat.step(steps)
        ref = lat.observables()
        for k in STATE_KEYS:
            a, r = getattr(ob, k), getattr(ref, k)
            assert (a == r) or (np.isnan(a) and np.isnan(r)), (rid, k, a, r)
        lat.close()
