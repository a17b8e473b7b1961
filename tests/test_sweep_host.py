"""Host logic of the sweep (paper_2105_08772_gb300.sweep): run plan, box sides,
run selection, signed curvature, hat-delta and the per-coupling fits (Sec. IV,
Eq. (22)).  The fits call lbm_tolman_fit, host code of liblbm.so, on exact
synthetic data whose answer is known in closed form."""
import pytest

S = pytest.importorskip("paper_2105_08772_gb300.sweep")
from paper_2105_08772_gb300 import _lib  # noqa: E402


def test_box_sides_of_the_sweep():
    """L = max(64, ceil(4R)): 64 up to R = 16, then 72 ... 160 in steps of 8."""
    assert [S.box_side(R) for R in (6, 16, 18, 20, 40)] == [64, 64, 72, 80, 160]
    assert S.box_side(16.5) == 66
    with pytest.raises(ValueError):
        S.box_side(50, L_max=160)


def test_plan_covers_every_problem_largest_first():
    runs = S.plan()
    assert len(runs) == 18 * 2 * 4
    assert len({(r.G, r.bubble, r.R) for r in runs}) == len(runs)
    assert [r.L for r in runs] == sorted((r.L for r in runs), reverse=True)
    assert runs[0].L == 160 and runs[-1].L == 64


def _outcome(G, bubble, R_s, sigma_s, R_e, status=0, bits=0):
    run = S.Run(G, bubble, R_s, S.box_side(R_s))
    return S.Outcome(run, status, {"R_s": R_s, "sigma_s": sigma_s, "R_e": R_e, "status_bits": bits})


def test_usable_follows_status_and_bits():
    assert _outcome(-5, False, 10, 0.03, 10.5).usable
    assert not _outcome(-5, False, 10, 0.03, 10.5, status=_lib.LBM_ENOTCONV).usable
    for bit in (1, 2, 4, 8, 16):
        assert not _outcome(-5, False, 10, 0.03, 10.5, bits=bit).usable
    assert not _outcome(-5, False, 0.0, 0.03, 10.5).usable


def test_signed_curvature_and_delta_hat():
    d = _outcome(-5, False, 10.0, 0.03, 10.4)
    b = _outcome(-5, True, 10.0, 0.03, 9.7)
    assert d.x == pytest.approx(0.1) and b.x == pytest.approx(-0.1)
    assert d.delta_hat == pytest.approx(0.4) and b.delta_hat == pytest.approx(0.3)


def test_tolman_recovers_exact_coefficients():
    """sigma_s = sigma_0 (1 - 2 delta x + c x^2), hat-delta = h0 + a x, exactly: the fits
    return sigma_0, delta, c and h0; unusable runs are left out."""
    s0, delta, c, h0, a = 0.0363, 0.57, 1.3, 0.41, -2.0
    outs = []
    for bubble in (False, True):
        for Rs in (8.0, 11.0, 15.0, 22.0, 31.0):
            x = (-1.0 if bubble else 1.0) / Rs
            ss = s0 * (1 - 2 * delta * x + c * x * x)
            dh = h0 + a * x
            Re = Rs + (-dh if bubble else dh)
            outs.append(_outcome(-5.0, bubble, Rs, ss, Re))
    outs.append(_outcome(-5.0, False, 5.0, 1.0, 3.0, bits=1))    # no minimum: ignored
    fit = S.tolman(outs)[-5.0]
    assert fit.n_used == 10
    assert fit.sigma0 == pytest.approx(s0, rel=1e-12)
    assert fit.delta == pytest.approx(delta, rel=1e-10)
    assert fit.c == pytest.approx(c, rel=1e-8)
    assert fit.delta_hat0 == pytest.approx(h0, rel=1e-12)


def test_tolman_needs_enough_runs_and_compare():
    outs = [_outcome(-5.0, False, R, 0.03 * (1 - 1.0 / R), R + 0.4) for R in (8.0, 12.0, 20.0)]
    assert S.tolman(outs) == {}
    a = {-5.0: S.TolmanResult(-5.0, 1.0, 0.5, 0.0, 0.4, 10)}
    b = {-5.0: S.TolmanResult(-5.0, 1.001, 0.5005, 0.0, 0.4, 10)}
    r = S.compare(a, b)[-5.0]
    assert r["sigma0"] == pytest.approx(0.001 / 1.001) and r["delta"] == pytest.approx(0.0005 / 0.5005)
    assert r["delta_hat0"] == 0.0


def test_paper_plan_and_couplings():
    """Sec. IV: G = G_c (1 + eps) with G_c = -e^2 and -4; odd L; R = L/4."""
    runs = S.plan_paper()
    assert len(runs) == 2 * 12 * 2 * 14
    assert all(r.L % 2 == 1 and r.R == r.L / 4 for r in runs)
    eps = sorted({round(S.reduced_coupling(r), 12) for r in runs if r.psi == "exp_inv"})
    assert eps == sorted(S.PAPER_EPS)
    assert S.critical_coupling("exp_inv") * (1 / 3) == pytest.approx(-2.463, abs=1e-3)
    assert S.critical_coupling("one_minus_exp") * (1 / 3) == pytest.approx(-1.333, abs=1e-3)
    assert runs[0].L == 335


def test_power_law_recovers_exponent():
    import numpy as np
    e = np.array(S.PAPER_EPS)
    A, lam = S.power_law(e, 0.3 * e ** -1.0)
    assert A == pytest.approx(0.3, rel=1e-12) and lam == pytest.approx(-1.0, abs=1e-12)
    A, lam = S.power_law([0.1, 0.2, 0.3], [-1.0, 2.0, 1.0])   # non-positive delta left out
    assert lam == pytest.approx(np.log(0.5) / np.log(1.5))


def test_paper_lists_match_the_printed_values():
    """The sweep's reduced couplings and box sides are the ones Sec. IV prints
    (tests/golden/paper_constants.json, with its citations)."""
    import json
    from pathlib import Path
    g = json.loads((Path(__file__).parent / "golden" / "paper_constants.json").read_text())
    assert list(S.PAPER_EPS) == g["reduced_couplings"]["values"]
    assert list(S.PAPER_L) == g["box_sizes"]["values"]


def test_flat_limit_of_delta_hat_matches_the_oracle():
    """sweep.tolman's hat-delta_0 against oracle.observables.delta_hat_flat_limit on the
    same (noisy) outcomes."""
    import numpy as np
    from oracle import observables as O
    rng = np.random.default_rng(3)
    outs = []
    for bubble in (False, True):
        for Rs in (9.0, 12.5, 16.0, 21.0, 27.0, 35.0):
            Re = Rs + (-1.0 if bubble else 1.0) * (0.8 + 0.1 * rng.standard_normal())
            outs.append(_outcome(-5.0, bubble, Rs, 0.036 + 1e-3 * rng.standard_normal(), Re))
    got = S.tolman(outs)[-5.0].delta_hat0
    want = O.delta_hat_flat_limit([o.obs["R_e"] for o in outs], [o.obs["R_s"] for o in outs],
                                  [o.run.bubble for o in outs])
    assert got == pytest.approx(want, rel=1e-12)
