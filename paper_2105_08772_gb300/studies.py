"""Measurement studies on single lattices.

configs: the plain-method workloads on one GPU -- a 32^3 FP64 droplet (R = 8,
  2000 steps) and 128^3 droplets and bubbles (R = 32) in FP64 and shifted FP32 run
  to the convergence tests of Sec. IV -- with R_e, Delta P, R_s, sigma_s, steps,
  wall time and throughput per run.

precision: one droplet per radius in an L^3 box (psi = 1 - exp(-n), E4), run to
  the convergence tests of Sec. IV with populations stored in FP64, shifted FP32
  and shifted FP16 (2^k scale); for each reduced precision, the error of the
  density field, R_e, Delta P, sigma_s and R_s against the FP64 run.

eos: the Carnahan-Starling-mapped pseudopotential (psi^2 = 2 (p_CS - n c_s^2) /
  (G c_s^2), G = -1, so that Eq. (10) returns p_CS) with the wider isotropic
  stencils E6 / E8: the flat interface of the same stencil gives n_g, n_l and
  sigma_0 (Eq. (25)); a droplet of radius R in an L^3 box then runs to
  convergence and gives R_e, Delta P, R_s, sigma_s.

Every run goes through liblbm.so on the GPU; this module only sequences the
calls and compares the results.

Command line:  python -m paper_2105_08772_gb300.studies configs
               python -m paper_2105_08772_gb300.studies precision --L 192
               python -m paper_2105_08772_gb300.studies eos --L 256 --R 48
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import _lib
from .lbm import Lattice, flat_interface


def cs_critical_point(a: float = 1.0, b: float = 4.0, Rgas: float = 1.0) -> tuple[float, float]:
    """(n_c, T_c) of the Carnahan-Starling pressure p = n R T Z(q) - a n^2, q = b n / 4.

    With g(q) = d(n Z)/dn = (1 + 4q + 4q^2 - 4q^3 + q^4) / (1 - q)^4, the conditions
    dp/dn = 0 and d^2p/dn^2 = 0 read R T g(q) = 8 a q / b and R T g'(q) b / 4 = 2 a,
    whose ratio g(q) = q g'(q) fixes q_c alone; then n_c = 4 q_c / b and
    T_c = 8 a q_c / (b R g(q_c))."""
    def g(q):
        return (1 + 4 * q + 4 * q * q - 4 * q ** 3 + q ** 4) / (1 - q) ** 4

    def dg(q):   # derivative of g, by the quotient rule
        num = 1 + 4 * q + 4 * q * q - 4 * q ** 3 + q ** 4
        dnum = 4 + 8 * q - 12 * q * q + 4 * q ** 3
        return (dnum * (1 - q) + 4 * num) / (1 - q) ** 5

    lo, hi = 0.01, 0.5         # g - q g' changes sign once in here
    f = lambda q: g(q) - q * dg(q)   # noqa: E731
    flo = f(lo)
    for _ in range(200):
        m = 0.5 * (lo + hi)
        fm = f(m)
        if (fm < 0) == (flo < 0):
            lo, flo = m, fm
        else:
            hi = m
    q = 0.5 * (lo + hi)
    return 4 * q / b, 8 * a * q / (b * Rgas * g(q))


def _sync():
    import torch
    torch.cuda.synchronize()


def _run_droplet(L, R, n_in, n_out, prec, G, psi="one_minus_exp", stencil="E4", cs_T=0.0,
                 max_steps=50_000):
    lat = Lattice(L, L, L, G=G, psi=psi, stencil=stencil, prec=prec, cs_T=cs_T)
    try:
        c = L // 2
        lat.init_drop((c, c, c), R, n_in, n_out)
        _sync()
        t0 = time.perf_counter()
        try:
            st, steps, crit = lat.run_to_convergence(max_steps=max_steps)
        except _lib.LBMError as e:
            st, crit = e.status, 0
        _sync()
        wall = time.perf_counter() - t0
        o = lat.observables().as_dict()
        o["criterion"] = crit
        rho = lat.rho()
        return st, o, rho, wall
    finally:
        lat.close()


def _rel(a, b):
    return abs(a - b) / abs(b) if b != 0 else abs(a - b)


def configs(G: float = -5.0, rho_l: float = 2.0, rho_g: float = 0.15, max_steps: int = 50_000) -> dict:
    """The 32^3 and 128^3 plain-method workloads (psi = 1 - exp(-n), E4, tau = 1, unit
    interface width): the literal initial densities 2.0 / 0.15, and at 128^3 also the
    flat-interface coexistence densities of the same G."""
    keys = ("R_e", "dP", "R_s", "sigma_s", "n_in", "n_out", "mass", "max_u", "status_bits")
    out = {"G": G, "rho_l": rho_l, "rho_g": rho_g, "runs": []}
    lat = Lattice(32, 32, 32, G=G, prec="f64")
    try:
        lat.init_drop((16, 16, 16), 8.0, rho_l, rho_g)
        _sync()
        t0 = time.perf_counter()
        lat.step(2000)
        o = lat.observables().as_dict()
        _sync()
        wall = time.perf_counter() - t0
        out["runs"].append({"box": 32, "kind": "droplet", "R": 8.0, "prec": "f64", "steps": 2000,
                            "wall_s": wall, **{k: o[k] for k in keys}})
    finally:
        lat.close()
    # the 128^3 runs from the literal densities and from the flat-interface ones
    # (a bubble started in liquid at 2.0 > n_l takes up its gas and dissolves)
    _, n_g, n_l, _, _ = flat_interface(G)
    out["flat"] = {"n_g": n_g, "n_l": n_l}
    for init, (hi, lo) in (("literal", (rho_l, rho_g)), ("flat", (n_l, n_g))):
        for prec in ("f64", "f32"):
            for kind, (a, b) in (("droplet", (hi, lo)), ("bubble", (lo, hi))):
                st, o, _, wall = _run_droplet(128, 32.0, a, b, prec, G, max_steps=max_steps)
                out["runs"].append({"box": 128, "kind": kind, "R": 32.0, "prec": prec, "init": init,
                                    "status": st, "steps": o["steps"], "criterion": o["criterion"],
                                    "wall_s": wall, "MLUPS": o["steps"] * 128 ** 3 / wall / 1e6,
                                    **{k: o[k] for k in keys}})
    return out


def precision(L: int | None = 192, radii=(12.0, 24.0, 48.0), G: float = -5.0, precs=("f32", "f16"),
              max_steps: int = 50_000, per_R: float | None = None) -> dict:
    """Errors of the reduced-precision storages against FP64, per radius; the box is
    L^3, or (per_R R)^3 when per_R is given."""
    _, n_g, n_l, _, _ = flat_interface(G)
    out = {"L": L, "per_R": per_R, "G": G, "n_g": n_g, "n_l": n_l, "runs": []}
    for R in radii:
        Lr = int(round(per_R * R)) if per_R else L
        st64, o64, rho64, wall64 = _run_droplet(Lr, R, n_l, n_g, "f64", G, max_steps=max_steps)
        row = {"R": R, "L": Lr, "f64": {"status": st64, "steps": o64["steps"], "wall_s": wall64,
                               **{k: o64[k] for k in ("R_e", "dP", "R_s", "sigma_s", "status_bits")}}}
        for p in precs:
            st, o, rho, wall = _run_droplet(Lr, R, n_l, n_g, p, G, max_steps=max_steps)
            row[p] = {"status": st, "steps": o["steps"], "wall_s": wall,
                      "status_bits": o["status_bits"],
                      "rho_max_abs": float(np.max(np.abs(rho - rho64))),
                      "rho_max_rel": float(np.max(np.abs(rho - rho64) / rho64)),
                      **{f"{k}_rel": _rel(o[k], o64[k]) for k in ("R_e", "dP", "R_s", "sigma_s")}}
        out["runs"].append(row)
    return out


def eos(L: int = 256, R: float = 48.0, T_fracs=(0.7, 0.8, 0.9), stencils=("E6", "E8"),
        prec: str = "f32", G: float = -1.0, a: float = 1.0, b: float = 4.0, Rgas: float = 1.0,
        max_steps: int = 50_000) -> dict:
    """Carnahan-Starling-mapped psi with the E6 / E8 stencils: flat coexistence, then a
    droplet of radius R in an L^3 box."""
    n_c, T_c = cs_critical_point(a, b, Rgas)
    out = {"L": L, "R": R, "G": G, "n_c": n_c, "T_c": T_c, "runs": []}
    for st_name in stencils:
        for tf in T_fracs:
            T = tf * T_c
            row = {"stencil": st_name, "T_over_Tc": tf}
            try:
                fs, n_g, n_l, s0, fsteps = flat_interface(G, psi="cs", stencil=st_name, cs_T=T)
            except _lib.LBMError as e:
                row["flat"] = {"error": str(e)}
                out["runs"].append(row)
                continue
            row["flat"] = {"status": fs, "n_g": n_g, "n_l": n_l, "sigma0": s0, "steps": fsteps}
            st, o, rho, wall = _run_droplet(L, R, n_l, n_g, prec, G, psi="cs", stencil=st_name,
                                            cs_T=T, max_steps=max_steps)
            row["droplet"] = {"status": st, "wall_s": wall,
                              "MLUPS": o["steps"] * L ** 3 / wall / 1e6,
                              **{k: o[k] for k in ("steps", "R_e", "dP", "R_s", "sigma_s",
                                                   "n_in", "n_out", "status_bits", "criterion")}}
            out["runs"].append(row)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    sub = ap.add_subparsers(dest="study", required=True)
    p1 = sub.add_parser("precision")
    p1.add_argument("--L", type=int, default=192)
    p1.add_argument("--per-R", type=float, default=0.0, help="box side per_R * R instead of L")
    p1.add_argument("--radii", default="12,24,48")
    p1.add_argument("--G", type=float, default=-5.0)
    p1.add_argument("--max-steps", type=int, default=50_000)
    p0 = sub.add_parser("configs")
    p0.add_argument("--max-steps", type=int, default=50_000)
    p2 = sub.add_parser("eos")
    p2.add_argument("--L", type=int, default=256)
    p2.add_argument("--R", type=float, default=48.0)
    p2.add_argument("--T-fracs", default="0.7,0.8,0.9")
    p2.add_argument("--stencils", default="E6,E8")
    p2.add_argument("--max-steps", type=int, default=50_000)
    for p in (p0, p1, p2):
        p.add_argument("--out", default="")
    a = ap.parse_args(argv)
    if a.study == "configs":
        res = configs(max_steps=a.max_steps)
    elif a.study == "precision":
        res = precision(a.L, tuple(float(r) for r in a.radii.split(",")), a.G, max_steps=a.max_steps,
                        per_R=a.per_R or None)
    else:
        res = eos(a.L, a.R, tuple(float(t) for t in a.T_fracs.split(",")), tuple(a.stencils.split(",")),
                  max_steps=a.max_steps)
    text = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    print(text)
    return res


if __name__ == "__main__":
    main()
