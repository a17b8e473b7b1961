"""The measurement sweep of Sec. IV: droplets and bubbles over radii and couplings.

For each coupling G the flat interface (Eq. (24), run on the GPU by
lbm_flat_interface) gives the bulk densities n_g, n_l that initialise the
droplets and bubbles (Eq. (23): droplets n_in = n_l, bubbles n_in = n_g) and the
flat tension sigma_0 of Eq. (25).  Every droplet and bubble then runs to
hydrostatic equilibrium under the two convergence tests of Sec. IV, and its
observables (R_e, Delta P, sigma[R], R_s, sigma_s = Delta P R_s / 2) feed

* the Tolman fit of Eq. (22): sigma_s = sigma_0 (1 - 2 delta x + c x^2) with
  x = +1/R_s for droplets and -1/R_s for bubbles (lbm_tolman_fit), and
* the alternative Tolman length of Sec. IV (last paragraph),
  hat-delta_+- = +-(R_e - R_s), extrapolated to the flat limit 1/R_s -> 0 by a
  straight line in the signed curvature x.

Two ways to run the same list of problems:
* run_batched: every lattice in a lbm_batch (uneven boxes advance together, one
  launch per time step, graph-captured, slots refilled as lattices finish);
* run_plain: one lattice at a time through lbm_create / lbm_run_to_convergence.

Everything runs on the GPU through liblbm.so; this module only plans the runs,
calls the library and collects the results.

Command lines:  python -m paper_2105_08772_gb300.sweep --couplings -5.0 --radii 6:40:2
                python -m paper_2105_08772_gb300.sweep --paper --max-L 157
(--paper: the paper's own sweep, 12 reduced couplings x 2 pseudopotentials x odd
boxes with R = L/4, and the power law delta = A eps^lambda of Sec. IV.  Boxes
above --big-L run only where the smaller ones cannot hold the wide interfaces,
eps <= --big-eps, as a second batch whose slot count fits the device memory.)
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import asdict, dataclass, field

import numpy as np

from . import _lib
from .lbm import Batch, Lattice, flat_interface, lbm_tolman_fit

RADII = tuple(range(6, 41, 2))
COUPLINGS = (-4.6, -5.0, -5.5, -6.0)

# the paper's own sweep (Sec. IV): reduced couplings G/G_c - 1, odd box sides, R = L/4
PAPER_EPS = (0.029, 0.033, 0.038, 0.045, 0.056, 0.070, 0.079, 0.091, 0.119, 0.159, 0.215, 0.293)
PAPER_L = (41, 43, 47, 51, 55, 61, 67, 77, 87, 103, 123, 157, 213, 335)
PAPER_PSI = ("exp_inv", "one_minus_exp")


def critical_coupling(psi: str) -> float:
    """G_c of Sec. IV: G_c c_s^2 = -2.463 (psi = exp(-1/n), G_c = -e^2) and -1.333
    (psi = 1 - exp(-n), G_c = -4)."""
    if psi == "exp_inv":
        return -math.e ** 2
    if psi == "one_minus_exp":
        return -4.0
    raise ValueError(f"no closed-form G_c for psi {psi!r}")

# lbm_obs.status_bits that disqualify a run from the fits
_BAD_BITS = 1 | 2 | 4 | 8 | 16     # no sigma minimum, collapsed, off centre, non-finite, timeout


def box_side(R: float, L_min: int = 64, per_R: float = 4.0, L_max: int | None = None) -> int:
    """Side of the periodic box of a run of initial radius R: max(L_min, ceil(per_R R))."""
    L = max(int(L_min), int(math.ceil(per_R * R - 1e-9)))
    if L_max is not None and L > L_max:
        raise ValueError(f"R = {R} needs a box of {L} > {L_max}")
    return L


@dataclass(frozen=True)
class Run:
    G: float
    bubble: bool
    R: float
    L: int
    psi: str = "one_minus_exp"
    tau: float = 1.0


@dataclass
class Outcome:
    run: Run
    status: int
    obs: dict = field(default_factory=dict)

    @property
    def usable(self) -> bool:
        """Converged, centred, with a minimum of sigma[R] (Sec. IV's analysis condition)."""
        return (self.status == _lib.LBM_OK and not (int(self.obs.get("status_bits", 0)) & _BAD_BITS)
                and self.obs.get("R_s", 0.0) > 0.0)

    @property
    def x(self) -> float:
        """Signed curvature: +1/R_s for droplets, -1/R_s for bubbles (Sec. IV)."""
        return (-1.0 if self.run.bubble else 1.0) / self.obs["R_s"]

    @property
    def delta_hat(self) -> float:
        """hat-delta_+- = +-(R_e - R_s), + for droplets, - for bubbles (Sec. IV)."""
        d = self.obs["R_e"] - self.obs["R_s"]
        return -d if self.run.bubble else d


def plan(couplings=COUPLINGS, radii=RADII, psi: str = "one_minus_exp", kinds=("drop", "bubble"),
         L_min: int = 64, per_R: float = 4.0, tau: float = 1.0) -> list[Run]:
    """All (G, kind, R) problems, largest box first (the longest runs start first)."""
    runs = [Run(float(G), k == "bubble", float(R), box_side(R, L_min, per_R), psi, tau)
            for G in couplings for k in kinds for R in radii]
    runs.sort(key=lambda r: (-r.L, r.G, r.bubble, r.R))
    return runs


def plan_paper(eps=PAPER_EPS, psis=PAPER_PSI, sizes=PAPER_L, kinds=("drop", "bubble"),
               tau: float = 1.0) -> list[Run]:
    """The paper's sweep: for each psi and reduced coupling eps, G = G_c (1 + eps), and
    for each odd side L a droplet and a bubble of initial radius R = L/4 centred on the
    node (L // 2, L // 2, L // 2).  Largest box first."""
    runs = [Run(critical_coupling(p) * (1.0 + e), k == "bubble", L / 4.0, int(L), p, tau)
            for p in psis for e in eps for k in kinds for L in sizes]
    runs.sort(key=lambda r: (-r.L, r.psi, r.G, r.bubble))
    return runs


def reduced_coupling(run: Run) -> float:
    return run.G / critical_coupling(run.psi) - 1.0


def power_law(eps, delta) -> tuple[float, float]:
    """(A, lambda) of delta = A eps^lambda by least squares in log-log (Sec. IV finds
    lambda close to -1); points with delta <= 0 are left out."""
    e = np.asarray(eps, dtype=np.float64)
    d = np.asarray(delta, dtype=np.float64)
    keep = (e > 0) & (d > 0)
    if keep.sum() < 2:
        return float("nan"), float("nan")
    lam, logA = np.polyfit(np.log(e[keep]), np.log(d[keep]), 1)
    return float(np.exp(logA)), float(lam)


def coexistence(couplings, psi: str = "one_minus_exp", stencil: str = "E4", Lx: int = 100,
                tol_du: float = 1e-13, max_steps: int = 400_000) -> dict:
    """Flat-interface bulk densities and sigma_0 per coupling, FP64 on the GPU, each
    started from the library's continuum estimate.
    G -> {"n_g", "n_l", "sigma0", "steps", "status"}."""
    out = {}
    for G in couplings:
        st, ng, nl, s0, steps = flat_interface(G, psi=psi, stencil=stencil, prec="f64", Lx=Lx,
                                               max_steps=max_steps, tol_du=tol_du)
        out[float(G)] = {"n_g": ng, "n_l": nl, "sigma0": s0, "steps": steps, "status": st}
    return out


def _densities(run: Run, coex: dict) -> tuple[float, float]:
    c = coex[run.G]
    return (c["n_g"], c["n_l"]) if run.bubble else (c["n_l"], c["n_g"])


def _sync():
    import torch
    torch.cuda.synchronize()


def run_batched(runs, coex, slots: int = 64, prec: str = "f32", stencil: str = "E4",
                max_steps: int = 50_000, check_every: int = 2048, tol_dP_rel: float = 1e-5,
                tol_du: float = 1e-12, width: float = 1.0, autotune: bool = False):
    """All runs through one lbm_batch (after lbm_batch_autotune if asked).  Returns
    (outcomes, wall seconds, lattice updates); the tuning time is in the wall time."""
    L = max(r.L for r in runs)
    slots = min(slots, len(runs), slots_that_fit((L, L, L), stencil, prec))
    _sync()
    t0 = time.perf_counter()
    b = Batch(slots, (L, L, L), stencil=stencil, prec=prec)
    try:
        ids = []
        for r in runs:
            n_in, n_out = _densities(r, coex)
            ids.append(b.enqueue((r.L, r.L, r.L), tau=r.tau, G=r.G, psi=r.psi, R=r.R, rho_in=n_in,
                                 rho_out=n_out, width=width))
        if autotune:
            b.autotune()
        lu = b.run(max_steps=max_steps, check_every=check_every, tol_dP_rel=tol_dP_rel, tol_du=tol_du)
        outs = []
        for r, rid in zip(runs, ids):
            st, o = b.result(rid)
            outs.append(Outcome(r, st, o.as_dict()))
    finally:
        b.close()
    _sync()
    return outs, time.perf_counter() - t0, lu


def slots_that_fit(max_box, stencil: str = "E4", prec: str = "f32", share: float = 0.85) -> int:
    """How many batch slots of max_box fit in `share` of the device's free memory."""
    import torch
    from ._lib import PRECS, STENCILS, lib
    from .lbm import make_box
    one = lib.lbm_batch_workspace_bytes(1, make_box(*max_box), STENCILS[stencil], PRECS[prec])
    two = lib.lbm_batch_workspace_bytes(2, make_box(*max_box), STENCILS[stencil], PRECS[prec])
    per_slot = max(two - one, 1)
    free, _ = torch.cuda.mem_get_info()
    return max(1, int((share * free - one) // per_slot) + 1)


def run_plain(runs, coex, prec: str = "f64", stencil: str = "E4", max_steps: int = 50_000,
              check_every: int = 2048, tol_dP_rel: float = 1e-5, tol_du: float = 1e-12,
              width: float = 1.0):
    """One lattice at a time.  Returns (outcomes, wall seconds, lattice updates)."""
    _sync()
    t0 = time.perf_counter()
    outs, lu = [], 0
    for r in runs:
        lat = Lattice(r.L, r.L, r.L, tau=r.tau, G=r.G, psi=r.psi, stencil=stencil, prec=prec)
        try:
            n_in, n_out = _densities(r, coex)
            c = r.L // 2
            lat.init_drop((c, c, c), r.R, n_in, n_out, width)
            crit = 0
            try:
                st, _, crit = lat.run_to_convergence(max_steps=max_steps, check_every=check_every,
                                                     tol_dP_rel=tol_dP_rel, tol_du=tol_du)
            except _lib.LBMError as e:
                st = e.status
            # the observables of the field the run ended on (recomputed, same values)
            o = lat.observables().as_dict()
            o["criterion"] = crit
            lu += int(o["steps"]) * lat.N
            outs.append(Outcome(r, st, o))
        finally:
            lat.close()
    _sync()
    return outs, time.perf_counter() - t0, lu


def shard(runs, rank: int, world: int):
    """The runs of one rank when the sweep is spread over `world` processes (one GPU
    each): round-robin over the largest-first plan, so every rank gets a similar mix
    of box sizes.  The lattices are independent; nothing is exchanged while they run."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world {world}")
    return list(runs[rank::world])


def gather_outcomes(local, group=None):
    """All ranks' outcomes on every rank (control plane only: small Python objects
    through torch.distributed.all_gather_object), in rank order."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return list(local)
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, [(asdict(o.run), o.status, dict(o.obs)) for o in local], group=group)
    return [Outcome(Run(**r), st, obs) for part in parts for (r, st, obs) in part]


def gather_outcomes_counts(count: int, group=None) -> list:
    """Every rank's count (lattice updates), in rank order."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return [count]
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, int(count), group=group)
    return parts


def max_over_ranks(seconds: float, group=None) -> float:
    """The slowest rank's wall time (the job's time)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return seconds
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, float(seconds), group=group)
    return max(parts)


@dataclass
class TolmanResult:
    G: float
    sigma0: float          # extrapolated flat tension (Eq. (22) at x = 0)
    delta: float           # Tolman length
    c: float               # second-order coefficient
    delta_hat0: float      # hat-delta extrapolated to 1/R_s -> 0
    n_used: int
    sigma0_lin: float = 0.0    # the same fit without the x^2 term (Sec. IV's straight lines)
    delta_lin: float = 0.0
    sigma0_flat: float | None = None


def tolman(outcomes, coex: dict | None = None, quadratic: bool = True, min_runs: int = 4) -> dict:
    """Per coupling: the fit of Eq. (22) over the usable runs, and the flat-limit
    hat-delta (straight line in x).  G -> TolmanResult."""
    res = {}
    for G in sorted({o.run.G for o in outcomes}):
        use = [o for o in outcomes if o.run.G == G and o.usable]
        if len(use) < min_runs:
            continue
        Rs = np.array([o.obs["R_s"] for o in use])
        ss = np.array([o.obs["sigma_s"] for o in use])
        bub = np.array([o.run.bubble for o in use], dtype=np.int32)
        s0, d, c = lbm_tolman_fit(Rs, ss, bub, quadratic=quadratic)
        s0l, dl, _ = lbm_tolman_fit(Rs, ss, bub, quadratic=False)
        x = np.array([o.x for o in use])
        dh = np.array([o.delta_hat for o in use])
        A = np.stack([np.ones_like(x), x], axis=1)
        dh0 = float(np.linalg.lstsq(A, dh, rcond=None)[0][0])
        res[G] = TolmanResult(G, s0, d, c, dh0, len(use), s0l, dl,
                              None if coex is None else coex[G]["sigma0"])
    return res


def compare(a: dict, b: dict) -> dict:
    """Relative differences of sigma_0 and delta (and hat-delta_0) between two fits."""
    out = {}
    for G in sorted(set(a) & set(b)):
        ra, rb = a[G], b[G]
        out[G] = {"sigma0": abs(ra.sigma0 - rb.sigma0) / abs(rb.sigma0),
                  "delta": abs(ra.delta - rb.delta) / abs(rb.delta),
                  "delta_hat0": abs(ra.delta_hat0 - rb.delta_hat0) / abs(rb.delta_hat0)}
    return out


def compare_runs(a, b) -> dict:
    """Largest relative difference of R_s and sigma_s over runs usable in both lists."""
    key = lambda o: (o.run.G, o.run.bubble, o.run.R)  # noqa: E731
    bm = {key(o): o for o in b}
    dRs = dss = 0.0
    n = 0
    for o in a:
        p = bm.get(key(o))
        if p is None or not (o.usable and p.usable):
            continue
        n += 1
        dRs = max(dRs, abs(o.obs["R_s"] - p.obs["R_s"]) / p.obs["R_s"])
        dss = max(dss, abs(o.obs["sigma_s"] - p.obs["sigma_s"]) / p.obs["sigma_s"])
    return {"runs": n, "R_s": dRs, "sigma_s": dss}


def _parse_radii(s: str):
    if ":" in s:
        a, b, c = (float(v) for v in s.split(":"))
        return tuple(np.arange(a, b + 0.5 * c, c))
    return tuple(float(v) for v in s.split(","))


def main(argv=None) -> dict:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--couplings", default=",".join(str(g) for g in COUPLINGS))
    ap.add_argument("--radii", default="6:40:2")
    ap.add_argument("--psi", default="one_minus_exp")
    ap.add_argument("--slots", type=int, default=64)
    ap.add_argument("--prec", default="f32")
    ap.add_argument("--max-steps", type=int, default=50_000)
    ap.add_argument("--L-min", type=int, default=64)
    ap.add_argument("--per-R", type=float, default=4.0)
    ap.add_argument("--plain", default="", help="couplings also run one lattice at a time in FP64")
    ap.add_argument("--out", default="")
    ap.add_argument("--autotune", action="store_true", help="lbm_batch_autotune before each batch run")
    ap.add_argument("--paper", action="store_true",
                    help="the paper's sweep: 12 reduced couplings x 2 psi x odd L (see --max-L)")
    ap.add_argument("--max-L", type=int, default=335, help="largest box side of --paper")
    ap.add_argument("--big-L", type=int, default=213,
                    help="--paper: boxes above this side run only at eps <= --big-eps, in a batch of their own")
    ap.add_argument("--big-eps", type=float, default=0.038)
    ap.add_argument("--big-max-steps", type=int, default=80_000)
    ap.add_argument("--distributed", action="store_true",
                    help="one process per GPU under torchrun: the runs are sharded over the ranks")
    a = ap.parse_args(argv)
    rank, world = 0, 1
    if a.distributed:
        import os

        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("gloo")   # only small Python objects travel
        rank, world = dist.get_rank(), dist.get_world_size()
    t0 = time.perf_counter()
    if a.paper:
        runs = plan_paper(sizes=tuple(L for L in PAPER_L if L <= a.max_L))
        runs = [r for r in runs if r.L <= a.big_L or reduced_coupling(r) <= a.big_eps + 1e-9]
        coex = {}
        for p in PAPER_PSI:
            coex.update(coexistence(sorted({r.G for r in runs if r.psi == p}), psi=p))
    else:
        couplings = tuple(float(g) for g in a.couplings.split(","))
        radii = _parse_radii(a.radii)
        runs = plan(couplings, radii, psi=a.psi, L_min=a.L_min, per_R=a.per_R)
        coex = coexistence(couplings, psi=a.psi)
    t_flat = time.perf_counter() - t0
    mine = shard(runs, rank, world)
    # boxes above --big-L (paper sweep) take slots of their own size: a second batch
    groups = [[r for r in mine if not a.paper or r.L <= a.big_L], [r for r in mine if a.paper and r.L > a.big_L]]
    outs, wall, lu = [], 0.0, 0
    for g, cap in zip(groups, (a.max_steps, max(a.max_steps, a.big_max_steps))):
        if not g:
            continue
        o, w, n = run_batched(g, coex, slots=a.slots, prec=a.prec, max_steps=cap, autotune=a.autotune)
        outs, wall, lu = outs + o, wall + w, lu + n
    if world > 1:
        outs = gather_outcomes(outs)
        wall = max_over_ranks(wall)
        lu = int(sum(gather_outcomes_counts(lu)))
    fit = tolman(outs, coex)
    report = {"runs": len(runs), "usable": sum(o.usable for o in outs), "flat_wall_s": t_flat,
              "ranks": world,
              "batched": {"prec": a.prec, "slots": a.slots, "wall_s": wall, "lattice_updates": lu,
                          "MLUPS": lu / wall / 1e6},
              "coexistence": {str(G): v for G, v in coex.items()},
              "fit": {str(G): asdict(r) for G, r in fit.items()}}
    if a.paper:
        rows = []
        for G, f in sorted(fit.items()):
            run = next(r for r in runs if r.G == G)
            rows.append({"psi": run.psi, "eps": reduced_coupling(run), "G": G, "delta": f.delta_lin,
                         "sigma0": f.sigma0_lin, "sigma0_flat": f.sigma0_flat,
                         "delta_quadratic": f.delta, "delta_hat0": f.delta_hat0, "n_used": f.n_used})
        report["paper"] = {"per_coupling": rows}
        # flat-interface sigma_0 against eps for every coupling (mean field: exponent 3/2)
        flat_rows = []
        for p in PAPER_PSI:
            for G in sorted({r.G for r in runs if r.psi == p}):
                e = G / critical_coupling(p) - 1.0
                flat_rows.append({"psi": p, "eps": e, "sigma0_flat": coex[G]["sigma0"],
                                  "n_g": coex[G]["n_g"], "n_l": coex[G]["n_l"]})
        report["paper"]["flat"] = flat_rows
        for p in PAPER_PSI:
            sel = [r for r in flat_rows if r["psi"] == p]
            A, mu = power_law([r["eps"] for r in sel], [r["sigma0_flat"] for r in sel])
            report["paper"][f"sigma0_power_law_{p}"] = {"A": A, "mu": mu}
        for p in PAPER_PSI + ("both",):
            sel = [r for r in rows if p == "both" or r["psi"] == p]
            A, lam = power_law([r["eps"] for r in sel], [r["delta"] for r in sel])
            Ah, lamh = power_law([r["eps"] for r in sel], [r["delta_hat0"] for r in sel])
            report["paper"][f"power_law_{p}"] = {"A": A, "lambda": lam, "A_hat": Ah, "lambda_hat": lamh,
                                                 "couplings": len(sel)}
    if a.plain and rank == 0 and world == 1:
        pc = tuple(float(g) for g in a.plain.split(","))
        sub = [r for r in runs if r.G in pc]
        sub_b = [o for o in outs if o.run.G in pc]
        outs_p, wall_p, lu_p = run_plain(sub, coex, prec="f64", max_steps=a.max_steps)
        fit_p = tolman(outs_p, coex)
        # the batched path on the same subset alone, for a like-for-like wall time
        outs_s, wall_s, lu_s = run_batched(sub, coex, slots=a.slots, prec=a.prec, max_steps=a.max_steps,
                                           autotune=a.autotune)
        report["plain_f64"] = {"runs": len(sub), "wall_s": wall_p, "lattice_updates": lu_p,
                               "MLUPS": lu_p / wall_p / 1e6,
                               "fit": {str(G): asdict(r) for G, r in fit_p.items()}}
        report["batched_subset"] = {"runs": len(sub), "wall_s": wall_s, "lattice_updates": lu_s,
                                    "MLUPS": lu_s / wall_s / 1e6}
        report["batched_vs_plain"] = {"fit": {str(G): v for G, v in compare(fit, fit_p).items()},
                                      "runs": compare_runs(sub_b, outs_p)}
    report["per_run"] = [{"psi": o.run.psi, "G": o.run.G, "bubble": o.run.bubble, "R": o.run.R, "L": o.run.L,
                          "status": o.status, "usable": o.usable,
                          **{k: o.obs[k] for k in ("R_e", "R_s", "sigma_s", "dP", "n_in", "n_out",
                                                   "steps", "status_bits", "criterion")}}
                         for o in outs]
    if rank != 0:
        return report
    text = json.dumps(report, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    print(json.dumps({k: v for k, v in report.items() if k != "per_run"}, indent=1))
    return report


if __name__ == "__main__":
    main()
