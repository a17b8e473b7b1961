"""Benchmark of the Shan-Chen droplet/bubble hot path (one JSON line on rank 0).

Workload (the 128^3 plain-method configuration): a droplet and a bubble of
radius 32 in periodic 128^3 boxes, psi = 1 - exp(-n), G = -5, tau = 1, E4
stencil, populations stored shifted in FP32 (FP64 observables).  One bench
step = one convergence interval of the paper (2^11 lattice-Boltzmann steps)
on both lattices, followed by the convergence/observable pass (pressure tensor
samples, FP64 reductions, R_e, Delta P, C, R_s) on both.  value = lattice
updates per second over all ranks (MLUPS).

--impl reference times the FP64 CPU oracle on the same workload and metric
(a bounded sample: one lattice-Boltzmann step per lattice per bench step).
Multi-GPU (torchrun): every rank advances its own pair of lattices (the sweep
shards into independent lattices; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

SIZE = 128
RADIUS = 32.0
G = -5.0
TAU = 1.0
RHO_L, RHO_G = 2.0, 0.15          # initial tanh densities of the workload
LBM_STEPS_PER_STEP = 2048         # the paper's convergence interval
BYTES_PER_LU = {"f64": 304, "f32": 152, "f16": 76}   # 19 loads + 19 stores per node
WORKLOAD = ("two 128^3 periodic lattices (droplet R=32, bubble R=32), psi=1-exp(-n), G=-5, "
            "tau=1, D3Q19 E4 Guo-BGK; 2048 LB steps + convergence/observable pass per step")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peak_gbs():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            return float(json.loads(p.read_text())["hbm_gbs"]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


KERNEL_SOURCES = ("lbm_common.cuh", "lbm_kernels.cuh", "lbm_kernels_async.cuh", "lbm_kernels_chunk.cuh",
                  "lbm_kernels_moment.cuh", "lbm_kernels_tma.cuh", "lbm_lattice_inst.cuh")


PROFILE_STEMS = {7: "lattice_tma", 6: "lattice_moment_elem", 5: "lattice_moment"}


def profile_fields(stem, prec, box=128):
    """The machine-readable lines (``key: value``) of a committed ncu summary, or None
    when there is none or the kernel sources changed since it was captured (its
    source_sha256 differs from the current sources')."""
    import hashlib
    summary = ROOT / "profiles" / f"{stem}_{prec}_{box}.md"
    if not summary.exists():
        return None
    fields = {}
    for line in summary.read_text().splitlines():
        if ":" in line and not line.startswith(("|", " ", "#")):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    csrc = ROOT / "paper_2105_08772_gb300" / "csrc"
    h = hashlib.sha256(b"".join((csrc / f).read_bytes() for f in KERNEL_SOURCES)).hexdigest()
    if fields.get("source_sha256") != h:
        return None
    fields["path"] = str(summary.relative_to(ROOT))
    return fields


def measured_traffic(prec, kind=5):
    """DRAM bytes per launch of the step kernel from the committed ncu summary of the
    128^3 workload, or None when there is none for this kernel and precision or the
    kernel sources changed since."""
    stem = PROFILE_STEMS.get(int(kind))
    fields = profile_fields(stem, prec) if stem else None
    if not fields or "traffic_bytes_per_launch" not in fields:
        return None
    return int(fields["traffic_bytes_per_launch"])


def fp64_bound(hbm_gbs, peak):
    """What bounds the FP64 step: this run's DRAM fraction, and the FP64 pipe's load
    from the committed ncu summary when it was taken on the current sources (else
    the bound is left null)."""
    frac = hbm_gbs / peak
    prof = profile_fields("lattice_moment", "f64")
    pipe = float(prof["fp64_pipe_pct"]) if prof and "fp64_pipe_pct" in prof else None
    bound = None
    evidence = f"this run: DRAM at {100 * frac:.1f}% of the measured HBM peak"
    if pipe is not None:
        bound = "alu" if pipe >= 50.0 and frac < 0.5 else ("hbm" if frac >= 0.5 else None)
        evidence += f"; ncu on the current sources: FP64 pipe {pipe:.1f}% busy ({prof['path']})"
    return {"hbm_frac": frac, "bound": bound, "evidence": evidence}


KERNEL_KINDS = {
    7: "lattice_tma_kernel (TMA tensor-tile pull + on-chip psi halo + SC force + Guo-BGK at tau = 1 + store)",
    6: "lattice_moment_kernel, element copies (pull + on-chip psi halo + SC force + Guo-BGK at tau = 1 + store)",
    5: "lattice_moment_kernel, row chunks (pull + on-chip psi halo + SC force + Guo-BGK at tau = 1 + store)",
    4: "lattice_chunk_kernel", 1: "lattice_async_kernel", 0: "lattice_kernel",
}


def kernel_name(tile_code):
    """The fused step kernel a tile code selects (kind = code / 10^8)."""
    return "fused step, " + KERNEL_KINDS.get(int(tile_code) // 100000000, f"kind {int(tile_code) // 100000000}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def host_cpu():
    """Core count and CPU model of this host (the oracle's timing runs on all of its cores)."""
    import platform
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in Path("/proc/cpuinfo").read_text().splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": cores, "model": model or platform.machine()}


def _mem_available_bytes():
    try:
        for line in Path("/proc/meminfo").read_text().splitlines():
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except Exception:
        pass
    return None


ORACLE_BYTES_PER_LATTICE = 2.5e9     # peak resident set of one 128^3 oracle step (measured 1.5 GB)


def _oracle_worker(conn, bubble):
    """One process, one 128^3 oracle lattice (droplet or bubble); steps it on request."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import eos as E
    from oracle import lbm3d
    m = lbm3d.Model(tau=TAU, G=G, eos=E.EOS("one_minus_exp"))
    a, b = (RHO_G, RHO_L) if bubble else (RHO_L, RHO_G)
    f = lbm3d.init_from_density(lbm3d.drop_density((SIZE,) * 3, (SIZE // 2,) * 3, RADIUS, a, b))
    conn.send("ready")
    while True:
        k = conn.recv()
        if k is None:
            break
        for _ in range(k):
            f = lbm3d.step(f, m)
        conn.send(k)


class OraclePool:
    """Independent 128^3 oracle lattices, one per host core (spawned processes, so the
    pool is safe to start after CUDA is initialised); droplets and bubbles alternate."""

    def __init__(self, workers=None):
        import multiprocessing as mp
        cpu = host_cpu()
        n = workers or cpu["nproc"]
        avail = _mem_available_bytes()
        if avail:
            n = max(1, min(n, int(0.8 * avail // ORACLE_BYTES_PER_LATTICE)))
        self.cpu = cpu
        self.workers = n
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for k in range(n):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, k % 2 == 1), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            assert c.recv() == "ready"

    def step(self, k=1):
        """k LB steps on every lattice; returns when all are done."""
        for c in self.conns:
            c.send(k)
        for c in self.conns:
            c.recv()

    def close(self):
        for c in self.conns:
            try:
                c.send(None)
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=10)
            if p.is_alive():
                p.kill()


def bench_reference(args):
    """FP64 CPU oracle on the same workload and metric, on every host core: one 128^3
    lattice per core (droplets and bubbles alternating), one LB step of each per bench step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            pool.step(1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.step(1)
        dt = time.perf_counter() - t0
    finally:
        pool.close()
    lu = pool.workers * SIZE ** 3 * args.steps
    val = lu / dt / 1e6
    line = {
        "impl": "reference", "metric": "MLUPS", "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "reference_step": f"1 LB step of each of {pool.workers} 128^3 lattices (bounded sample)"},
        "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": pool.workers, "kind": "oracle",
                         "host": pool.cpu,
                         "sample": f"{args.steps} x (1 LB step of each of {pool.workers} independent 128^3 "
                                   f"lattices, one process per core), numpy FP64"},
        "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(seconds_target=12.0):
    """The oracle as it stands on every host core: one 128^3 lattice per core, whole LB
    steps of all of them until about 12 s have passed."""
    pool = OraclePool()
    try:
        pool.step(1)                      # first step outside the sample
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < seconds_target or n == 0:
            pool.step(1)
            n += 1
        dt = time.perf_counter() - t0
    finally:
        pool.close()
    return {"value": pool.workers * SIZE ** 3 * n / dt / 1e6, "unit": "MLUPS", "cores": pool.workers,
            "kind": "oracle", "host": pool.cpu,
            "sample": f"{n} LB steps of each of {pool.workers} independent 128^3 lattices "
                      f"(one process per core), numpy FP64"}


SWEEP_RADII = (18.0, 20.0, 22.0, 24.0)


def sweep_leg():
    """The sweep of Sec. IV in miniature: G = -5, droplets and bubbles of R in
    {18, 20, 22, 24} at L = 4R, from the GPU flat-interface coexistence to the Tolman
    fit; batched shifted-FP32 storage against one-lattice-at-a-time FP64, wall time
    of each (set-up, runs to convergence and observables included)."""
    from paper_2105_08772_gb300 import sweep as S
    runs = S.plan(couplings=(G,), radii=SWEEP_RADII, L_min=0, per_R=4.0)
    t0 = time.perf_counter()
    coex = S.coexistence((G,))
    t_flat = time.perf_counter() - t0
    ob, wall_b, lu_b = S.run_batched(runs, coex, slots=len(runs), prec="f32", max_steps=30_000)
    op, wall_p, lu_p = S.run_plain(runs, coex, prec="f64", max_steps=30_000)
    fb, fp = S.tolman(ob, coex), S.tolman(op, coex)
    fit = S.compare(fb, fp).get(G)
    return {"workload": f"G={G}, psi=1-exp(-n), droplets+bubbles R in {list(SWEEP_RADII)}, L=4R",
            "runs": len(runs), "usable_f32": sum(o.usable for o in ob),
            "usable_f64": sum(o.usable for o in op), "flat_interface_s": t_flat,
            "batched_f32_s": wall_b, "plain_f64_s": wall_p, "speedup": wall_p / wall_b,
            "batched_f32_MLUPS": lu_b / wall_b / 1e6, "plain_f64_MLUPS": lu_p / wall_p / 1e6,
            "delta_f64": fp[G].delta if G in fp else None,
            "sigma0_f64": fp[G].sigma0 if G in fp else None,
            "rel_diff": {**(fit or {}), **{k: v for k, v in S.compare_runs(ob, op).items() if k != "runs"}}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="f32", choices=["f64", "f32", "f16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-leg", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--no-sweep-leg", action="store_true")
    ap.add_argument("--no-large-leg", action="store_true")
    ap.add_argument("--kernel-only", action="store_true",
                    help="build one droplet lattice (128^3 unless --box), run two single steps and exit "
                         "(a small, fixed launch sequence for ncu captures)")
    ap.add_argument("--tile", type=int, default=0, help="tile code for --kernel-only (0: default)")
    ap.add_argument("--box", type=int, default=SIZE,
                    help="cubic box side for --kernel-only (odd sides take the element-copy kernel)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return bench_reference(args)

    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2105_08772_gb300 as P

    if args.kernel_only:
        L = args.box
        lat = P.Lattice(L, L, L, tau=TAU, G=G, psi="one_minus_exp", stencil="E4", prec=args.prec)
        lat.init_drop((L // 2,) * 3, RADIUS * L / SIZE, RHO_L, RHO_G)
        if args.tile:
            lat.set_tile(args.tile)
        lat.step(1)
        lat.step(1)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_only": True, "box": L, "tile": lat.get_tile(), "prec": args.prec}))
        return

    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    c = (SIZE // 2,) * 3

    def make(prec):
        with torch.cuda.stream(stream):
            lats = [P.Lattice(SIZE, SIZE, SIZE, tau=TAU, G=G, psi="one_minus_exp", stencil="E4",
                              prec=prec, stream=stream) for _ in range(2)]
        lats[0].init_drop(c, RADIUS, RHO_L, RHO_G)
        lats[1].init_drop(c, RADIUS, RHO_G, RHO_L)
        return lats

    lats = make(args.prec)
    if args.autotune:
        for lat in lats:
            lat.autotune(reps=8)
            lat.init_drop(c, RADIUS, RHO_L if lat is lats[0] else RHO_G, RHO_G if lat is lats[0] else RHO_L)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]

    def bench_step(record):
        kern_ms = 0.0
        for k, lat in enumerate(lats):
            if record:
                ev[k][0].record(stream)
            lat.step(LBM_STEPS_PER_STEP)
            if record:
                ev[k][1].record(stream)
            lat.observables()          # synchronises the stream
            if record:
                kern_ms += ev[k][0].elapsed_time(ev[k][1])
        return kern_ms

    for _ in range(args.warmup):
        bench_step(False)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    kern_ms = 0.0
    with ClockSampler(dev) as clk:
        t_start.record(stream)
        for _ in range(args.steps):
            kern_ms += bench_step(True)
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier()
    elapsed_ms = t_start.elapsed_time(t_end)
    if ws > 1:
        t = torch.tensor([elapsed_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    N = SIZE ** 3
    lu_rank = len(lats) * N * LBM_STEPS_PER_STEP * args.steps
    value = lu_rank * ws / (elapsed_ms * 1e-3) / 1e6
    launches_per_step = len(lats) * (LBM_STEPS_PER_STEP + 3)

    # roofline of the dominant kernel (the fused step): algorithmic bytes per launch over the
    # average launch time seen by CUDA events around the step-only part of the timed region
    peak, peak_kind = measured_peak_gbs()
    n_launch = len(lats) * LBM_STEPS_PER_STEP * args.steps
    avg_launch_s = kern_ms * 1e-3 / n_launch
    bytes_per_launch = BYTES_PER_LU[args.prec] * N
    achieved = bytes_per_launch / avg_launch_s / 1e9
    traffic = measured_traffic(args.prec, lats[0].get_tile() // 100000000)

    # end to end through the public API with host buffers
    host = []
    for lat in lats:
        pinned = torch.empty((SIZE, SIZE, SIZE), dtype=torch.float64, pin_memory=True)
        pinned.numpy()[...] = lat.rho()
        host.append(pinned)
    for k, lat in enumerate(lats):        # warm the host path once
        lat.init_rho(host[k].numpy())
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for k, lat in enumerate(lats):
            lat.init_rho(host[k].numpy())
            lat.step(LBM_STEPS_PER_STEP)
            lat.observables()
    e2e_s = time.perf_counter() - t0
    e2e_val = len(lats) * N * LBM_STEPS_PER_STEP * e2e_steps * ws / e2e_s / 1e6

    fp64 = None
    if not args.no_fp64_leg and args.prec != "f64":
        lat64 = make("f64")[0]
        lat64.step(LBM_STEPS_PER_STEP)
        lat64.observables()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        lat64.step(LBM_STEPS_PER_STEP)
        e1.record(stream)
        lat64.observables()
        ms = e0.elapsed_time(e1)
        fp64 = {"value": N * LBM_STEPS_PER_STEP / (ms * 1e-3) / 1e6, "unit": "MLUPS",
                "sample": "one 2048-step interval of the 128^3 droplet, FP64 storage and arithmetic",
                "hbm_gbs": BYTES_PER_LU["f64"] * N * LBM_STEPS_PER_STEP / (ms * 1e-3) / 1e9,
                **fp64_bound(BYTES_PER_LU["f64"] * N * LBM_STEPS_PER_STEP / (ms * 1e-3) / 1e9, peak)}

    # the same step kernel on a 256^3 lattice (4x the 128^3 working set): the
    # roofline fraction at a size well past L2
    large = None
    if not args.no_large_leg and args.prec != "f64":
        L = 256
        with torch.cuda.stream(stream):
            big = P.Lattice(L, L, L, tau=TAU, G=G, psi="one_minus_exp", stencil="E4", prec=args.prec,
                            stream=stream)
        big.init_drop((L // 2,) * 3, L / 4, RHO_L, RHO_G)
        big.step(256)
        big.observables()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_big = 1024
        torch.cuda.synchronize()
        e0.record(stream)
        big.step(n_big)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / n_big
        ach = BYTES_PER_LU[args.prec] * L ** 3 / (us * 1e-6) / 1e9
        large = {"box": L, "avg_launch_us": us, "MLUPS": L ** 3 / us, "achieved": ach, "unit": "GB/s",
                 "frac": ach / peak, "tile": big.get_tile(),
                 "sample": f"{n_big} steps of a 256^3 droplet (R=64), same kernel and storage"}
        big.close()

    sweep = None
    if not args.no_sweep_leg and ws == 1:
        sweep = sweep_leg()

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline or ws > 1 else cpu_baseline_sample()
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.prec != "f64" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "box": SIZE, "lattices_per_gpu": len(lats),
                   "storage": {"f32": "f32 shifted", "f16": "f16 shifted, 2^k scale", "f64": "f64"}[args.prec],
                   "lb_steps_per_step": LBM_STEPS_PER_STEP,
                   "l2": "inputs larger than L2: 2 lattices x 2 population buffers x 159 MB",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                     "kernel": kernel_name(lats[0].get_tile()), "tile": lats[0].get_tile(),
                     "bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_launch_s * 1e6},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": len(lats) * N * 8,
                "d2h_bytes_per_step": len(lats) * 152, "steps": e2e_steps},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
        "fp64": fp64,
        "roofline_256": large,
        "sweep": sweep,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
