"""Oracle runs that take minutes (1000 steps of 41^3 and 64^3 boxes), started in
spawned worker processes when the GPU parity tests that need them are
selected, so they run on the host cores while earlier GPU tests run.

Each job returns the oracle's density field after its steps; the workloads
follow Sec. IV (a tanh droplet of Eq. (23) at the flat-interface densities,
fluid at rest)."""
from __future__ import annotations

import numpy as np

# flat-interface coexistence densities of psi = 1 - exp(-n) at G = -5 (oracle flat run)
N_L, N_G = 1.8883, 0.1193

JOBS = {
    # name: (box side, radius, steps)
    "droplet64": (64, 16.0, 1000),
    "droplet41": (41, 10.25, 1000),
}


def centre(L: int) -> int:
    return L // 2


def run_job(name: str) -> np.ndarray:
    from oracle import eos as E
    from oracle import lbm3d
    L, R, steps = JOBS[name]
    c = centre(L)
    n = lbm3d.drop_density((L, L, L), (c, c, c), R, N_L, N_G)
    f = lbm3d.init_from_density(n)
    m = lbm3d.Model(tau=1.0, G=-5.0, eos=E.EOS("one_minus_exp"), stencil="E4")
    f = lbm3d.run(f, m, steps)
    return lbm3d.density(f)


_POOL = None
_FUT = {}


def start(names) -> None:
    """Submit the named jobs to a spawn-started pool (idempotent)."""
    global _POOL
    import concurrent.futures as cf
    import multiprocessing as mp
    names = [n for n in names if n not in _FUT]
    if not names:
        return
    if _POOL is None:
        _POOL = cf.ProcessPoolExecutor(max_workers=len(JOBS), mp_context=mp.get_context("spawn"))
    for n in names:
        _FUT[n] = _POOL.submit(run_job, n)


def result(name: str) -> np.ndarray:
    start([name])
    return _FUT[name].result()


def shutdown() -> None:
    global _POOL
    if _POOL is not None:
        _POOL.shutdown(wait=False, cancel_futures=True)
        _POOL = None
