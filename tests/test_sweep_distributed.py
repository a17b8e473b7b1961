"""The sweep spread over ranks (one process per GPU): sharding and the gathering of
outcomes, run as two gloo processes on the CPU with stand-in outcomes (no GPU).
The lattices of a sweep are independent, so ranks exchange nothing while they run;
the only collectives are the final gathers of small Python objects."""
import os
import socket

import pytest

S = pytest.importorskip("paper_2105_08772_gb300.sweep")
torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fake_outcome(run):
    """A converged-looking outcome whose sigma_s follows Eq. (22) exactly."""
    x = (-1.0 if run.bubble else 1.0) / run.R
    ss = 0.0363 * (1 - 2 * 0.57 * x + 1.3 * x * x)
    dh = 0.41 - 2.0 * x
    Re = run.R + (-dh if run.bubble else dh)
    return S.Outcome(run, 0, {"R_s": run.R, "sigma_s": ss, "R_e": Re, "status_bits": 0, "com": [0.0] * 3})


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        runs = S.plan(couplings=(-5.0, -5.5), radii=(8.0, 12.0, 16.0, 20.0, 24.0))
        mine = S.shard(runs, rank, world)
        local = [_fake_outcome(r) for r in mine]
        allo = S.gather_outcomes(local)
        wall = S.max_over_ranks(1.0 + rank)
        counts = S.gather_outcomes_counts(100 * (rank + 1))
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            keys = sorted((o.run.G, o.run.bubble, o.run.R) for o in allo)
            full = sorted((r.G, r.bubble, r.R) for r in runs)
            fit_all = S.tolman(allo)
            fit_ref = S.tolman([_fake_outcome(r) for r in runs])
            ok = (keys == full and len(allo) == len(runs) and wall == float(world)
                  and counts == [100 * (k + 1) for k in range(world)]
                  and all(abs(fit_all[G].delta - fit_ref[G].delta) < 1e-12 for G in fit_ref))
            f.write("ok" if ok else f"bad {len(allo)} {wall} {counts}")
    finally:
        dist.destroy_process_group()


def test_shard_partitions_the_plan():
    runs = S.plan()
    parts = [S.shard(runs, r, 3) for r in range(3)]
    assert sum(len(p) for p in parts) == len(runs)
    assert sorted(map(id, sum(parts, []))) == sorted(map(id, runs))
    # largest-first round robin: the box volumes per rank are within one box of each other
    vols = [sum(r.L ** 3 for r in p) for p in parts]
    assert max(vols) - min(vols) <= max(r.L ** 3 for r in runs)
    with pytest.raises(ValueError):
        S.shard(runs, 3, 3)


def test_two_gloo_ranks_gather_every_outcome(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    for r in range(world):
        assert (tmp_path / f"rank{r}.txt").read_text() == "ok"
