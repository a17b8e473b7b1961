"""bench.py's host-side contract, without a GPU: the oracle arm's JSON line and
the lookup of the committed ncu traffic figure."""
import importlib.util
import json
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_under_test", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "MLUPS" and d["unit"] == "MLUPS"
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("two 128^3 periodic lattices")


def test_traffic_lookup_follows_the_source_hash(tmp_path, monkeypatch):
    b = _bench_module()
    csrc = tmp_path / "paper_2105_08772_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in b.KERNEL_SOURCES:
        (csrc / f).write_text(f"// {f}\n")
    import hashlib
    h = hashlib.sha256(b"".join((csrc / f).read_bytes() for f in b.KERNEL_SOURCES)).hexdigest()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "lattice_moment_f32_128.md").write_text(
        f"# summary\n\n| a | b |\n\ntraffic_bytes_per_launch: 1234\nsource_sha256: {h}\n")
    monkeypatch.setattr(b, "ROOT", tmp_path)
    assert b.measured_traffic("f32") == 1234
    assert b.measured_traffic("f16") is None                  # no summary for this storage
    (csrc / b.KERNEL_SOURCES[0]).write_text("// changed\n")
    assert b.measured_traffic("f32") is None                  # kernel changed since the capture


def test_fp64_bound_is_measured_or_null(tmp_path, monkeypatch):
    """The FP64 leg's bound comes from this run's DRAM fraction and, only when the
    FP64 summary was captured on the current sources, its FP64-pipe figure."""
    b = _bench_module()
    csrc = tmp_path / "paper_2105_08772_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in b.KERNEL_SOURCES:
        (csrc / f).write_text(f"// {f}\n")
    import hashlib
    h = hashlib.sha256(b"".join((csrc / f).read_bytes() for f in b.KERNEL_SOURCES)).hexdigest()
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(b, "ROOT", tmp_path)
    r = b.fp64_bound(500.0, 6800.0)
    assert r["bound"] is None and "ncu" not in r["evidence"]          # no summary
    assert abs(r["hbm_frac"] - 500.0 / 6800.0) < 1e-15
    (prof / "lattice_moment_f64_128.md").write_text(
        f"# summary\n\nfp64_pipe_pct: 81.1\nsource_sha256: {h}\n")
    r = b.fp64_bound(500.0, 6800.0)
    assert r["bound"] == "alu" and "81.1" in r["evidence"] and "lattice_moment_f64_128.md" in r["evidence"]
    (csrc / b.KERNEL_SOURCES[1]).write_text("// changed\n")
    assert b.fp64_bound(500.0, 6800.0)["bound"] is None                # stale summary
