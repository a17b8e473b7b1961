"""Register and spill budget of the default step kernels, from ptxas's own
report (-Xptxas -v) of the FP32 and FP16 translation units compiled with the
build's flags.  Occupancy is what the moment kernels are designed around:
  * kind 5, 32 x 8, depth 1: three 256-thread CTAs per SM need <= 85
    registers a thread (65536 / 768);
  * kind 5 depth 2 and kind 6 (element copies): two CTAs per SM, <= 128;
  * kind 7 (TMA tensor-tile copies), 32 x 8: three CTAs per SM, <= 85;
  * FP16 kind 5, 32 x 8, depth 1: four CTAs per SM, <= 64;
and none of them may spill or keep a local-memory stack frame (a run-time index
into a constant table would put the table there).  A change that breaks a budget
shows up here, on the CPU, before any GPU measurement.
"""
import importlib.util
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
PKG = ROOT / "paper_2105_08772_gb300"

ENTRY = re.compile(r"Compiling entry function '(\S+)'")
USED = re.compile(r"Used (\d+) registers")
SPILL = re.compile(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads")
# lattice_moment_kernel<P, ST, BX, BY, D, ELEM> / lattice_moment_batch_kernel<...>, mangled
MOMENT = re.compile(r"(lattice_moment_kernel|lattice_moment_batch_kernel)"
                    r"ILi(\d+)ELi(\d+)ELi(\d+)ELi(\d+)ELi(\d+)ELb([01])E")
# lattice_tma_kernel<ST, BX, BY>
TMA = re.compile(r"(lattice_tma_kernel)ILi(\d+)ELi(\d+)ELi(\d+)EE")


def _build_module():
    spec = importlib.util.spec_from_file_location("_lbm_build_for_ptxas", PKG / "build.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def moment_kernels(tmp_path_factory):
    b = _build_module()
    try:
        nvcc = b.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    from concurrent.futures import ThreadPoolExecutor
    tmp = tmp_path_factory.mktemp("ptxas")

    def compile_tu(name):
        cmd = [nvcc, *b.ARCH, *b.NVCC_FLAGS, "-Xptxas", "-v", "-c", str(PKG / "csrc" / f"{name}.cu"),
               "-o", str(tmp / f"{name}.o")]
        return subprocess.run(cmd, capture_output=True, text=True, timeout=900)

    with ThreadPoolExecutor(2) as ex:
        rs = list(ex.map(compile_tu, ["lbm_lattice_f32", "lbm_lattice_f16"]))
    for r in rs:
        assert r.returncode == 0, r.stderr[-2000:]
    out, cur, spill = {}, None, (0, 0, 0)
    for line in "\n".join(r.stdout + r.stderr for r in rs).splitlines():
        m = ENTRY.search(line)
        if m:
            cur, spill = m.group(1), (0, 0, 0)
            continue
        m = SPILL.search(line)
        if cur and m:
            spill = (int(m.group(1)), int(m.group(2)), int(m.group(3)))
        m = USED.search(line)
        if cur and m:
            k = MOMENT.search(cur) or TMA.search(cur)
            if k:
                key = (k.group(1),) + tuple(int(v) for v in k.groups()[1:])
                out[key] = (int(m.group(1)), spill)
            cur = None
    assert out, "no moment kernels found in the ptxas report"
    return out


def test_moment_kernels_do_not_spill(moment_kernels):
    bad = {k: v for k, v in moment_kernels.items() if v[1] != (0, 0, 0)}
    assert not bad, bad


@pytest.mark.parametrize("key,limit", [
    (("lattice_moment_kernel", 1, 4, 32, 8, 1, 0), 85),        # kind 5, 3 CTAs/SM
    (("lattice_moment_batch_kernel", 1, 4, 32, 8, 1, 0), 85),
    (("lattice_moment_kernel", 1, 4, 32, 8, 2, 0), 128),       # kind 5 depth 2, 2 CTAs/SM
    (("lattice_moment_kernel", 1, 4, 32, 8, 1, 1), 128),       # kind 6, 2 CTAs/SM
    (("lattice_moment_batch_kernel", 1, 4, 32, 8, 1, 1), 128),
    (("lattice_tma_kernel", 4, 32, 8), 85),                    # kind 7, 3 CTAs/SM
    (("lattice_moment_kernel", 2, 4, 32, 8, 1, 0), 64),        # FP16 kind 5, 4 CTAs/SM
    (("lattice_moment_batch_kernel", 2, 4, 32, 8, 1, 0), 64),
])
def test_register_budget_for_the_designed_occupancy(moment_kernels, key, limit):
    assert key in moment_kernels, sorted(moment_kernels)
    regs = moment_kernels[key][0]
    assert regs <= limit, (key, regs, limit)
