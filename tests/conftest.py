import json
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
for p in (str(ROOT), str(ROOT / "tests")):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the liblbm.so kernels)")
    config.addinivalue_line("markers", "long_oracle(*names): uses the background oracle runs of tests/long_oracle.py")


@pytest.fixture(scope="session")
def paper():
    return json.loads((ROOT / "tests" / "golden" / "paper_constants.json").read_text())


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_collection_finish(session):
    """Start the minutes-long oracle runs in the background as soon as the tests
    that need them are known to run on a GPU."""
    need = set()
    for it in session.items:
        if "gpu" in it.keywords and not it.get_closest_marker("skip"):
            for m in it.iter_markers("long_oracle"):
                need.update(m.args)
    if need:
        import long_oracle
        long_oracle.start(sorted(need))


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get("long_oracle")
    if mod is not None:
        mod.shutdown()
