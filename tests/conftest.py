import pathlib
import sys

ROOT = pathlib.Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

GOLDEN = ROOT / "tests" / "golden"


import pytest


@pytest.fixture(scope="session")
def uwb():
    """The CUDA library's Python binding, built in-tree if needed (nvcc
    cross-compiles without a GPU)."""
    from paper_1709_02549_gb300 import build
    try:
        build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(f"libuwb.so cannot be built here: {e}")
    import paper_1709_02549_gb300 as u
    return u


@pytest.fixture(scope="module")
def gpu(uwb):
    """The binding on a CUDA device; the device status word must stay clear."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    uwb.uwb_device_status(clear=True)
    yield uwb
    assert uwb.uwb_device_status(clear=True) == 0


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def read_golden(name: str) -> dict:
    """Parse a 'key value...' text fixture; '#' starts a comment."""
    out = {}
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, *vals = line.split()
        out[key] = vals
    return out
