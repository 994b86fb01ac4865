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
    cross-compiles without a GPU); with UWB_LIBRARY=checked, the bounds-checked
    build."""
    import os
    from paper_1709_02549_gb300 import build
    try:
        build.build(checked=os.environ.get("UWB_LIBRARY") == "checked")
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


@pytest.fixture(autouse=True)
def _parity_tally_name(request):
    """Files the oracle comparisons of each test under its node id."""
    mod = sys.modules.get("parity")
    if mod is not None:
        mod.CURRENT_TEST = request.node.nodeid
    yield


def pytest_terminal_summary(terminalreporter):
    """Per test: scans whose localisation was compared with the oracle, and the
    near-ties among them (a child choice, a stop test or an argmax within the
    1e-4 margin, where the oracle was replayed along the GPU's trajectory)."""
    mod = sys.modules.get("parity")
    if mod is None or not mod.TIE_LOG:
        return
    tr = terminalreporter
    tr.section("oracle comparisons of localisations (near-ties resolved by replay)")
    total = {}
    for node, c in sorted(mod.TIE_LOG.items()):
        tr.write_line(f"{node}: {c['scans']} scans, near-ties child {c['child']} "
                      f"stop {c['stop']} argmax {c['argmax']}, replayed {c['replayed']}")
        for k, v in c.items():
            total[k] = total.get(k, 0) + v
    tr.write_line(f"total: {total.get('scans', 0)} scans, near-ties child "
                  f"{total.get('child', 0)} stop {total.get('stop', 0)} argmax "
                  f"{total.get('argmax', 0)}, replayed {total.get('replayed', 0)}")


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
