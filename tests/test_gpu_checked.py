"""The bounds-checked build (nvcc -DUWB_CHECK), the library's stand-in for a
memory checker: every staged-window run, image index and compact-profile index
the image kernels compute is checked, and one outside its buffer records
UWB_ERR_BOUNDS (in the device status word, which the `gpu` fixture requires
clear after each module, or in every result record of a localisation, whose
status the parity comparison requires equal to the oracle's).

The image, localisation, tiling and progressive suites run once more here, in
a child process with UWB_LIBRARY=checked: the images, decisions and locations
must match the oracle as before, and no index may leave its buffer."""
import os
import pathlib
import re
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = pathlib.Path(__file__).resolve().parent.parent
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_ragged.py", "tests/test_gpu_progressive.py",
          "tests/test_gpu_balance.py"]


def test_checked_build_passes_the_image_suites_without_a_bounds_error():
    from paper_1709_02549_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, UWB_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-m", "pytest", *SUITES, "-m", "gpu", "-x", "-q",
                        "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = r.stdout[-4000:] + r.stderr[-2000:]
    assert r.returncode == 0, tail
    m = re.search(r"(\d+) passed", r.stdout)
    assert m and int(m.group(1)) >= 100 and " failed" not in r.stdout, tail
