"""The index-checked build (needs a GB300).

libpic_checked.so is the library compiled with PIC_CHECKED: every shared-
memory window index of the push and charge kernels and every slot index of
the sort is checked on the device; a failed check skips the access and sets
an error bit that the next synchronising call turns into PIC_EOVERFLOW.
Running the GPU parity suites against it, in a child process with
PIC_LIBRARY=checked, shows no index leaves its buffer on those cases.  (It
stands in for a memory checker, which this toolchain's GPUs do not offer.)
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suites_under_the_checked_build():
    from paper_1503_02464_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, PIC_LIBRARY="checked")
    suites = ["tests/test_parity_gpu.py", "tests/test_boundary_gpu.py", "tests/test_variants_gpu.py",
              "tests/test_twostream_gpu.py", "tests/test_output_gpu.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"] + suites,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout


def test_checked_library_is_the_one_loaded():
    code = ("import os; from paper_1503_02464_gb300 import capi; capi.load(); "
            "print(os.path.basename(capi.library_path()))")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=dict(os.environ, PIC_LIBRARY="checked"),
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "libpic_checked.so"
