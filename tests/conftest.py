import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Set in the child process that runs a `hidden_gpu` test.
_CHILD = "MPCL_TEST_GPU_HIDDEN"


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    config.addinivalue_line(
        "markers",
        "hidden_gpu: passes placeholder device addresses that host-side validation must reject; "
        "the test body runs in a child process that sees no GPU, so a validation regression "
        "cannot launch a kernel on them")


def pytest_pyfunc_call(pyfuncitem):
    """Run `hidden_gpu` tests in a child pytest with CUDA_VISIBLE_DEVICES=''.

    A call that wrongly got past validation then fails with a CUDA error in
    the child instead of launching on an invalid address."""
    if pyfuncitem.get_closest_marker("hidden_gpu") is None or os.environ.get(_CHILD) == "1":
        return None
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", **{_CHILD: "1"})
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "-m", "gpu or not gpu", pyfuncitem.nodeid],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, f"child run of {pyfuncitem.nodeid} failed:\n{r.stdout[-4000:]}\n{r.stderr[-2000:]}"
    return True
