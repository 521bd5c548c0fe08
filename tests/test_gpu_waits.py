"""Failure detection on the GPU without a fault: a bounded device-side wait on
a barrier that nothing arrives at gives up after its limit, the kernel
returns, the host reads the timeout status, and the context stays usable
(a tensor-core layer afterwards is still bit-exact)."""
import numpy as np
import pytest

import oracle as O
import synth
from paper_2311_04406_gb300 import abi, build

from gpuhelp import gpu_share

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    abi.load()


def test_bounded_wait_gives_up_and_context_survives():
    import time
    assert abi.mpc_device_status() == 0
    t0 = time.perf_counter()
    assert abi.mpc_selftest_wait(2_000_000) == abi.MPC_E_TIMEOUT      # about 1 ms of waiting
    assert time.perf_counter() - t0 < 30.0
    assert abi.mpc_device_status() == abi.MPC_E_TIMEOUT              # the flag the GEMM roles set
    assert abi.mpc_device_status() == 0                              # read and cleared
    ring = synth.Z64
    M, K, N = 130, 256, 64
    u = lambda t, shape: synth.uniform(3, t, 0, shape, 64)
    E, F, A, B, C = u(1, (M, K)), u(2, (K, N)), u(3, (M, K)), u(4, (K, N)), u(5, (M, N))
    assert abi.mpc_gemm_path(abi.make_layer(M, K, N)) == 1
    Z = gpu_share(ring, 0, E, F, A, B, C)
    assert np.array_equal(Z, O.linear_share(64, 0, E, F, A, B, C))
    assert abi.mpc_device_status() == 0


def test_selftest_rejects_bad_limits():
    assert abi.mpc_selftest_wait(10) == abi.MPC_E_SHAPE
    assert abi.mpc_selftest_wait(10**11) == abi.MPC_E_SHAPE
