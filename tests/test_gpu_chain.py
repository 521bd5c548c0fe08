"""Calls chained on one stream, each reading the previous call's output.

Within a call the GEMM starts as a programmatic dependent of its prologue, and
the first kernel of every call is a dependent of the kernel before it, so each
kernel must wait for its predecessor before touching memory.  Here the output
Z of one share call is the addend C of the next and the left operand E of the
one after, with no host synchronisation in between (the first layer is large,
so its GEMM is still running while the next calls are enqueued); every result
must equal the oracle's chain bit for bit.
"""
import numpy as np
import pytest

import oracle as O
import synth
from paper_2311_04406_gb300 import abi, build

from gpuhelp import dev, empty_like_ring, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    abi.load()


def _rand(rng, ring, *shape):
    full = tuple(shape) + ((2,) if ring.words == 2 else ())
    return rng.integers(0, 2**64, size=full, dtype=np.uint64)


@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=["z64", "z128"])
def test_chained_share_calls(ring):
    rng = np.random.default_rng(2311 + ring.words)
    bits = 64 * ring.words
    M, K1, N = 1024, 1024, 256        # the longest call first
    K2, N3 = 384, 96
    layers = [abi.make_layer(M, K1, N, ring.k, ring.s, 0, 2), abi.make_layer(M, K2, N, ring.k, ring.s, 1, 2),
              abi.make_layer(M, N, N3, ring.k, ring.s, 0, 2)]
    assert [abi.mpc_gemm_path(L) for L in layers] == [1, 1, 1], "all three calls take the tensor-core path"
    E1, F1, A1, B1, C1 = (_rand(rng, ring, M, K1), _rand(rng, ring, K1, N), _rand(rng, ring, M, K1),
                          _rand(rng, ring, K1, N), _rand(rng, ring, M, N))
    E2, F2, A2, B2 = _rand(rng, ring, M, K2), _rand(rng, ring, K2, N), _rand(rng, ring, M, K2), _rand(rng, ring, K2, N)
    F3, A3, B3, C3 = _rand(rng, ring, N, N3), _rand(rng, ring, M, N), _rand(rng, ring, N, N3), _rand(rng, ring, M, N3)

    # device: Z1 -> C of call 2 -> Z2 -> E of call 3, one stream, no synchronisation
    Z1, Z2, Z3 = empty_like_ring((M, N), ring.words), empty_like_ring((M, N), ring.words), \
        empty_like_ring((M, N3), ring.words)
    d = {k: dev(v) for k, v in dict(E1=E1, F1=F1, A1=A1, B1=B1, C1=C1, E2=E2, F2=F2, A2=A2, B2=B2,
                                    F3=F3, A3=A3, B3=B3, C3=C3).items()}
    abi.mpc_linear_share(layers[0], d["E1"], d["F1"], d["A1"], d["B1"], d["C1"], Z1)
    abi.mpc_linear_share(layers[1], d["E2"], d["F2"], d["A2"], d["B2"], Z1, Z2)
    abi.mpc_linear_share(layers[2], Z2, d["F3"], d["A3"], d["B3"], d["C3"], Z3)

    z1 = O.linear_share(bits, 0, E1, F1, A1, B1, C1)
    z2 = O.linear_share(bits, 1, E2, F2, A2, B2, z1)
    z3 = O.linear_share(bits, 0, z2, F3, A3, B3, C3)
    assert np.array_equal(host(Z1), z1)
    assert np.array_equal(host(Z2), z2)
    assert np.array_equal(host(Z3), z3)
    assert abi.mpc_device_status() == 0
