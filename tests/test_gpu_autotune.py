"""The launch table: every choice it can hold (tensor cores with any swizzle
width, integer pipes with any K split) gives the same bits as the oracle, and
mpc_autotune fills the table from measured times."""
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
    abi.mpc_autotune_clear()
    yield
    abi.mpc_autotune_clear()


def operands(ring, M, K, N, seed):
    u = lambda t, shape: synth.uniform(seed, t, 1, shape, ring.bits)
    return u(1, (M, K)), u(2, (K, N)), u(3, (M, K)), u(4, (K, N)), u(5, (M, N))


CHOICES = [(1, 1, 0), (1, 4, 0), (1, 16, 0), (1, 64, 0), (0, 0, 1), (0, 0, 2), (0, 0, 8)]


@pytest.mark.parametrize("ring,shape", [(synth.Z64, (300, 200, 96)), (synth.Z64, (1100, 64, 66)),
                                        (synth.Z128, (200, 130, 48)), (synth.Z64, (16, 4096, 512))],
                         ids=lambda x: str(x) if isinstance(x, tuple) else None)
def test_every_choice_is_exact(ring, shape):
    M, K, N = shape
    E, F, A, B, C = operands(ring, M, K, N, sum(shape))
    want = O.linear_share(ring.bits, 0, E, F, A, B, C)
    L = abi.make_layer(M, K, N, ring.k, ring.s, 0, 2)
    for path, gm, waves in CHOICES:
        abi.mpc_autotune_set(L, path, gm if path else 0, waves)
        assert abi.mpc_gemm_path(L) == path
        Z = empty_like_ring((M, N), ring.words)
        abi.mpc_linear_share(L, dev(E), dev(F), dev(A), dev(B), dev(C), Z)
        assert np.array_equal(host(Z), want), (path, gm, waves)
    abi.mpc_autotune_clear()
    assert abi.mpc_device_status() == 0


def test_grouped_with_mixed_choices():
    ring = synth.Z64
    shapes = [(300, 200, 96), (1100, 64, 66), (64, 256, 256), (520, 128, 130)]
    layers = [abi.make_layer(M, K, N) for M, K, N in shapes]
    for L, (path, gm, waves) in zip(layers, [(1, 1, 0), (0, 0, 4), (1, 16, 0), (1, 4, 0)]):
        abi.mpc_autotune_set(L, path, gm, waves)
    data = [operands(ring, M, K, N, 7 * M + K) for M, K, N in shapes]
    Zs = [empty_like_ring((M, N), 1) for M, K, N in shapes]
    abi.mpc_linear_share_grouped(layers, [dict(E=dev(E), F=dev(F), A_i=dev(A), B_i=dev(B), C_i=dev(C), Z_i=Z)
                                          for (E, F, A, B, C), Z in zip(data, Zs)])
    for (E, F, A, B, C), Z in zip(data, Zs):
        assert np.array_equal(host(Z), O.linear_share(64, 0, E, F, A, B, C))
    abi.mpc_autotune_clear()


def test_autotune_fills_the_table(tmp_path):
    abi.mpc_autotune_clear()
    layers = [abi.make_layer(M, K, N) for M, K, N in [(1024, 576, 64), (128, 1024, 1024), (4, 512, 512),
                                                        (1024, 576, 64)]]
    assert abi.mpc_autotune(layers) == 3
    for L in layers:
        path, gm, waves, tuned = abi.mpc_autotune_choice(L)
        assert tuned
        assert path in (0, 1)
    assert abi.mpc_autotune_choice(layers[2])[0] == 0      # M <= 8: integer pipes only
    f = tmp_path / "t.txt"
    assert abi.mpc_autotune_save(str(f)) == 3
    abi.mpc_autotune_clear()
    assert abi.mpc_autotune_load(str(f)) == 3
    abi.mpc_autotune_clear()
