"""The launch table: every choice it can hold (tensor cores with either tile
height and any swizzle width, integer pipes with any K split) gives the same
bits as the oracle, and mpc_autotune fills the table from measured times."""
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


def rows_of(rows, ring):
    return (32 if ring.words == 1 else 16) if rows == "wide" else rows


def operands(ring, M, K, N, seed):
    u = lambda t, shape: synth.uniform(seed, t, 1, shape, ring.bits)
    return u(1, (M, K)), u(2, (K, N)), u(3, (M, K)), u(4, (K, N)), u(5, (M, N))


CHOICES = [(1, 1, 0), (1, 4, 0), (1, 16, 0), (1, 64, 0), (0, 0, 1), (0, 0, 2), (0, 0, 8)]
# tensor cores ("wide": 128 columns x 32 rows, Z_2^64, or 16, Z_2^128; -128: the tall tile, whose
# left operand the GEMM converts itself)
TILE_ROWS = (128, 64, "wide", -128)
SIMT_ROWS = (0, 64, 16)        # integer pipes (0: chosen by grid size)


@pytest.mark.parametrize("ring,shape", [(synth.Z64, (300, 200, 96)), (synth.Z64, (1100, 64, 66)),
                                        (synth.Z128, (200, 130, 48)), (synth.Z64, (16, 4096, 512)),
                                        (synth.Z64, (1024, 27, 64)), (synth.Z128, (33, 27, 70))],
                         ids=lambda x: str(x) if isinstance(x, tuple) else None)
def test_every_choice_is_exact(ring, shape):
    M, K, N = shape
    E, F, A, B, C = operands(ring, M, K, N, sum(shape))
    want = O.linear_share(ring.bits, 0, E, F, A, B, C)
    L = abi.make_layer(M, K, N, ring.k, ring.s, 0, 2)
    for path, gm, waves in CHOICES:
        for rows in (TILE_ROWS if path else SIMT_ROWS):
            rows = rows_of(rows, ring)
            if rows == -128 and (K * ring.words) % 2:
                continue                    # the tall tile's 2-D loads need an even row stride
            abi.mpc_autotune_set(L, path, gm if path else 0, waves, tile_rows=rows)
            assert abi.mpc_gemm_path(L) == path
            assert abi.mpc_autotune_choice(L)[4] == rows
            Z = empty_like_ring((M, N), ring.words)
            abi.mpc_linear_share(L, dev(E), dev(F), dev(A), dev(B), dev(C), Z)
            assert np.array_equal(host(Z), want), (path, rows, gm, waves)
    abi.mpc_autotune_clear()
    assert abi.mpc_device_status() == 0


# ragged heights around both tile heights (M <= 8 runs on the integer pipes
# only), ragged K (one partial 16-deep stage; a K below one stage) and N
@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=["w1", "w2"])
@pytest.mark.parametrize("M", [9, 15, 16, 17, 31, 32, 33, 63, 64, 65, 130, 300])
def test_every_tile_is_exact(ring, M):
    for K, N in ((27, 34), (300, 96), (5, 66), (40, 258)):
        E, F, A, B, C = operands(ring, M, K, N, 1000 * M + K)
        mA, mB, mC = operands(ring, M, K, N, 2000 * M + K)[2:]
        alpha = synth.uniform(M, 9, 0, (1,), ring.bits)
        want_z = O.linear_share(ring.bits, 0, E, F, A, B, C)
        want_t = O.linear_tag_full(ring.bits, alpha, E, F, mA, mB, mC)
        L = abi.make_layer(M, K, N, ring.k, ring.s, 0, 2)
        for rows in TILE_ROWS:
            rows = rows_of(rows, ring)
            if rows == -128 and (K * ring.words) % 2:
                with pytest.raises(abi.MpcError):
                    abi.mpc_autotune_set(L, 1, 8, 0, tile_rows=rows)
                continue
            for gm in (1, 8):
                abi.mpc_autotune_set(L, 1, gm, 0, tile_rows=rows)
                Z = empty_like_ring((M, N), ring.words)
                abi.mpc_linear_share(L, dev(E), dev(F), dev(A), dev(B), dev(C), Z)
                assert np.array_equal(host(Z), want_z), (M, K, N, rows, gm)
                mZ = empty_like_ring((M, N), ring.words)
                abi.mpc_linear_tag(L, abi.MPC_TAG_FULL, dev(alpha), dev(E), dev(F), dev(mA), dev(mB), dev(mC), mZ)
                assert np.array_equal(host(mZ), want_t), (M, K, N, rows, gm, "tag")
        abi.mpc_autotune_clear()
    assert abi.mpc_device_status() == 0


def test_built_in_rule_takes_short_tiles_for_short_layers():
    abi.mpc_autotune_clear()
    assert abi.mpc_autotune_choice(abi.make_layer(64, 4608, 512))[::4] == (1, 32)        # wide
    assert abi.mpc_autotune_choice(abi.make_layer(65, 4608, 512))[::4] == (1, 128)
    assert abi.mpc_autotune_choice(abi.make_layer(16, 2304, 512, 64, 64))[::4] == (1, 16)
    assert abi.mpc_autotune_choice(abi.make_layer(40, 2304, 512, 64, 64))[::4] == (1, 16)    # wide: 864 units
    assert abi.mpc_autotune_choice(abi.make_layer(64, 576, 128, 64, 64))[::4] == (1, 64)     # wide: 72 units
    assert abi.mpc_autotune_choice(abi.make_layer(64, 2304, 256))[::4] == (1, 32)            # Z_2^64: wide to 64
    assert abi.mpc_autotune_choice(abi.make_layer(32768, 576, 64))[::4] == (1, -128)           # tall
    assert abi.mpc_autotune_choice(abi.make_layer(2048, 576, 64))[::4] == (1, -128)
    assert abi.mpc_autotune_choice(abi.make_layer(1024, 576, 64))[::4] == (1, 128)    # Z_2^64 tall from 2048 rows
    assert abi.mpc_autotune_choice(abi.make_layer(32768, 576, 64, 64, 64))[::4] == (1, -128)   # Z_2^128 tall
    assert abi.mpc_autotune_choice(abi.make_layer(1024, 576, 64, 64, 64))[::4] == (1, -128)
    assert abi.mpc_autotune_choice(abi.make_layer(512, 576, 64, 64, 64))[::4] == (1, 128)
    assert abi.mpc_autotune_choice(abi.make_layer(32768, 1152, 128, 64, 64))[::4] == (1, -128)  # N <= 128
    assert abi.mpc_autotune_choice(abi.make_layer(2048, 1152, 128, 64, 64))[::4] == (1, 128)    # from 4096 rows
    assert abi.mpc_autotune_choice(abi.make_layer(8192, 2304, 256, 64, 64))[::4] == (1, 128)    # N > 128
    assert abi.mpc_autotune_choice(abi.make_layer(1024, 27, 64))[::4] == (0, 0)                 # small: SIMT
    assert abi.mpc_autotune_choice(abi.make_layer(4096, 575, 64))[::4] == (1, 128)   # odd K: not tall


@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=["w1", "w2"])
def test_grouped_with_mixed_choices(ring):
    """One grouped call over layers with 128-row tiles, 64-row tiles and the
    integer pipes (the tensor-core layers of each tile height share a
    persistent launch)."""
    shapes = [(300, 200, 96), (1100, 64, 66), (64, 256, 256), (520, 128, 130), (40, 300, 96), (17, 1000, 34),
              (64, 27, 64), (130, 600, 66), (12, 700, 300), (100, 64, 130), (33, 1500, 258), (1300, 576, 64),
              (257, 40, 34), (200, 130, 300)]
    choices = [(1, 1, 0, 128), (0, 0, 4, 16), (1, 16, 0, 64), (1, 4, 0, 128), (1, 8, 0, 64), (1, 1, 0, 64),
               (1, 8, 0, 128), (0, 0, 2, 64), (1, 8, 0, "wide"), (1, 1, 0, "wide"), (1, 4, 0, "wide"),
               (1, 8, 0, -128), (1, 1, 0, -128), (1, 4, 0, -128)]
    choices = [(p_, g_, w_, rows_of(r_, ring)) for p_, g_, w_, r_ in choices]
    layers = [abi.make_layer(M, K, N, ring.k, ring.s) for M, K, N in shapes]
    for L, (path, gm, waves, rows) in zip(layers, choices):
        abi.mpc_autotune_set(L, path, gm, waves, tile_rows=rows)
    data = [operands(ring, M, K, N, 7 * M + K) for M, K, N in shapes]
    Zs = [empty_like_ring((M, N), ring.words) for M, K, N in shapes]
    abi.mpc_linear_share_grouped(layers, [dict(E=dev(E), F=dev(F), A_i=dev(A), B_i=dev(B), C_i=dev(C), Z_i=Z)
                                          for (E, F, A, B, C), Z in zip(data, Zs)])
    for (E, F, A, B, C), Z, sh in zip(data, Zs, shapes):
        assert np.array_equal(host(Z), O.linear_share(ring.bits, 0, E, F, A, B, C)), sh
    abi.mpc_autotune_clear()
    assert abi.mpc_device_status() == 0


def test_autotune_fills_the_table(tmp_path):
    abi.mpc_autotune_clear()
    layers = [abi.make_layer(M, K, N) for M, K, N in [(1024, 576, 64), (128, 1024, 1024), (4, 512, 512),
                                                        (1024, 576, 64), (32, 4608, 512)]]
    assert abi.mpc_autotune(layers) == 4
    for L in layers:
        path, gm, waves, tuned, rows = abi.mpc_autotune_choice(L)
        assert tuned
        assert path in (0, 1)
        assert rows in ((0, 16, 64) if path == 0 else (128, 64, 32, -128))
    assert abi.mpc_autotune_choice(layers[2])[0] == 0      # M <= 8: integer pipes only
    f = tmp_path / "t.txt"
    assert abi.mpc_autotune_save(str(f)) == 4
    saved = {tuple(abi.mpc_autotune_choice(L)) for L in layers}
    abi.mpc_autotune_clear()
    assert abi.mpc_autotune_load(str(f)) == 4
    assert {tuple(abi.mpc_autotune_choice(L)) for L in layers} == saved
    abi.mpc_autotune_clear()
