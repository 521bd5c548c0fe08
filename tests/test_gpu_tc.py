"""Parity of the tensor-core ring GEMM (fp16 digit products on tcgen05).

Shapes are chosen above the library's tensor-core threshold so that the
tcgen05 kernel runs (checked with mpc_gemm_path): ragged row and column tiles,
split-K plans and single-pass plans, the share (c = 0 and c = 1) and the full
tag (c = alpha), and digit patterns at the ends of the signed range -- all
digits -128 makes every accumulator reach exactly 2^24, the bound the exact
fp32 accumulation relies on.  Results must equal the oracle bit for bit.
"""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import dealer
from paper_2311_04406_gb300 import abi, build

from gpuhelp import gpu_share, gpu_tag_full

pytestmark = pytest.mark.gpu

SHAPES = [(130, 256, 70), (300, 640, 96), (128, 32, 1024), (500, 96, 1000), (9, 4096, 512),
          (257, 1024, 34)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    abi.load()


def _path(M, K, N, k=32, s=32):
    return abi.mpc_gemm_path(abi.make_layer(M, K, N, k, s))


@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_tc_path_parity(shape):
    M, K, N = shape
    assert _path(M, K, N) == 1, "shape should take the tensor-core path"
    d = dealer.deal(synth.Z64, M, K, N, n=2, seed=M * 7 + K)
    for i, p in enumerate(d.parties):
        Z = gpu_share(synth.Z64, i, d.E, d.F, p.A, p.B, p.C)
        assert np.array_equal(Z, O.linear_share(64, i, d.E, d.F, p.A, p.B, p.C)), f"share party {i}"
        mZ = gpu_tag_full(synth.Z64, i, p.alpha, d.E, d.F, p.mA, p.mB, p.mC)
        assert np.array_equal(mZ, O.linear_tag_full(64, p.alpha, d.E, d.F, p.mA, p.mB, p.mC)), \
            f"full tag party {i}"
    assert abi.mpc_device_status() == 0


PATTERNS = [0x7F7F7F7F7F7F7F80,   # every signed digit -128
            0x7F7F7F7F7F7F7F7F,   # every digit 127
            0xFFFFFFFFFFFFFFFF, 0x8080808080808080, 0x0000000000000080, 0x0123456789ABCDEF]


@pytest.mark.parametrize("pat", PATTERNS, ids=hex)
@pytest.mark.parametrize("shape", [(130, 256, 70), (128, 1024, 64)], ids=str)
def test_tc_digit_extremes(pat, shape):
    M, K, N = shape
    assert _path(M, K, N) == 1
    mk = lambda *s: np.full(s, pat, dtype=np.uint64)
    E, F, A, B, C = mk(M, K), mk(K, N), mk(M, K), mk(K, N), mk(M, N)
    for party in (0, 1):
        assert np.array_equal(gpu_share(synth.Z64, party, E, F, A, B, C),
                              O.linear_share(64, party, E, F, A, B, C))
    alpha = np.array([pat], dtype=np.uint64)
    assert np.array_equal(gpu_tag_full(synth.Z64, 1, alpha, E, F, A, B, C),
                          O.linear_tag_full(64, alpha, E, F, A, B, C))
    assert abi.mpc_device_status() == 0


def test_tc_mixed_extremes():
    """Rows and columns alternating between the digit extremes, so diagonal
    sums mix +2^14 and -2^14 products."""
    M, K, N = 130, 512, 66
    lo, hi = np.uint64(0x7F7F7F7F7F7F7F80), np.uint64(0x7F7F7F7F7F7F7F7F)
    a = np.where((np.arange(M * K) % 3) == 0, lo, hi).astype(np.uint64)
    b = np.where((np.arange(K * N) % 5) == 0, lo, np.uint64(0x8080808080808080)).astype(np.uint64)
    E, A = a.reshape(M, K), a[::-1].copy().reshape(M, K)
    F, B = b.reshape(K, N), b[::-1].copy().reshape(K, N)
    C = synth.uniform(5, 5, 0, (M, N), 64)
    for party in (0, 1):
        assert np.array_equal(gpu_share(synth.Z64, party, E, F, A, B, C),
                              O.linear_share(64, party, E, F, A, B, C))


def test_tc_repeated_runs_stable():
    """Many consecutive runs of a layer whose work units span tile boundaries
    on every SM: every run must equal the oracle (guards the pipeline's
    cross-proxy ordering, whose absence corrupted a few tiles per run)."""
    M, K, N = 128, 2048, 4096
    assert _path(M, K, N) == 1
    g = lambda name, shape: synth.uniform(99, synth.TID[name], 0, shape, 64)
    E, F, A, B, C = g("E", (M, K)), g("F", (K, N)), g("A", (M, K)), g("B", (K, N)), g("C", (M, N))
    rows = np.repeat(np.array([3, 70, 127]), N).astype(np.int64)
    cols = np.tile(np.arange(N), 3).astype(np.int64)
    want = O.linear_share_at(64, 0, E, F, A, B, C, rows, cols)
    import torch
    from gpuhelp import dev, empty_like_ring, host
    L = abi.make_layer(M, K, N, 32, 32, 0, 2)
    d = [dev(a) for a in (E, F, A, B, C)]
    ws = torch.empty(abi.mpc_workspace_size(L, abi.MPC_WS_SHARE), dtype=torch.uint8, device="cuda")
    for rep in range(60):
        Z = empty_like_ring((M, N), 1)
        abi.mpc_linear_share(L, *d, Z, ws=ws)
        assert np.array_equal(host(Z)[rows, cols], want), f"run {rep}"
    assert abi.mpc_device_status() == 0


SHAPES_128 = [(130, 64, 70), (64, 256, 33), (200, 512, 100), (9, 1024, 512), (257, 96, 48)]


@pytest.mark.parametrize("shape", SHAPES_128, ids=str)
def test_tc_path_parity_z128(shape):
    """Z_2^128 (k = s = 64): 16 digits per element, 136 digit products."""
    M, K, N = shape
    assert abi.mpc_gemm_path(abi.make_layer(M, K, N, 64, 64)) == 1
    d = dealer.deal(synth.Z128, M, K, N, n=2, seed=M * 11 + K)
    for i, p in enumerate(d.parties):
        Z = gpu_share(synth.Z128, i, d.E, d.F, p.A, p.B, p.C)
        assert np.array_equal(Z, O.linear_share(128, i, d.E, d.F, p.A, p.B, p.C)), f"share party {i}"
        mZ = gpu_tag_full(synth.Z128, i, p.alpha, d.E, d.F, p.mA, p.mB, p.mC)
        assert np.array_equal(mZ, O.linear_tag_full(128, p.alpha, d.E, d.F, p.mA, p.mB, p.mC)), \
            f"full tag party {i}"
    assert abi.mpc_device_status() == 0


PATTERNS_128 = [(0x7F7F7F7F7F7F7F80, 0x7F7F7F7F7F7F7F7F),   # every digit -128
                (0x7F7F7F7F7F7F7F7F, 0x7F7F7F7F7F7F7F7F),   # every digit 127
                (0xFFFFFFFFFFFFFFFF, 0xFFFFFFFFFFFFFFFF),
                (0x8080808080808080, 0x8080808080808080),
                (0x0123456789ABCDEF, 0xFEDCBA9876543210)]


@pytest.mark.parametrize("pat", PATTERNS_128, ids=lambda p: hex(p[1]))
def test_tc_digit_extremes_z128(pat):
    M, K, N = 130, 256, 40
    assert abi.mpc_gemm_path(abi.make_layer(M, K, N, 64, 64)) == 1
    mk = lambda *s: np.broadcast_to(np.array(pat, dtype=np.uint64), s + (2,)).copy()
    E, F, A, B, C = mk(M, K), mk(K, N), mk(M, K), mk(K, N), mk(M, N)
    for party in (0, 1):
        assert np.array_equal(gpu_share(synth.Z128, party, E, F, A, B, C),
                              O.linear_share(128, party, E, F, A, B, C))
    alpha = np.array([list(pat)], dtype=np.uint64)
    assert np.array_equal(gpu_tag_full(synth.Z128, 1, alpha, E, F, A, B, C),
                          O.linear_tag_full(128, alpha, E, F, A, B, C))
    assert abi.mpc_device_status() == 0


RAGGED_K = [(synth.Z64, (2100, 27, 64)), (synth.Z64, (300, 100, 80)), (synth.Z64, (600, 37, 98)),
            (synth.Z128, (400, 27, 50)), (synth.Z128, (300, 45, 41))]


@pytest.mark.parametrize("ring,shape", RAGGED_K, ids=lambda x: str(x) if isinstance(x, tuple) else "")
def test_tc_ragged_k(ring, shape):
    """K not a multiple of 16 (each K half is zero-padded to Kp): im2col layers
    such as the first 3x3 convolution on 3 channels (K = 27)."""
    M, K, N = shape
    assert abi.mpc_gemm_path(abi.make_layer(M, K, N, ring.k, ring.s)) == 1
    d = dealer.deal(ring, M, K, N, n=2, seed=K * 13 + N)
    for i, p in enumerate(d.parties):
        assert np.array_equal(gpu_share(ring, i, d.E, d.F, p.A, p.B, p.C),
                              O.linear_share(ring.bits, i, d.E, d.F, p.A, p.B, p.C))
        assert np.array_equal(gpu_tag_full(ring, i, p.alpha, d.E, d.F, p.mA, p.mB, p.mC),
                              O.linear_tag_full(ring.bits, p.alpha, d.E, d.F, p.mA, p.mB, p.mC))
    assert abi.mpc_device_status() == 0


@pytest.mark.parametrize("ring,shape", [(synth.Z64, (1024, 512, 2048)), (synth.Z128, (1024, 256, 512))],
                         ids=["z64_waves", "z128_waves"])
def test_tc_waves_repeated_runs_stable(ring, shape):
    """Repeated runs of a layer with more tiles than CTAs (full data-parallel
    waves written directly through the staged epilogue, then a stream-K
    remainder): every run is bit-identical to the first, which equals the oracle."""
    M, K, N = shape
    assert _path(M, K, N, ring.k, ring.s) == 1
    g = lambda name, shape: synth.uniform(77, synth.TID[name], 0, shape, ring.bits)
    E, F, A, B, C = g("E", (M, K)), g("F", (K, N)), g("A", (M, K)), g("B", (K, N)), g("C", (M, N))
    import torch
    from gpuhelp import dev, empty_like_ring, host
    L = abi.make_layer(M, K, N, ring.k, ring.s, 1, 2)
    d = [dev(a) for a in (E, F, A, B, C)]
    ws = torch.empty(abi.mpc_workspace_size(L, abi.MPC_WS_SHARE), dtype=torch.uint8, device="cuda")
    first = None
    for rep in range(30):
        Z = empty_like_ring((M, N), ring.words)
        abi.mpc_linear_share(L, *d, Z, ws=ws)
        if first is None:
            first = Z.clone()
            assert np.array_equal(host(Z), O.linear_share(ring.bits, 1, E, F, A, B, C))
        else:
            assert torch.equal(Z, first), f"run {rep}"
    assert abi.mpc_device_status() == 0
