"""GPU parity: every output of the CUDA path equals the oracle's bit for bit.

The integer outputs are exact, so the tolerance is zero.  Small and ragged
shapes are compared in full (several tiles plus ragged tails); the full-size
CNN-style layers (im2col 1024 x 576 x 64 and dense 128 x 4096 x 4096) are
compared in full where the oracle is fast (CompactTag path, conv layer) and at
sampled output positions otherwise.
"""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import dealer
from paper_2311_04406_gb300 import abi, build

from gpuhelp import (gpu_check_batchrec, gpu_check_compact, gpu_share, gpu_tag_compact,
                     gpu_tag_full)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    abi.load()


SHAPES_64 = [(1, 1, 1), (1, 5, 1), (3, 1, 4), (64, 128, 64), (65, 129, 67), (128, 27, 64),
             (4, 512, 10), (130, 200, 260), (257, 64, 96), (0, 5, 4), (5, 0, 4), (5, 4, 0)]
SHAPES_128 = [(1, 1, 1), (3, 4, 5), (33, 70, 17), (64, 128, 64), (129, 40, 33)]


def _layer_parity(ring, shape, n, seed):
    M, K, N = shape
    d = dealer.deal(ring, M, K, N, n=n, seed=seed)
    ref = dealer.run_layer(d)
    for i, p in enumerate(d.parties):
        Z = gpu_share(ring, i, d.E, d.F, p.A, p.B, p.C, nparties=n)
        assert np.array_equal(Z, ref["Z"][i]), f"share party {i}"
        mZf = gpu_tag_full(ring, i, p.alpha, d.E, d.F, p.mA, p.mB, p.mC, nparties=n)
        assert np.array_equal(mZf, ref["mZ_full"][i]), f"full tag party {i}"
        mZ, mDc, Dc = gpu_tag_compact(ring, i, p.alpha, d.E, d.F, p.mA, p.mB, p.mC, p.mR,
                                      ref["Dt"], d.chi, nparties=n)
        assert np.array_equal(mZ, ref["mZ_opt"][i]), f"optmac tag party {i}"
        assert np.array_equal(mDc, ref["mDc"][i]), f"compact tag party {i}"
        assert np.array_equal(Dc, ref["Dc"]), "compressed D"
        cs = gpu_check_compact(ring, p.alpha, d.chi_hat, Dc, mDc)
        assert np.array_equal(cs.reshape(-1), ref["cs"][i].reshape(-1)), f"check party {i}"


@pytest.mark.parametrize("shape", SHAPES_64, ids=str)
def test_layer_parity_z64(shape):
    _layer_parity(synth.Z64, shape, 2, seed=hash(shape) & 0xFFFF)


@pytest.mark.parametrize("shape", SHAPES_128, ids=str)
def test_layer_parity_z128(shape):
    _layer_parity(synth.Z128, shape, 2, seed=(hash(shape) & 0xFFFF) + 7)


@pytest.mark.parametrize("n", [1, 3])
def test_layer_parity_party_counts(n):
    _layer_parity(synth.Z64, (40, 33, 50), n, seed=50 + n)


def test_single_dense_two_party_mac_relation():
    """The single dense layer (X 64x128, W 128x64, two parties, Z_2^64):
    GPU shares and tags reconstruct to X.W and alpha X.W (MAC relation)."""
    ring = synth.Z64
    L = synth.single_dense()
    d = dealer.deal(ring, L.M, L.K, L.N, n=2, seed=0xC0FFEE00)
    Z = [gpu_share(ring, i, d.E, d.F, p.A, p.B, p.C) for i, p in enumerate(d.parties)]
    mZ = [gpu_tag_full(ring, i, p.alpha, d.E, d.F, p.mA, p.mB, p.mC) for i, p in enumerate(d.parties)]
    XY = O.ring_gemm(64, d.X, d.Y)
    assert np.array_equal(dealer.total(64, Z), XY)
    assert np.array_equal(dealer.total(64, mZ), O.smul(64, d.alpha, XY))
    D = [O.sub(64, p.R, z) for p, z in zip(d.parties, Z)]
    Dt = dealer.total(64, D)
    comp = [gpu_tag_compact(ring, i, p.alpha, d.E, d.F, p.mA, p.mB, p.mC, p.mR, Dt, d.chi)
            for i, p in enumerate(d.parties)]
    assert np.array_equal(dealer.total(64, [c[0] for c in comp]), O.smul(64, d.alpha, XY))
    cs = [gpu_check_compact(ring, p.alpha, d.chi_hat, c[2], c[1]) for p, c in zip(d.parties, comp)]
    assert int(dealer.total(64, cs)[0]) == 0


@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=["z64", "z128"])
def test_all_ones_operands(ring):
    """All-0xFF words: the worst case for every accumulator's magnitude."""
    M, K, N = 130, 300, 70
    w = ring.words
    full = lambda *s: np.full(tuple(s) + ((2,) if w == 2 else ()), 0xFFFFFFFFFFFFFFFF, dtype=np.uint64)
    E, F, A, B, C = full(M, K), full(K, N), full(M, K), full(K, N), full(M, N)
    alpha = full(1)
    for party in (0, 1):
        assert np.array_equal(gpu_share(ring, party, E, F, A, B, C),
                              O.linear_share(ring.bits, party, E, F, A, B, C))
    assert np.array_equal(gpu_tag_full(ring, 1, alpha, E, F, A, B, C),
                          O.linear_tag_full(ring.bits, alpha, E, F, A, B, C))
    chi = full(N)
    mZ, mDc, Dc = gpu_tag_compact(ring, 0, alpha, E, F, A, B, C, C, C, chi)
    rmDc, rDc, _ = O.compact_tag(ring.bits, alpha, E, F, A, B, C, C, C, chi)
    assert np.array_equal(mZ, O.optmac(ring.bits, alpha, C, C))
    assert np.array_equal(mDc, rmDc) and np.array_equal(Dc, rDc)


@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=["z64", "z128"])
def test_signed_digit_extremes(ring):
    """Words whose bytes are all 0x80 or 0x7F (the ends of the signed-digit
    range) and alternating patterns."""
    M, K, N = 97, 260, 45
    w = ring.words
    pats = [0x8080808080808080, 0x7F7F7F7F7F7F7F7F, 0x807F807F807F807F, 0x0000000000000080]
    rng_words = synth.words(77, 1, 0, 6)
    for t, pat in enumerate(pats):
        def mk(*s, off=0):
            a = np.full(tuple(s) + ((2,) if w == 2 else ()), pat, dtype=np.uint64)
            return a
        E, F, A, B, C = mk(M, K), mk(K, N), mk(M, K), mk(K, N), mk(M, N)
        for party in (0, 1):
            assert np.array_equal(gpu_share(ring, party, E, F, A, B, C),
                                  O.linear_share(ring.bits, party, E, F, A, B, C)), hex(pat)
        alpha = np.array([int(rng_words[t])] * w, dtype=np.uint64).reshape((1,) + ((2,) if w == 2 else ()))
        assert np.array_equal(gpu_tag_full(ring, 1, alpha, E, F, A, B, C),
                              O.linear_tag_full(ring.bits, alpha, E, F, A, B, C)), hex(pat)


def test_batchrec_check_parity():
    ring = synth.Z64
    for (M, N) in [(1, 1), (3, 5), (200, 333), (1024, 64)]:
        W = synth.uniform(1, 1, 0, (M, N), 64)
        mW = synth.uniform(1, 2, 0, (M, N), 64)
        chi = synth.uniform(1, 3, 0, (M, N), 32)
        alpha = synth.uniform(1, 4, 0, (1,), 32)
        assert np.array_equal(gpu_check_batchrec(ring, alpha, chi, W, mW).reshape(-1),
                              O.check_batchrec(64, alpha, chi, W, mW).reshape(-1))
    ring = synth.Z128
    W = synth.uniform(2, 1, 0, (77, 31), 128)
    mW = synth.uniform(2, 2, 0, (77, 31), 128)
    chi = O.from_int(O.to_int(synth.uniform(2, 3, 0, (77, 31), 64), 64), 128)
    alpha = O.from_int(np.array([12345678901234567]), 128)
    assert np.array_equal(gpu_check_batchrec(ring, alpha, chi, W, mW).reshape(-1),
                          O.check_batchrec(128, alpha, chi, W, mW).reshape(-1))


def test_tamper_caught_on_gpu():
    """A tampered D~ seen by all parties makes the GPU checksums sum to non-zero."""
    ring = synth.Z64
    d = dealer.deal(ring, 40, 30, 20, n=2, seed=4242)
    ref = dealer.run_layer(d, tamper={"Dt": (7, 1 << 5)})
    comp = [gpu_tag_compact(ring, i, p.alpha, d.E, d.F, p.mA, p.mB, p.mC, p.mR, ref["Dt"], d.chi)
            for i, p in enumerate(d.parties)]
    cs = [gpu_check_compact(ring, p.alpha, d.chi_hat, c[2], c[1]) for p, c in zip(d.parties, comp)]
    assert int(dealer.total(64, cs)[0]) != 0


# ---------------------------------------------------------------------------
# full-size CNN-style layers (the benchmark's workload), uniform inputs

def _uniform_layer(ring, M, K, N, seed):
    T = synth.TID
    b = ring.bits
    g = lambda name, shape, bits=b: synth.uniform(seed, T[name], 0, shape, bits)
    key = lambda name, shape: dealer.key_range(ring, seed, T[name], 0, shape)
    return dict(E=g("E", (M, K)), F=g("F", (K, N)), A=g("A", (M, K)), B=g("B", (K, N)),
                C=g("C", (M, N)), mA=g("mA", (M, K)), mB=g("mB", (K, N)), mC=g("mC", (M, N)),
                mR=g("mR", (M, N)), Dt=g("Dt", (M, N)), chi=key("chi", (N,)),
                chi_hat=key("chi_hat", (M,)), alpha=key("alpha", (1,)))


@pytest.mark.parametrize("layer", synth.cnn_pair(), ids=lambda l: l.name)
def test_cnn_layers_full_size(layer):
    ring = synth.Z64
    M, K, N = layer.M, layer.K, layer.N
    x = _uniform_layer(ring, M, K, N, seed=0xC0FFEE01)
    Z = gpu_share(ring, 0, x["E"], x["F"], x["A"], x["B"], x["C"])
    mZf = gpu_tag_full(ring, 1, x["alpha"], x["E"], x["F"], x["mA"], x["mB"], x["mC"])
    sw = synth.words(99, 1, 0, 2 * 512)
    rows = (sw[:512] % np.uint64(M)).astype(np.int64)
    cols = (sw[512:] % np.uint64(N)).astype(np.int64)
    rows[:4] = [0, 0, M - 1, M - 1]
    cols[:4] = [0, N - 1, 0, N - 1]
    want_z = O.linear_share_at(64, 0, x["E"], x["F"], x["A"], x["B"], x["C"], rows, cols)
    assert np.array_equal(Z[rows, cols], want_z)
    want_t = O.linear_tag_full_at(64, x["alpha"], x["E"], x["F"], x["mA"], x["mB"], x["mC"], rows, cols)
    assert np.array_equal(mZf[rows, cols], want_t)
    mZ, mDc, Dc = gpu_tag_compact(ring, 1, x["alpha"], x["E"], x["F"], x["mA"], x["mB"], x["mC"],
                                  x["mR"], x["Dt"], x["chi"])
    rmDc, rDc, _ = O.compact_tag(64, x["alpha"], x["E"], x["F"], x["mA"], x["mB"], x["mC"], x["mR"],
                                 x["Dt"], x["chi"])
    assert np.array_equal(mDc, rmDc)
    assert np.array_equal(Dc, rDc)
    assert np.array_equal(mZ, O.optmac(64, x["alpha"], x["mR"], x["Dt"]))
    cs = gpu_check_compact(ring, x["alpha"], x["chi_hat"], Dc, mDc)
    assert np.array_equal(cs.reshape(-1), O.check_compact(64, x["alpha"], x["chi_hat"], rDc, rmDc).reshape(-1))


SKINNY = [(synth.Z64, (1, 4096, 512)), (synth.Z64, (8, 300, 70)), (synth.Z64, (3, 2048, 130)),
          (synth.Z64, (1, 4096, 10)), (synth.Z128, (2, 1024, 96)), (synth.Z128, (7, 33, 5)),
          (synth.Z64, (4, 4608, 512)), (synth.Z64, (5, 1000, 71)), (synth.Z128, (8, 4608, 50)),
          (synth.Z64, (1, 7, 3))]


@pytest.mark.parametrize("ring,shape", SKINNY, ids=lambda x: str(x) if isinstance(x, tuple) else "")
def test_skinny_layers(ring, shape):
    """M <= 8 (dense layers at batch 1-8): the split-K GEMV kernel."""
    M, K, N = shape
    assert abi.mpc_gemm_path(abi.make_layer(M, K, N, ring.k, ring.s)) == 0
    _layer_parity(ring, shape, 2, seed=M + K + N)


@pytest.mark.parametrize("ring,shape", [(synth.Z64, (100, 3000, 21)), (synth.Z128, (70, 500, 9))],
                         ids=lambda x: str(x) if isinstance(x, tuple) else "")
def test_simt_split_k(ring, shape):
    """Layers the tensor path does not take (odd N in Z_2^64, small products)
    with a small output grid: the SIMT tile kernel splits K over blocks and
    adds the partial sums atomically."""
    M, K, N = shape
    assert abi.mpc_gemm_path(abi.make_layer(M, K, N, ring.k, ring.s)) == 0
    _layer_parity(ring, shape, 2, seed=M * 3 + K)


@pytest.mark.parametrize("ring,shape", [(synth.Z64, (3000, 27, 64)), (synth.Z128, (700, 9, 20)),
                                        (synth.Z64, (513, 63, 12))],
                         ids=lambda x: str(x) if isinstance(x, tuple) else "")
def test_compact_small_k(ring, shape):
    """K < 64 (e.g. the first im2col convolution, K = 27): the CompactTag GEMV
    runs one thread per row."""
    _layer_parity(ring, shape, 2, seed=shape[0] + shape[1])
