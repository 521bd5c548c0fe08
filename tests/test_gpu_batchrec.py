"""GPU parity of Pi_BatchRec (§2.5): the open-phase masking and the tag check
with combiners expanded from a seed in-kernel, against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle import dealer
from paper_2311_04406_gb300 import abi, build

from gpuhelp import dev, empty_like_ring, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    abi.load()


def _mask(ring, X, A, R, mX, mA, mR):
    rows, cols = X.shape[:2]
    W = empty_like_ring((rows, cols), ring.words)
    mW = empty_like_ring((rows, cols), ring.words)
    abi.mpc_batchrec_mask(ring.k, ring.s, rows, cols, dev(X), None if A is None else dev(A), dev(R), dev(mX),
                          None if mA is None else dev(mA), dev(mR), W, mW)
    return host(W), host(mW)


def _check_seeded(ring, alpha, seed, W, mW):
    rows, cols = W.shape[:2]
    L = abi.make_layer(rows, 1, cols, ring.k, ring.s)
    cs = empty_like_ring((1,), ring.words)
    seed_t = torch.tensor([np.int64(np.uint64(seed).view(np.int64))], dtype=torch.int64, device="cuda")
    abi.mpc_tag_check(L, abi.MPC_CHECK_BATCHREC_SEEDED, dev(alpha), seed_t, dev(W), dev(mW), cs)
    return host(cs)


@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=["z64", "z128"])
@pytest.mark.parametrize("shape", [(1, 1), (7, 5), (300, 257), (1024, 576)], ids=str)
def test_mask_and_seeded_check_parity(ring, shape):
    bits = ring.bits
    d = dealer.deal_batchrec(ring, *shape, n=2, seed=shape[0] * 3 + shape[1])
    for i in range(2):
        W, mW = _mask(ring, d.X[i], d.A[i], d.R[i], d.mX[i], d.mA[i], d.mR[i])
        rW, rmW = O.batchrec_mask(bits, d.X[i], d.A[i], d.R[i], d.mX[i], d.mA[i], d.mR[i])
        assert np.array_equal(W, rW) and np.array_equal(mW, rmW)
        # without A (V = X)
        W2, mW2 = _mask(ring, d.X[i], None, d.R[i], d.mX[i], None, d.mR[i])
        z = np.zeros_like(d.A[i])
        rW2, rmW2 = O.batchrec_mask(bits, d.X[i], z, d.R[i], d.mX[i], z, d.mR[i])
        assert np.array_equal(W2, rW2) and np.array_equal(mW2, rmW2)
    for seed in (0, 1, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF):
        chi = O.chi_seeded(bits, ring.s, seed, shape)
        W = synth.uniform(seed & 0xFFFF, 1, 0, shape, bits)
        mW = synth.uniform(seed & 0xFFFF, 2, 0, shape, bits)
        alpha = dealer.key_range(ring, 5, 5, 0, (1,))
        got = _check_seeded(ring, alpha, seed, W, mW)
        assert np.array_equal(got.reshape(-1), O.check_batchrec(bits, alpha, chi, W, mW).reshape(-1))


@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=["z64", "z128"])
def test_opening_round_trip_on_gpu(ring):
    """Two parties mask on the GPU, the harness opens W, each party's seeded
    check share comes from the GPU: honest -> sum 0, tampered W -> nonzero."""
    bits = ring.bits
    d = dealer.deal_batchrec(ring, 64, 48, n=2, seed=77)
    outs = [_mask(ring, d.X[i], d.A[i], d.R[i], d.mX[i], d.mA[i], d.mR[i]) for i in range(2)]
    W = dealer.total(bits, [o[0] for o in outs])
    assert np.array_equal(O.to_int(W, bits) % (1 << ring.k), O.to_int(d.V, bits) % (1 << ring.k))
    cs = [_check_seeded(ring, d.alphas[i], 0xC0FFEE, W, outs[i][1]) for i in range(2)]
    assert O.to_int(dealer.total(bits, cs), bits)[0] == 0
    bad = W.copy()
    bad.reshape(-1, ring.words)[100, 0] ^= np.uint64(1 << 7)
    cs = [_check_seeded(ring, d.alphas[i], 0xC0FFEE, bad, outs[i][1]) for i in range(2)]
    assert O.to_int(dealer.total(bits, cs), bits)[0] != 0
