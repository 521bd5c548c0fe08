"""Pins of the oracle's Pi_BatchRec open phase and seeded combiners (§2.5)."""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import dealer


def ints(a, bits):
    return O.to_int(a, bits)


def mod(v, bits):
    return np.vectorize(lambda x: int(x) % (1 << bits), otypes=[object])(np.asarray(v, dtype=object))


@pytest.mark.parametrize("s", [32, 64])
@pytest.mark.parametrize("bits", [64, 128])
def test_seeded_combiners_are_splitmix64(s, bits):
    """The C oracle's stream against synth's independent numpy SplitMix64
    mixing function: chi_i = mix(seed + (i+1) gamma) mod 2^s."""
    seed = 0x1234ABCD5678
    n = 1000
    got = ints(O.chi_seeded(bits, s, seed, (n,)), bits)
    with np.errstate(over="ignore"):
        state = np.uint64(seed) + np.arange(1, n + 1, dtype=np.uint64) * synth.GAMMA
    want = synth._mix(state).astype(object) % (1 << s)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=lambda r: f"k{r.k}")
@pytest.mark.parametrize("n", [2, 3])
def test_masked_opening_keeps_the_value_mod_2k(ring, n):
    """W = V + R~ with R~ = 0 mod 2^k: the opened W equals V mod 2^k, and the
    tag relation holds for the masked shares."""
    bits = ring.bits
    d = dealer.deal_batchrec(ring, 7, 5, n=n, seed=11 + n)
    outs = [O.batchrec_mask(bits, d.X[i], d.A[i], d.R[i], d.mX[i], d.mA[i], d.mR[i]) for i in range(n)]
    W = ints(dealer.total(bits, [o[0] for o in outs]), bits)
    mW = ints(dealer.total(bits, [o[1] for o in outs]), bits)
    V = ints(d.V, bits)
    assert np.array_equal(mod(W, ring.k), mod(V, ring.k))
    a = ints(d.alpha, bits)[0]
    assert np.array_equal(mW, mod(W * a, bits))
    assert not np.array_equal(W, V)          # the top s bits are masked


@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=lambda r: f"k{r.k}")
def test_batchrec_check_with_seeded_combiners(ring):
    """Honest openings pass the tag check with seeded combiners; an error on the
    opened W (as every party sees it) is caught."""
    bits = ring.bits
    for seed in range(30):
        d = dealer.deal_batchrec(ring, 4, 6, n=2, seed=100 + seed)
        outs = [O.batchrec_mask(bits, d.X[i], d.A[i], d.R[i], d.mX[i], d.mA[i], d.mR[i]) for i in range(2)]
        W = dealer.total(bits, [o[0] for o in outs])
        chi = O.chi_seeded(bits, ring.s, 0xBEEF + seed, (4, 6))
        cs = [O.check_batchrec(bits, d.alphas[i], chi, W, outs[i][1]) for i in range(2)]
        assert ints(dealer.total(bits, cs), bits)[0] == 0
        bad = W.copy()
        bad.reshape(-1, ring.words)[seed % 24, 0] ^= np.uint64(1 << (seed % 32))
        cs = [O.check_batchrec(bits, d.alphas[i], chi, bad, outs[i][1]) for i in range(2)]
        assert ints(dealer.total(bits, cs), bits)[0] != 0
