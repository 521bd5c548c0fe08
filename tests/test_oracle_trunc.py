"""Pins of the oracle's truncated layer (Fig. Pi_OptMAC&Trunc and the
truncated Fig. Pi_CompactMatMul, §3.4).

Independent routes: the textbook product X.Y (numpy object matmul), the MAC
relation of §2.4, the f = 0 reduction (truncation by 2^0 is the identity), the
probabilistic-truncation bound, the unit-combiner special case against the
full-tag oracle with alpha = 0, and tamper detection.
"""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import dealer

RINGS = [synth.Z64, synth.Z128]


def ints(a, bits):
    return O.to_int(a, bits)


def mod(v, bits):
    return np.vectorize(lambda x: int(x) % (1 << bits), otypes=[object])(np.asarray(v, dtype=object))


def xy(d, bits):
    return mod(ints(d.X, bits).dot(ints(d.Y, bits)), bits)


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}")
@pytest.mark.parametrize("n", [1, 2, 3])
def test_trunc_mac_relation(ring, n):
    bits = ring.bits
    t = dealer.deal_trunc(ring, 5, 7, 6, n=n, seed=60 + n, f=13)
    out = dealer.run_layer_trunc(t)
    a = ints(t.base.alpha, bits)[0]
    Zf = ints(dealer.total(bits, out["Zf"]), bits)
    assert np.array_equal(ints(dealer.total(bits, out["mZf"]), bits), mod(Zf * a, bits))


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}")
def test_trunc_by_zero_bits_is_the_product(ring):
    """f = 0: sum_i [Z^f]_i = R~ + E.U - D = X.Y (mod 2^k)."""
    bits = ring.bits
    t = dealer.deal_trunc(ring, 4, 9, 5, n=2, seed=70, f=0)
    out = dealer.run_layer_trunc(t)
    Zf = ints(dealer.total(bits, out["Zf"]), bits)
    assert np.array_equal(mod(Zf, ring.k), mod(xy(t.base, bits), ring.k))


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}")
@pytest.mark.parametrize("f", [1, 8, 16, 20])
def test_trunc_error_at_most_one(ring, f):
    """For every input: sum_i [Z^f]_i = (X.Y mod 2^k) / 2^f + e (mod 2^(k-f))
    with e in {-1, 0, 1} (probabilistic truncation; floor division)."""
    bits = ring.bits
    for seed in range(5):
        t = dealer.deal_trunc(ring, 6, 11, 7, n=2, seed=80 + seed, f=f)
        out = dealer.run_layer_trunc(t)
        Zf = ints(dealer.total(bits, out["Zf"]), bits)
        want = np.vectorize(lambda v: (int(v) % (1 << ring.k)) >> f, otypes=[object])(xy(t.base, bits))
        err = mod(Zf - want, ring.k - f)
        top = (1 << (ring.k - f)) - 1
        assert all(e in (0, 1, top) for e in err.reshape(-1)), (f, seed)


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}")
def test_trunc_compact_relations_and_check(ring):
    bits = ring.bits
    t = dealer.deal_trunc(ring, 6, 5, 7, n=3, seed=90, f=12)
    out = dealer.run_layer_trunc(t)
    a = ints(t.base.alpha, bits)[0]
    Dt = ints(out["Dt"], bits)
    chi = ints(t.base.chi, bits)
    assert np.array_equal(ints(out["Dc"], bits), mod(Dt.dot(chi), bits))
    assert np.array_equal(ints(dealer.total(bits, out["mDc"]), bits), mod(Dt.dot(chi) * a, bits))
    assert ints(out["cs_total"], bits)[0] == 0


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}")
def test_trunc_tamper_detected(ring):
    bits = ring.bits
    for seed in range(40):
        t = dealer.deal_trunc(ring, 3, 4, 5, n=2, seed=300 + seed, f=8)
        e = int(synth.words(seed, 91, 0, 1)[0]) | 1        # odd: nonzero mod 2^k
        out = dealer.run_layer_trunc(t, tamper={"Dt": (seed % 15, e)})
        assert ints(out["cs_total"], bits)[0] != 0


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}")
def test_trunc_compact_unit_combiner(ring):
    """chi = e_j: the truncated compact tag share equals column j of
    m(C)_i + E.m(B)_i + m(A)_i.F, i.e. the full-tag oracle with alpha = 0."""
    bits = ring.bits
    M, K, N = 4, 5, 6
    t = dealer.deal_trunc(ring, M, K, N, n=2, seed=95, f=4)
    d = t.base
    out = dealer.run_layer_trunc(t)
    zero = O.from_int(np.array([0], dtype=object), bits)
    for p in d.parties:
        base = ints(O.linear_tag_full(bits, zero, d.E, d.F, p.mA, p.mB, p.mC), bits)
        for j in range(N):
            e = np.zeros(N, dtype=object); e[j] = 1
            _, _, mZc = O.compact_tag_trunc(bits, p.alpha, d.E, d.F, p.mA, p.mB, p.mC, p.mR, out["Dt"],
                                            O.from_int(e, bits))
            assert np.array_equal(ints(mZc, bits), base[:, j])
