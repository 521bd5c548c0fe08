"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests retypes an oracle formula: each checks the oracle against an
independent route (numpy's object-dtype matrix product on Python integers, the
MAC relation of §2.4 after reconstruction, special cases with a known answer,
tamper detection, Theorem 1's bound, values the paper prints).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import synth
from oracle import dealer

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RINGS = [synth.Z64, synth.Z128, synth.Ring(4, 4)]
SHAPES = [(1, 1, 1), (2, 3, 2), (3, 1, 4), (3, 4, 5), (5, 7, 3), (1, 9, 1)]


def ints(a, bits):
    return O.to_int(a, bits)


def matmul_int(X, Y, bits):
    """Textbook product with numpy's object matmul on Python ints, reduced."""
    return np.vectorize(lambda v: v % (1 << bits), otypes=[object])(X.dot(Y))


def mod(v, bits):
    return np.vectorize(lambda x: int(x) % (1 << bits), otypes=[object])(np.asarray(v, dtype=object))


def eq(a, b):
    return np.array_equal(np.asarray(a, dtype=object), np.asarray(b, dtype=object))


# ---------------------------------------------------------------------------
# ring GEMM and the share (a1)

@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}s{r.s}")
@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_ring_gemm_matches_object_matmul(ring, shape):
    M, K, N = shape
    bits = ring.bits
    X = synth.uniform(11, 1, 0, (M, K), bits)
    Y = synth.uniform(11, 2, 0, (K, N), bits)
    got = ints(O.ring_gemm(bits, X, Y), bits)
    assert eq(got, matmul_int(ints(X, bits), ints(Y, bits), bits))


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}s{r.s}")
@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_single_party_share_is_textbook_product(ring, shape):
    """n = 1 and C~ = A~B~: a1 reduces to (A + E)(B + F) = X . Y (P1 pin)."""
    M, K, N = shape
    d = dealer.deal(ring, M, K, N, n=1, seed=3)
    p = d.parties[0]
    Z = O.linear_share(ring.bits, 0, d.E, d.F, p.A, p.B, p.C)
    assert eq(ints(Z, ring.bits), matmul_int(ints(d.X, ring.bits), ints(d.Y, ring.bits), ring.bits))


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}s{r.s}")
@pytest.mark.parametrize("n", [2, 3, 5])
def test_share_reconstruction(ring, n):
    """I1: sum_i [Z]_i == X~ . Y~ mod 2^{k+s}; also mod 2^k (A10)."""
    bits = ring.bits
    d = dealer.deal(ring, 4, 6, 5, n=n, seed=100 + n)
    out = dealer.run_layer(d)
    Zt = ints(dealer.total(bits, out["Z"]), bits)
    XY = matmul_int(ints(d.X, bits), ints(d.Y, bits), bits)
    assert eq(Zt, XY)
    assert eq(mod(Zt, ring.k), mod(XY, ring.k))


def test_share_party_roles_differ():
    """Only party 0 adds E.F: moving the term to party 1 changes both shares
    but keeps the reconstruction (the term is public)."""
    ring = synth.Z64
    d = dealer.deal(ring, 3, 4, 5, n=2, seed=9)
    p0, p1 = d.parties
    z0 = O.linear_share(64, 0, d.E, d.F, p0.A, p0.B, p0.C)
    z0_as1 = O.linear_share(64, 1, d.E, d.F, p0.A, p0.B, p0.C)
    EF = O.ring_gemm(64, d.E, d.F)
    assert eq(ints(O.sub(64, z0, z0_as1), 64), ints(EF, 64))


# ---------------------------------------------------------------------------
# tags: full (a2), optimistic (a3), compact (a4, a5), check (a6)

@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}s{r.s}")
@pytest.mark.parametrize("n", [1, 2, 3])
def test_full_tag_mac_relation(ring, n):
    """I2 for the full tag: sum_i [m(Z)]_i == alpha . X~Y~."""
    bits = ring.bits
    d = dealer.deal(ring, 4, 3, 6, n=n, seed=200 + n)
    out = dealer.run_layer(d)
    mZ = ints(dealer.total(bits, out["mZ_full"]), bits)
    XY = matmul_int(ints(d.X, bits), ints(d.Y, bits), bits)
    a = ints(d.alpha, bits)[0]
    assert eq(mZ, mod(XY * a, bits))


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}s{r.s}")
@pytest.mark.parametrize("full_alpha", [False, True])
def test_optimistic_tag_mac_relation(ring, full_alpha):
    """I2 for the OptMAC tag: sum_i [m(Z)]_i == alpha . sum_i [Z]_i, for alpha_i
    in [0, 2^s) and for full-width alpha_i (A7)."""
    bits = ring.bits
    d = dealer.deal(ring, 5, 4, 3, n=3, seed=300, alpha_full_width=full_alpha)
    out = dealer.run_layer(d)
    mZ = ints(dealer.total(bits, out["mZ_opt"]), bits)
    Zt = ints(dealer.total(bits, out["Z"]), bits)
    a = ints(d.alpha, bits)[0]
    assert eq(mZ, mod(Zt * a, bits))


def test_reading_alpha_EF_every_party():
    """A1: only the reading 'every party adds alpha_i (E.F)' satisfies I2."""
    bits = 64
    d = dealer.deal(synth.Z64, 3, 4, 5, n=2, seed=17)
    out = dealer.run_layer(d)
    EF = O.ring_gemm(bits, d.E, d.F)
    p1 = d.parties[1]
    # the P1-only reading: party index 1 would not add alpha_1 (E.F)
    mz1_alt = O.sub(bits, out["mZ_full"][1], O.smul(bits, p1.alpha, EF))
    alt = ints(dealer.total(bits, [out["mZ_full"][0], mz1_alt]), bits)
    Zt = ints(dealer.total(bits, out["Z"]), bits)
    a = ints(d.alpha, bits)[0]
    assert not eq(alt, mod(Zt * a, bits))


def test_reading_lifted_D():
    """A3: using D mod 2^k instead of the lifted D~ breaks I2 whenever D~ >= 2^k."""
    ring = synth.Z64
    bits = ring.bits
    d = dealer.deal(ring, 4, 4, 4, n=2, seed=23)
    out = dealer.run_layer(d)
    Dk = O.from_int(mod(ints(out["Dt"], bits), ring.k), bits)
    assert (ints(out["Dt"], bits) >= (1 << ring.k)).any()
    alt = [O.optmac(bits, p.alpha, p.mR, Dk) for p in d.parties]
    Zt = ints(dealer.total(bits, out["Z"]), bits)
    a = ints(d.alpha, bits)[0]
    assert not eq(ints(dealer.total(bits, alt), bits), mod(Zt * a, bits))


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}s{r.s}")
@pytest.mark.parametrize("n", [1, 2, 4])
def test_compact_relations(ring, n):
    """I3: sum_i m(Z^c)_i == alpha (Z~ chi), D^c == D~ chi,
    sum_i m(D^c)_i == alpha D^c, and the honest checksum is 0."""
    bits = ring.bits
    d = dealer.deal(ring, 6, 5, 7, n=n, seed=400 + n)
    out = dealer.run_layer(d)
    a = ints(d.alpha, bits)[0]
    chi = ints(d.chi, bits)
    Zt = ints(dealer.total(bits, out["Z"]), bits)
    Dt = ints(out["Dt"], bits)
    assert eq(ints(dealer.total(bits, out["mZc"]), bits), mod(Zt.dot(chi) * a, bits))
    assert eq(ints(out["Dc"], bits), mod(Dt.dot(chi), bits))
    assert eq(ints(dealer.total(bits, out["mDc"]), bits), mod(Dt.dot(chi) * a, bits))
    assert ints(out["cs_total"], bits)[0] == 0


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}s{r.s}")
def test_compact_tag_unit_combiner_is_full_tag_column(ring):
    """chi = e_j: per party, m(Z^c)_i equals column j of the full-tag share
    (bit-exact, no reconstruction), and D^c is column j of D~."""
    bits = ring.bits
    M, K, N = 4, 5, 6
    d = dealer.deal(ring, M, K, N, n=2, seed=31)
    out = dealer.run_layer(d)
    for j in range(N):
        e = np.zeros(N, dtype=object); e[j] = 1
        chi = O.from_int(e, bits)
        for i, p in enumerate(d.parties):
            mDc, Dc, mZc = O.compact_tag(bits, p.alpha, d.E, d.F, p.mA, p.mB, p.mC, p.mR,
                                         out["Dt"], chi)
            full = ints(out["mZ_full"][i], bits)
            assert eq(ints(mZc, bits), full[:, j])
            assert eq(ints(Dc, bits), ints(out["Dt"], bits)[:, j])
            mR = ints(p.mR, bits)
            assert eq(ints(mDc, bits), mod(mR[:, j] - full[:, j], bits))


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}s{r.s}")
def test_compress_special_combiners(ring):
    """Pi_Compress: chi = e_j picks column j; chi = all ones gives row sums."""
    bits = ring.bits
    Mat = synth.uniform(5, 1, 0, (4, 7), bits)
    Mi = ints(Mat, bits)
    for j in range(7):
        e = np.zeros(7, dtype=object); e[j] = 1
        assert eq(ints(O.compress(bits, Mat, O.from_int(e, bits)), bits), Mi[:, j])
    ones = O.from_int(np.ones(7, dtype=object), bits)
    assert eq(ints(O.compress(bits, Mat, ones), bits), mod(Mi.sum(axis=1), bits))


@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=lambda r: f"k{r.k}s{r.s}")
def test_check_unit_combiner(ring):
    """chi^ = e_r: the check share is alpha_i Dc_r - m(D^c)_{i,r}."""
    bits = ring.bits
    d = dealer.deal(ring, 5, 3, 4, n=2, seed=37)
    out = dealer.run_layer(d)
    p = d.parties[1]
    for r in range(5):
        e = np.zeros(5, dtype=object); e[r] = 1
        cs = O.check_compact(bits, p.alpha, O.from_int(e, bits), out["Dc"], out["mDc"][1])
        want = ints(p.alpha, bits)[0] * ints(out["Dc"], bits)[r] - ints(out["mDc"][1], bits)[r]
        assert ints(cs, bits)[0] == want % (1 << bits)


# ---------------------------------------------------------------------------
# tamper tests (must be caught)

def _tamper_runs(ring, kind, seeds, n=2, shape=(3, 4, 5)):
    bits = ring.bits
    caught = 0
    for sd in seeds:
        d = dealer.deal(ring, *shape, n=n, seed=sd)
        ws = synth.words(sd, 90, 0, 4)
        j = int(ws[0] % (shape[0] * shape[2]))
        e = int(ws[1]) % (1 << bits)
        if e % (1 << ring.k) == 0:
            e += 1
        if kind == "Dt":
            t = {"Dt": (j, e)}
        elif kind == "Z":
            t = {"Z": (int(ws[2] % n), j, e)}
        else:
            t = {"alpha": (int(ws[2] % n), e)}
        out = dealer.run_layer(d, tamper=t)
        if ints(out["cs_total"], bits)[0] != 0:
            caught += 1
    return caught


@pytest.mark.parametrize("kind", ["Dt", "Z", "alpha"])
@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=lambda r: f"k{r.k}s{r.s}")
def test_tamper_detected(ring, kind):
    """P6: an error e != 0 mod 2^k in D~, in one [Z]_i, or in one alpha_i makes
    the reconstructed checksum nonzero (escape probability <= 2^-26, Thm. 1)."""
    seeds = range(1000, 1150)
    assert _tamper_runs(ring, kind, seeds) == len(seeds)


def test_tampered_tag_caught_by_batchrec():
    """An error added to one full-tag share is caught by the Pi_BatchRec tag
    check on the reconstructed Z; honest tags pass it."""
    ring = synth.Z64
    bits = 64
    for sd in range(50):
        d = dealer.deal(ring, 3, 4, 5, n=2, seed=2000 + sd)
        out = dealer.run_layer(d)
        W = dealer.total(bits, out["Z"])
        chiW = synth.uniform(sd, synth.TID["chiW"], 0, (3, 5), ring.s)
        cs = [O.check_batchrec(bits, p.alpha, chiW, W, m) for p, m in zip(d.parties, out["mZ_full"])]
        assert ints(dealer.total(bits, cs), bits)[0] == 0
        bad = out["mZ_full"][1].copy()
        bad.reshape(-1)[sd % 15] ^= np.uint64(1 << (sd % 32))
        cs[1] = O.check_batchrec(bits, d.parties[1].alpha, chiW, W, bad)
        assert ints(dealer.total(bits, cs), bits)[0] != 0


def test_batchrec_all_ones_combiner():
    """chi = 1 everywhere: the BatchRec share is sum (m(W)_i - alpha_i W)."""
    bits = 64
    W = synth.uniform(3, 1, 0, (2, 3), bits)
    mW = synth.uniform(3, 2, 0, (2, 3), bits)
    ones = O.from_int(np.ones((2, 3), dtype=object), bits)
    alpha = synth.uniform(3, 3, 0, (1,), 32)
    cs = ints(O.check_batchrec(bits, alpha, ones, W, mW), bits)[0]
    want = (ints(mW, bits) - ints(W, bits) * int(alpha[0])).sum() % (1 << bits)
    assert cs == want


def test_theorem1_false_accept_rate():
    """P7: at k = s = 4 random errors (not 0 mod 2^k) on D~ escape the compact
    check with frequency <= 2^(-s + log2(s+1)) = 0.3125."""
    ring = synth.Ring(4, 4)
    trials = 400
    caught = _tamper_runs(ring, "Dt", range(5000, 5000 + trials), shape=(2, 3, 2))
    rate = 1.0 - caught / trials
    bound = 2.0 ** (-4 + math.log2(5))
    assert rate <= bound, (rate, bound)


def test_literal_check_modulus_fails_honest_runs():
    """A4: the printed mod 2^{k+2s} check rejects honest runs at (k, s) =
    (32, 32), while the mod 2^{k+s} reading accepts them (parity unpinned
    form, recorded only)."""
    ring = synth.Z64
    rejected = 0
    for sd in range(20):
        d = dealer.deal(ring, 3, 4, 5, n=2, seed=3000 + sd)
        out = dealer.run_layer(d)
        assert ints(out["cs_total"], 64)[0] == 0
        lit = sum(O.check_compact_literal(32, 32, p.alpha, d.chi_hat, out["Dc"], m)
                  for p, m in zip(d.parties, out["mDc"])) % (1 << 96)
        rejected += lit != 0
    assert rejected > 0


# ---------------------------------------------------------------------------
# closed forms printed by the paper

def test_paper_constants():
    from paper_2311_04406_gb300 import costmodel as cm
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    for r in g["rings"]:
        assert cm.sigma(r["s"]) == r["sigma"]
        assert r["k"] + r["s"] == r["share_bits"]
    t = g["tag_mult_reduction"]
    ratio = cm.tag_mult_ratio(t["M"], t["K"], t["N"])
    assert round(ratio) == t["printed_ratio"]
    h = g["fp64_limb_headroom"]
    assert 2 ** (h["fraction_bits"] - h["product_bits"]) == h["accumulations"]
    assert cm.digit_products(64) == 36 and cm.digit_products(128) == 136
    assert abs(cm.check_failure_bound(4) - 0.3125) < 1e-12


def test_cost_model_counts_by_enumeration():
    """The §3.4.3 counts against an explicit tally of the products in the
    definitions (tiny shapes)."""
    from paper_2311_04406_gb300 import costmodel as cm
    for M, K, N in [(1, 1, 1), (2, 3, 4), (5, 2, 7)]:
        full = M * K * N * 3 + M * N          # E.m(B), m(A).U, E.U, alpha * (E.U)
        compact = (3 * M * N + 2 * K * N) + (3 * M * K + M) + M * N
        assert cm.full_tag_mults(M, K, N) == full
        assert cm.compact_tag_mults(M, K, N) == compact


def test_storage_roundtrip():
    for bits in (8, 64, 128):
        v = np.array([0, 1, (1 << bits) - 1, 12345 % (1 << bits)], dtype=object)
        assert eq(O.to_int(O.from_int(v, bits), bits), v)
