"""Pins of the oracle functions that the other oracle tests reach only
indirectly: the sampled checkers used by every full-size GPU comparison and the
literal mod 2^{k+2s} form of the compact check.

* `linear_share_at` / `linear_tag_full_at` compute a1 and a2 (Eq. compute-z,
  Eq. compute-ztag, §2.5) at chosen positions.  They are compared element by
  element with the full functions -- themselves pinned against numpy's
  object-dtype product and the MAC relation in test_oracle.py -- on non-square
  shapes, with row and column indices drawn independently, repeated positions,
  both share rings and both party roles.  Positions outside the matrix are
  rejected by the Python wrapper before the C code runs.
* `check_compact_literal` is the check share of Fig. Pi_CompactMatMul
  verification steps 3-5 as printed: step 3 reduces alpha_i * D^c mod 2^{k+s},
  steps 4-5 multiply by chi^ and sum mod 2^{k+2s}.  It is pinned by a case
  worked by hand at k = s = 4 (numbers in the test), by special cases with a
  known answer, and by its relation to the canonical check, which it must
  equal mod 2^{k+s}.
"""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import dealer

RINGS = [synth.Z64, synth.Z128]


def _ints(a, bits):
    return O.to_int(a, bits)


def _positions(M, N, cnt, seed):
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, M, cnt)
    cols = rng.integers(0, N, cnt)
    # repeated positions and the four corners
    rows = np.concatenate([rows, rows[:5], [0, 0, M - 1, M - 1]])
    cols = np.concatenate([cols, cols[:5], [0, N - 1, 0, N - 1]])
    return rows.astype(np.int64), cols.astype(np.int64)


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"w{r.words}")
@pytest.mark.parametrize("shape", [(7, 5, 11), (13, 9, 3), (1, 4, 17), (16, 1, 2)], ids=str)
@pytest.mark.parametrize("party", [0, 1])
def test_sampled_share_equals_full_share(ring, shape, party):
    M, K, N = shape
    b = ring.bits
    g = lambda tid, sh: synth.uniform(0x5A17, tid, party, sh, b)
    E, F, A, B, C = g(1, (M, K)), g(2, (K, N)), g(3, (M, K)), g(4, (K, N)), g(5, (M, N))
    full = O.linear_share(b, party, E, F, A, B, C)
    rows, cols = _positions(M, N, 40, seed=M * 100 + N + party)
    got = O.linear_share_at(b, party, E, F, A, B, C, rows, cols)
    want = full[rows, cols]
    assert np.array_equal(got, want)


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"w{r.words}")
@pytest.mark.parametrize("shape", [(7, 5, 11), (13, 9, 3), (1, 4, 17), (16, 1, 2)], ids=str)
@pytest.mark.parametrize("full_alpha", [False, True])
def test_sampled_full_tag_equals_full_tag(ring, shape, full_alpha):
    M, K, N = shape
    b = ring.bits
    g = lambda tid, sh, bits=b: synth.uniform(0x7A6, tid, 0, sh, bits)
    alpha = g(9, (1,), b if full_alpha else ring.s)
    E, F, mA, mB, mC = g(1, (M, K)), g(2, (K, N)), g(3, (M, K)), g(4, (K, N)), g(5, (M, N))
    full = O.linear_tag_full(b, alpha, E, F, mA, mB, mC)
    rows, cols = _positions(M, N, 40, seed=M * 100 + N + full_alpha)
    got = O.linear_tag_full_at(b, alpha, E, F, mA, mB, mC, rows, cols)
    assert np.array_equal(got, full[rows, cols])


def test_sampled_checkers_follow_party_role():
    """Party 0 alone adds E.F: the sampled share of party 0 minus that of
    party 1 is (E.F) at the sampled positions."""
    ring = synth.Z64
    b = ring.bits
    M, K, N = 6, 7, 9
    g = lambda tid, sh: synth.uniform(42, tid, 0, sh, b)
    E, F, A, B, C = g(1, (M, K)), g(2, (K, N)), g(3, (M, K)), g(4, (K, N)), g(5, (M, N))
    rows, cols = _positions(M, N, 20, seed=3)
    z0 = _ints(O.linear_share_at(b, 0, E, F, A, B, C, rows, cols), b)
    z1 = _ints(O.linear_share_at(b, 1, E, F, A, B, C, rows, cols), b)
    EF = _ints(O.ring_gemm(b, E, F), b)
    assert all((int(x) - int(y)) % (1 << b) == int(EF[r, c]) for x, y, r, c in zip(z0, z1, rows, cols))


@pytest.mark.parametrize("bad", [(-1, 0), (0, -1), (6, 0), (0, 9)])
def test_sampled_checkers_reject_positions_outside(bad):
    b = 64
    M, K, N = 6, 7, 9
    g = lambda tid, sh: synth.uniform(1, tid, 0, sh, b)
    E, F, A, B, C = g(1, (M, K)), g(2, (K, N)), g(3, (M, K)), g(4, (K, N)), g(5, (M, N))
    rows, cols = np.array([1, bad[0]]), np.array([2, bad[1]])
    with pytest.raises(IndexError):
        O.linear_share_at(b, 0, E, F, A, B, C, rows, cols)
    with pytest.raises(IndexError):
        O.linear_tag_full_at(b, np.array([3], dtype=np.uint64), E, F, A, B, C, rows, cols)
    with pytest.raises(ValueError):
        O.linear_share_at(b, 0, E, F, A, B, C, np.array([1, 2]), np.array([1]))


# ---------------------------------------------------------------------------
# the literal check (Fig. Pi_CompactMatMul verification steps 3-5, Theorem 1)

def _vec(vals, bits):
    return O.from_int(np.array(vals, dtype=object), bits)


def test_literal_check_hand_worked_k4_s4():
    """k = s = 4: shares mod 2^8, the literal sum mod 2^12.

    alpha_i = 13, D^c = (200, 17), m(D^c)_i = (7, 250), chi^ = (9, 14).
      step 3: 13 * 200 = 2600 = 10 * 256 + 40  -> 40;  13 * 17 = 221 -> 221
      step 4: 40 * 9 - 7 * 9 = 360 - 63 = 297;  221 * 14 - 250 * 14 = 3094 - 3500 = -406
      step 5: 297 - 406 = -109 = 3987 mod 4096
    Skipping the step-3 reduction gives 23400 - 63 - 406 = 22931 = 2451 mod 4096,
    reducing the sum mod 2^8 instead gives 147, and swapping the two terms of
    step 4 gives 109: none of them is 3987.
    """
    k = s = 4
    bits = k + s
    got = O.check_compact_literal(k, s, np.array([13], dtype=np.uint64), _vec([9, 14], bits),
                                  _vec([200, 17], bits), _vec([7, 250], bits))
    assert got == 3987
    # the canonical check (mod 2^8) of the same inputs is 147 = 3987 mod 256
    can = O.check_compact(bits, 13, _vec([9, 14], bits), _vec([200, 17], bits), _vec([7, 250], bits))
    assert _ints(can, bits)[0] == 147


def test_literal_check_hand_worked_one_row():
    """k = s = 4, M = 1: alpha_i = 5, D^c = 100, m(D^c) = 1, chi^ = 15.
    step 3: 500 = 256 + 244 -> 244; step 4: 244 * 15 - 15 = 3645; 3645 < 4096."""
    got = O.check_compact_literal(4, 4, np.array([5], dtype=np.uint64), _vec([15], 8), _vec([100], 8),
                                  _vec([1], 8))
    assert got == 3645


@pytest.mark.parametrize("M", [1, 2, 7])
def test_literal_check_special_cases(M):
    """At (k, s) = (32, 32): chi^ = 0 gives 0; alpha_i = 0 gives -chi^.m(D^c)
    mod 2^96; with alpha_i D^c_r < 2^64 for every r the step-3 reduction is the
    identity and the result is the exact integer sum reduced mod 2^96."""
    k, s = 32, 32
    bits = k + s
    rng = np.random.default_rng(M)
    Dc = [int(x) for x in rng.integers(0, 1 << 62, M, dtype=np.uint64)]
    mDc = [int(x) for x in rng.integers(0, 1 << 63, M, dtype=np.uint64)]
    chi = [int(x) for x in rng.integers(1, 1 << 32, M, dtype=np.uint64)]
    assert O.check_compact_literal(k, s, np.array([7], dtype=np.uint64), _vec([0] * M, bits), _vec(Dc, bits),
                                   _vec(mDc, bits)) == 0
    got = O.check_compact_literal(k, s, np.array([0], dtype=np.uint64), _vec(chi, bits), _vec(Dc, bits),
                                  _vec(mDc, bits))
    assert got == (-sum(c * m for c, m in zip(chi, mDc))) % (1 << 96)
    # alpha_i = 3 and D^c < 2^62: alpha_i D^c < 2^64, no step-3 wrap
    got = O.check_compact_literal(k, s, np.array([3], dtype=np.uint64), _vec(chi, bits), _vec(Dc, bits),
                                  _vec(mDc, bits))
    assert got == sum(c * (3 * d - m) for c, d, m in zip(chi, Dc, mDc)) % (1 << 96)


@pytest.mark.parametrize("ring,seed", [(synth.Z64, 1), (synth.Z64, 2), (synth.Ring(4, 4), 3),
                                       (synth.Ring(16, 48), 4)],
                         ids=["k32s32a", "k32s32b", "k4s4", "k16s48"])
def test_literal_check_agrees_with_canonical_mod_2_ks(ring, seed):
    """Both forms sum the same terms; mod 2^{k+s} they are equal, while the
    literal keeps s more bits (unit combiners make the difference visible)."""
    k, s, bits = ring.k, ring.s, ring.bits
    M = 9
    alpha = synth.uniform(seed, 1, 0, (1,), bits)
    chi = synth.uniform(seed, 2, 0, (M,), s)
    Dc = synth.uniform(seed, 3, 0, (M,), bits)
    mDc = synth.uniform(seed, 4, 0, (M,), bits)
    lit = O.check_compact_literal(k, s, alpha, chi, Dc, mDc)
    can = _ints(O.check_compact(bits, alpha, chi, Dc, mDc), bits)[0]
    assert lit % (1 << bits) == can
    assert 0 <= lit < (1 << (k + 2 * s))
    # chi^ = e_r: the literal is ((alpha D^c_r mod 2^{k+s}) - m(D^c)_r) mod 2^{k+2s}
    a = _ints(alpha, bits)[0]
    D = _ints(Dc, bits)
    mD = _ints(mDc, bits)
    for r in (0, M - 1):
        e = [0] * M
        e[r] = 1
        lit = O.check_compact_literal(k, s, alpha, _vec(e, bits), Dc, mDc)
        assert lit == ((a * int(D[r])) % (1 << bits) - int(mD[r])) % (1 << (k + 2 * s))


def test_literal_check_rejects_rings_beyond_128_bits():
    with pytest.raises(ValueError):
        O.check_compact_literal(64, 64, np.array([1, 0], dtype=np.uint64), np.zeros((1, 2), np.uint64),
                                np.zeros((1, 2), np.uint64), np.zeros((1, 2), np.uint64))
