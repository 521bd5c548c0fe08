"""Operation-count model of the tag computation (§3.4.3) and ring parameters.

Host logic only: closed forms the paper prints, used by the benchmark to put
the measured tag-overhead ratio beside the paper's multiplication counts.
"""
from __future__ import annotations

import math


def full_tag_mults(M: int, K: int, N: int) -> int:
    """Local multiplications of Eq. (compute-ztag): at most 3 T1T2T3 + T1T3."""
    return 3 * M * K * N + M * N


def compact_tag_mults(M: int, K: int, N: int) -> int:
    """Local multiplications of the CompactTag tag: 4 T1T3 + 2 T2T3 + 3 T1T2 + T1."""
    return 4 * M * N + 2 * K * N + 3 * M * K + M


def tag_mult_ratio(M: int, K: int, N: int) -> float:
    return full_tag_mults(M, K, N) / compact_tag_mults(M, K, N)


def sigma(s: int) -> int:
    """sigma = s - log2(s + 1), rounded down (§4.1 prints 26 for s=32, 57 for s=64)."""
    return math.floor(s - math.log2(s + 1))


def check_failure_bound(s: int) -> float:
    """Theorem 1: an error escapes the compact check with probability <= 2^(-s+log2(s+1))."""
    return 2.0 ** (-s + math.log2(s + 1))


def digit_count(ring_bits: int, digit_bits: int = 8) -> int:
    return -(-ring_bits // digit_bits)


def digit_products(ring_bits: int, digit_bits: int = 8) -> int:
    """Digit products (i, j) with weight 2^(digit_bits (i + j)) below 2^ring_bits.

    A product mod 2^b of two b-bit numbers split into n = b / digit_bits digits
    needs the pairs i + j <= n - 1: n (n + 1) / 2 of them (36 for Z_2^64 and 136
    for Z_2^128 with 8-bit digits).
    """
    n = digit_count(ring_bits, digit_bits)
    return sum(1 for i in range(n) for j in range(n) if i + j <= n - 1)
