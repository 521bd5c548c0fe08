"""CPU oracle for the CompactTag linear layer -- TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package.  The CUDA library never calls it and shares no code
with it.  The arithmetic lives in `oracle.c` (plain loops over wrapping
unsigned __int128, one sequential sum per output element); this module only
marshals numpy arrays into it.

Storage convention: ring elements of Z_{2^b} are numpy uint64 arrays, shape
`(..., )` for b <= 64 and `(..., 2)` holding (lo, hi) for 64 < b <= 128.

Parity of every function is pinned in `tests/test_oracle*.py` against what the
paper and the mathematics fix (a textbook product on the reduction n=1, the MAC
relation, closed forms, special cases, cases worked by hand and tamper
detection).  The sampled checkers `linear_share_at` / `linear_tag_full_at` are
pinned element by element against the full functions, and the literal
mod 2^{k+2s} check (`check_compact_literal`) by a hand-worked case at k = s = 4
and its special cases (`tests/test_oracle_pins.py`); the paper's printed form
fails on honest inputs, which a test records.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-std=gnu11", "-shared", "-fPIC",
                        _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            sig = {
                "orc_words": (_int, [_int]),
                "orc_add": (None, [_int, _i64, _u64p, _u64p, _u64p]),
                "orc_sub": (None, [_int, _i64, _u64p, _u64p, _u64p]),
                "orc_smul": (None, [_int, _i64, _u64p, _u64p, _u64p]),
                "orc_reduce": (None, [_int, _i64, _u64p, _u64p]),
                "orc_ring_gemm": (None, [_int, _i64, _i64, _i64, _u64p, _u64p, _u64p]),
                "orc_linear_share": (None, [_int, _i64, _i64, _i64, _int] + [_u64p] * 6),
                "orc_linear_share_at": (None, [_int, _i64, _i64, _i64, _int] + [_u64p] * 5
                                        + [_i64, _i64p, _i64p, _u64p]),
                "orc_linear_tag_full": (None, [_int, _i64, _i64, _i64] + [_u64p] * 7),
                "orc_linear_tag_full_at": (None, [_int, _i64, _i64, _i64] + [_u64p] * 6
                                           + [_i64, _i64p, _i64p, _u64p]),
                "orc_optmac": (None, [_int, _i64, _i64, _u64p, _u64p, _u64p, _u64p]),
                "orc_compress": (None, [_int, _i64, _i64, _u64p, _u64p, _u64p]),
                "orc_compact_tag": (_int, [_int, _i64, _i64, _i64] + [_u64p] * 12),
                "orc_check_compact": (None, [_int, _i64] + [_u64p] * 5),
                "orc_linear_share_trunc": (None, [_int, _i64, _i64, _i64] + [_u64p] * 6),
                "orc_batchrec_mask": (None, [_int, _i64] + [_u64p] * 8),
                "orc_chi_seeded": (None, [_int, _int, ctypes.c_uint64, _i64, _u64p]),
                "orc_optmac_trunc": (None, [_int, _int, _i64, _i64, _int, _int] + [_u64p] * 7),
                "orc_compact_tag_trunc": (_int, [_int, _i64, _i64, _i64] + [_u64p] * 12),
                "orc_check_compact_literal": (_int, [_int, _int, _i64] + [_u64p] * 5),
                "orc_check_batchrec": (None, [_int, _i64, _i64] + [_u64p] * 5),
                "orc_im2col": (None, [_int, _i64, _i64, _i64, _i64, _int, _int, _int, _u64p, _u64p]),
                "orc_set_threads": (_int, [_int]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"], "oracle wants C-contiguous uint64"
    return a.ctypes.data_as(_u64p)


def words(bits: int) -> int:
    return 1 if bits <= 64 else 2


def _new(bits: int, *shape) -> np.ndarray:
    w = words(bits)
    return np.zeros(tuple(shape) + ((2,) if w == 2 else ()), dtype=np.uint64)


def _n(a: np.ndarray, bits: int) -> int:
    return a.size // words(bits)


def _scalar(x, bits: int) -> np.ndarray:
    """A ring scalar as a 1-element storage array (accepts int or array)."""
    if isinstance(x, np.ndarray):
        return np.ascontiguousarray(x.reshape(-1)[: words(bits)].astype(np.uint64))
    x = int(x) % (1 << bits)
    if words(bits) == 1:
        return np.array([x], dtype=np.uint64)
    return np.array([x & (2**64 - 1), x >> 64], dtype=np.uint64)


def to_int(a: np.ndarray, bits: int):
    """Storage array -> Python int (scalar) or object array of ints."""
    a = np.asarray(a, dtype=np.uint64)
    if words(bits) == 1:
        return a.astype(object) if a.ndim else int(a)
    if a.ndim == 1:
        return int(a[0]) + (int(a[1]) << 64)
    lo = a[..., 0].astype(object)
    hi = a[..., 1].astype(object)
    return lo + (hi << 64)


def from_int(v, bits: int) -> np.ndarray:
    """Object array (or int) of Python ints -> storage array, reduced mod 2^bits."""
    v = np.asarray(v, dtype=object)
    m = (1 << bits) - 1
    v = np.vectorize(lambda x: int(x) & m, otypes=[object])(v) if v.size else v
    if words(bits) == 1:
        return np.ascontiguousarray(v.astype(np.uint64))
    lo = np.vectorize(lambda x: x & (2**64 - 1), otypes=[object])(v) if v.size else v
    hi = np.vectorize(lambda x: x >> 64, otypes=[object])(v) if v.size else v
    return np.ascontiguousarray(np.stack([lo.astype(np.uint64), hi.astype(np.uint64)], axis=-1))


# ---------------------------------------------------------------------------
# elementwise

def add(bits, x, y):
    out = np.empty_like(x); _load().orc_add(bits, _n(x, bits), _p(x), _p(y), _p(out)); return out


def sub(bits, x, y):
    out = np.empty_like(x); _load().orc_sub(bits, _n(x, bits), _p(x), _p(y), _p(out)); return out


def smul(bits, c, x):
    out = np.empty_like(x)
    _load().orc_smul(bits, _n(x, bits), _p(_scalar(c, bits)), _p(x), _p(out))
    return out


def reduce(bits, x):
    out = np.empty_like(x); _load().orc_reduce(bits, _n(x, bits), _p(x), _p(out)); return out


# ---------------------------------------------------------------------------
# the hot path's quantities

def ring_gemm(bits, X, Y):
    M, K = X.shape[:2]
    N = Y.shape[1]
    out = _new(bits, M, N)
    _load().orc_ring_gemm(bits, M, K, N, _p(X), _p(Y), _p(out))
    return out


def linear_share(bits, party, E, F, A, B, C):
    """a1: [Z]_i = [C]_i + E.[B]_i + [A]_i.F (+ E.F for party 0)."""
    M, K = E.shape[:2]
    N = F.shape[1]
    out = _new(bits, M, N)
    _load().orc_linear_share(bits, M, K, N, int(party), _p(E), _p(F), _p(A), _p(B), _p(C), _p(out))
    return out


def _positions(M, N, rows, cols):
    """Sampled positions as int64 arrays; every (row, col) must lie in the M x N output."""
    rows = np.ascontiguousarray(rows, dtype=np.int64).reshape(-1)
    cols = np.ascontiguousarray(cols, dtype=np.int64).reshape(-1)
    if rows.size != cols.size:
        raise ValueError("rows and cols must have the same length")
    if rows.size and (rows.min() < 0 or rows.max() >= M or cols.min() < 0 or cols.max() >= N):
        raise IndexError(f"sampled position outside the {M} x {N} output")
    return rows, cols


def linear_share_at(bits, party, E, F, A, B, C, rows, cols):
    """a1 at the positions (rows[j], cols[j]) only."""
    M, K = E.shape[:2]
    N = F.shape[1]
    rows, cols = _positions(M, N, rows, cols)
    out = _new(bits, rows.size)
    _load().orc_linear_share_at(bits, M, K, N, int(party), _p(E), _p(F), _p(A), _p(B), _p(C),
                                rows.size, rows.ctypes.data_as(_i64p), cols.ctypes.data_as(_i64p),
                                _p(out))
    return out


def linear_tag_full(bits, alpha, E, F, mA, mB, mC):
    """a2: [m(Z)]_i = [m(C)]_i + E.[m(B)]_i + [m(A)]_i.F + alpha_i (E.F)."""
    M, K = E.shape[:2]
    N = F.shape[1]
    out = _new(bits, M, N)
    _load().orc_linear_tag_full(bits, M, K, N, _p(_scalar(alpha, bits)), _p(E), _p(F), _p(mA),
                                _p(mB), _p(mC), _p(out))
    return out


def linear_tag_full_at(bits, alpha, E, F, mA, mB, mC, rows, cols):
    """a2 at the positions (rows[j], cols[j]) only."""
    M, K = E.shape[:2]
    N = F.shape[1]
    rows, cols = _positions(M, N, rows, cols)
    out = _new(bits, rows.size)
    _load().orc_linear_tag_full_at(bits, M, K, N, _p(_scalar(alpha, bits)), _p(E), _p(F), _p(mA),
                                   _p(mB), _p(mC), rows.size, rows.ctypes.data_as(_i64p),
                                   cols.ctypes.data_as(_i64p), _p(out))
    return out


def optmac(bits, alpha, mR, Dt):
    """a3: [m(Z)]_i = [m(R)]_i - alpha_i * D~."""
    M, N = mR.shape[:2]
    out = _new(bits, M, N)
    _load().orc_optmac(bits, M, N, _p(_scalar(alpha, bits)), _p(mR), _p(Dt), _p(out))
    return out


def compress(bits, Mat, chi):
    """a4: Mat . chi (Fig. Pi_Compress)."""
    rows, cols = Mat.shape[:2]
    out = _new(bits, rows)
    _load().orc_compress(bits, rows, cols, _p(Mat), _p(chi), _p(out))
    return out


def compact_tag(bits, alpha, E, F, mA, mB, mC, mR, Dt, chi):
    """a4 + a5: returns (mDc, Dc, mZc), each an M-vector."""
    M, K = E.shape[:2]
    N = F.shape[1]
    mDc, Dc, mZc = _new(bits, M), _new(bits, M), _new(bits, M)
    rc = _load().orc_compact_tag(bits, M, K, N, _p(_scalar(alpha, bits)), _p(E), _p(F), _p(mA),
                                 _p(mB), _p(mC), _p(mR), _p(Dt), _p(chi), _p(mDc), _p(Dc), _p(mZc))
    if rc != 0:
        raise MemoryError("oracle compact_tag: allocation failed")
    return mDc, Dc, mZc


def check_compact(bits, alpha, chi_hat, Dc, mDc):
    """a6: cs_i = sum_r chi^_r (alpha_i Dc_r - mDc_r) mod 2^{k+s}."""
    M = Dc.shape[0]
    out = _new(bits, 1)
    _load().orc_check_compact(bits, M, _p(_scalar(alpha, bits)), _p(chi_hat), _p(Dc), _p(mDc), _p(out))
    return out


def check_compact_literal(k, s, alpha, chi_hat, Dc, mDc) -> int:
    """The printed mod 2^{k+2s} form of the check share (Fig. Pi_CompactMatMul
    verification steps 3-5): alpha_i D^c reduced mod 2^{k+s}, then the chi^
    combination summed mod 2^{k+2s}."""
    bits = k + s
    M = Dc.shape[0]
    out = np.zeros(2, dtype=np.uint64)
    rc = _load().orc_check_compact_literal(k, s, M, _p(_scalar(alpha, bits)), _p(chi_hat), _p(Dc),
                                           _p(mDc), _p(out))
    if rc != 0:
        raise ValueError("literal check needs k + 2s <= 128")
    return int(out[0]) + (int(out[1]) << 64)


def check_batchrec(bits, alpha, chi, W, mW):
    """Fig. Pi_BatchRec tag check share: sum chi * (m(W)_i - alpha_i W)."""
    M, N = W.shape[:2]
    out = _new(bits, 1)
    _load().orc_check_batchrec(bits, M, N, _p(_scalar(alpha, bits)), _p(chi), _p(W), _p(mW), _p(out))
    return out


# ---------------------------------------------------------------------------
# truncated layer (Fig. Pi_OptMAC&Trunc, Fig. Pi_CompactMatMul)

def linear_share_trunc(bits, E, F, A, B, C):
    """Step 2: [Z]_i = [C]_i + E.[B]_i + [A]_i.F for every party (no E.F)."""
    M, K = E.shape[:2]
    N = F.shape[1]
    out = _new(bits, M, N)
    _load().orc_linear_share_trunc(bits, M, K, N, _p(E), _p(F), _p(A), _p(B), _p(C), _p(out))
    return out


def public_product(bits, E, F):
    """The public E.F (computed by every party from opened values)."""
    return ring_gemm(bits, E, F)


def optmac_trunc(k, s, f, party, alpha, Rf, mRf, Dt, P):
    """Steps 3-4: returns ([Z^f]_i, [m(Z^f)]_i)."""
    bits = k + s
    M, N = Rf.shape[:2]
    Zf, mZf = _new(bits, M, N), _new(bits, M, N)
    _load().orc_optmac_trunc(k, s, M, N, int(f), int(party), _p(_scalar(alpha, bits)), _p(Rf), _p(mRf),
                             _p(Dt), _p(P), _p(Zf), _p(mZf))
    return Zf, mZf


def compact_tag_trunc(bits, alpha, E, F, mA, mB, mC, mR, Dt, chi):
    """Steps 6-7 (no E.U^c term): returns (mDc, Dc, mZc)."""
    M, K = E.shape[:2]
    N = F.shape[1]
    mDc, Dc, mZc = _new(bits, M), _new(bits, M), _new(bits, M)
    rc = _load().orc_compact_tag_trunc(bits, M, K, N, _p(_scalar(alpha, bits)), _p(E), _p(F), _p(mA),
                                       _p(mB), _p(mC), _p(mR), _p(Dt), _p(chi), _p(mDc), _p(Dc), _p(mZc))
    if rc != 0:
        raise MemoryError("oracle compact_tag_trunc: allocation failed")
    return mDc, Dc, mZc


# ---------------------------------------------------------------------------
# Pi_BatchRec open phase and seeded combiners

def batchrec_mask(bits, X, A, R, mX, mA, mR):
    """([W]_i, [m(W)]_i) = ([X]_i - [A]_i + [R]_i, [m(X)]_i - [m(A)]_i + [m(R)]_i)."""
    W, mW = np.empty_like(X), np.empty_like(X)
    _load().orc_batchrec_mask(bits, _n(X, bits), _p(X), _p(A), _p(R), _p(mX), _p(mA), _p(mR),
                              _p(W), _p(mW))
    return W, mW


def chi_seeded(bits, s, seed, shape):
    """Public combiners in [0, 2^s), s <= 64: the SplitMix64 sequence started at `seed`."""
    if not 1 <= s <= 64:
        raise ValueError("combiners are drawn from Z_2^s with s <= 64")
    shape = tuple(shape)
    out = _new(bits, *shape)
    n = int(np.prod(shape, dtype=np.int64)) if shape else 1
    _load().orc_chi_seeded(bits, s, int(seed) & 0xFFFFFFFFFFFFFFFF, n, _p(out))
    return out


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's loops; returns the previous maximum."""
    return int(_load().orc_set_threads(int(n)))


def im2col(x: np.ndarray, f: int, pad: int, stride: int, bits: int) -> np.ndarray:
    """im2col view of NCHW ring-element images x for an f x f convolution (§2.6)."""
    w = words(bits)
    B, C, H, W = x.shape[:4]
    Ho, Wo = (H - f + 2 * pad) // stride + 1, (W - f + 2 * pad) // stride + 1
    out = _new(bits, B * Ho * Wo, C * f * f)
    xc = np.ascontiguousarray(x)
    _load().orc_im2col(w, B, C, H, W, f, pad, stride, _p(xc), _p(out))
    return out
