"""Thin ctypes binding of the C ABI in include/mpclinear.h.

Argument marshalling only: torch tensors supply device pointers and the
current CUDA stream; every step of the computation runs in the library's
kernels.  Each function has the C name and raises `MpcError` on a non-zero
status.  If the shared library is missing, loading raises immediately: there
is no fallback path.

Tensors hold ring elements as 64-bit words (torch.int64 bit patterns):
shape (rows, cols) for Z_2^64 and (rows, cols, 2) for Z_2^128 (lo, hi).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

MPC_TAG_FULL, MPC_TAG_COMPACT, MPC_TAG_COMPACT_TRUNC = 0, 1, 2
MPC_CHECK_COMPACT, MPC_CHECK_BATCHREC, MPC_CHECK_BATCHREC_SEEDED = 0, 1, 2
(MPC_WS_SHARE, MPC_WS_TAG_FULL, MPC_WS_TAG_COMPACT, MPC_WS_CHECK_COMPACT, MPC_WS_CHECK_BATCHREC,
 MPC_WS_PUBLIC_PRODUCT, MPC_WS_OPTMAC_TRUNC, MPC_WS_SHARE_TRUNC) = range(8)

# the functions include/mpclinear.h declares
ABI_FUNCTIONS = ("mpc_linear_share", "mpc_linear_tag", "mpc_tag_check", "mpc_workspace_size",
                 "mpc_gemm_path", "mpc_launch_count", "mpc_device_status", "mpc_status_str",
                 "mpc_version",
                 "mpc_linear_tag_compact_noalloc", "mpc_linear_share_trunc", "mpc_public_product",
                 "mpc_optmac_trunc", "mpc_batchrec_mask", "mpc_transpose",
                 "mpc_linear_share_grouped", "mpc_linear_tag_grouped", "mpc_workspace_size_grouped",
                 "mpc_launch_count_grouped", "mpc_autotune", "mpc_autotune_set", "mpc_autotune_choice",
                 "mpc_autotune_save", "mpc_autotune_load", "mpc_autotune_clear", "mpc_selftest_wait", "mpc_lincomb", "mpc_im2col",
                 "mpc_tag_check_grouped", "mpc_lincomb_grouped")
(MPC_E_NULL, MPC_E_SHAPE, MPC_E_RING, MPC_E_ALIGN, MPC_E_WORKSPACE, MPC_E_CUDA, MPC_E_MODE, MPC_E_PARTY,
 MPC_E_TIMEOUT, MPC_E_SCRATCH_LIMIT, MPC_E_IO) = range(-1, -12, -1)
MPC_NOALLOC_SCRATCH_BYTES = 4 << 20


class mpc_ring(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("s", ctypes.c_int32), ("words", ctypes.c_int32)]


class mpc_layer(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("K", ctypes.c_int64), ("N", ctypes.c_int64),
                ("ring", mpc_ring), ("party", ctypes.c_int32), ("nparties", ctypes.c_int32)]


SHARE_PTR_FIELDS = ("E", "F", "A_i", "B_i", "C_i", "Z_i")
TAG_PTR_FIELDS = ("alpha_i", "E", "F", "mA_i", "mB_i", "mC_i", "mR_i", "Dtilde", "chi", "mZ_i", "mDc_i", "Dc")


class mpc_share_ptrs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in SHARE_PTR_FIELDS]


class mpc_tag_ptrs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in TAG_PTR_FIELDS]


CHECK_PTR_FIELDS = ("alpha_i", "chi_hat", "Dc", "mDc_i", "cs_i")


class mpc_check_ptrs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in CHECK_PTR_FIELDS]


class MpcError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn}: status {status}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libmpclinear.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if build_if_missing:
                _build.build()
            else:
                raise RuntimeError(f"libmpclinear.so is not built ({path}); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L = ctypes.POINTER(mpc_layer)
        lib.mpc_linear_share.argtypes = [L] + [P] * 6 + [P, ctypes.c_size_t, P]
        lib.mpc_linear_share.restype = ctypes.c_int
        lib.mpc_linear_tag.argtypes = [L, ctypes.c_int] + [P] * 12 + [P, ctypes.c_size_t, P]
        lib.mpc_linear_tag.restype = ctypes.c_int
        lib.mpc_tag_check.argtypes = [L, ctypes.c_int] + [P] * 5 + [P, ctypes.c_size_t, P]
        lib.mpc_tag_check.restype = ctypes.c_int
        lib.mpc_workspace_size.argtypes = [L, ctypes.c_int]
        lib.mpc_workspace_size.restype = ctypes.c_size_t
        lib.mpc_status_str.argtypes = [ctypes.c_int]
        lib.mpc_status_str.restype = ctypes.c_char_p
        lib.mpc_linear_tag_compact_noalloc.argtypes = [L] + [P] * 12 + [P]
        lib.mpc_linear_tag_compact_noalloc.restype = ctypes.c_int
        lib.mpc_linear_share_trunc.argtypes = [L] + [P] * 6 + [P, ctypes.c_size_t, P]
        lib.mpc_linear_share_trunc.restype = ctypes.c_int
        lib.mpc_public_product.argtypes = [L, P, P, P, P, ctypes.c_size_t, P]
        lib.mpc_public_product.restype = ctypes.c_int
        lib.mpc_optmac_trunc.argtypes = [L, ctypes.c_int] + [P] * 7 + [P]
        lib.mpc_optmac_trunc.restype = ctypes.c_int
        lib.mpc_batchrec_mask.argtypes = [ctypes.POINTER(mpc_ring), ctypes.c_int64, ctypes.c_int64] + \
            [P] * 8 + [P]
        lib.mpc_batchrec_mask.restype = ctypes.c_int
        lib.mpc_lincomb.argtypes = [ctypes.POINTER(mpc_ring), ctypes.c_int64, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_void_p), P, P]
        lib.mpc_lincomb.restype = ctypes.c_int
        lib.mpc_lincomb_grouped.argtypes = [ctypes.POINTER(mpc_ring), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), P]
        lib.mpc_lincomb_grouped.restype = ctypes.c_int
        lib.mpc_tag_check_grouped.argtypes = [L, ctypes.c_int, ctypes.POINTER(mpc_check_ptrs), P]
        lib.mpc_tag_check_grouped.restype = ctypes.c_int
        lib.mpc_im2col.argtypes = [ctypes.POINTER(mpc_ring)] + [ctypes.c_int64] * 4 + [ctypes.c_int] * 3 + [P, P, P]
        lib.mpc_im2col.restype = ctypes.c_int
        lib.mpc_transpose.argtypes = [ctypes.POINTER(mpc_ring), ctypes.c_int64, ctypes.c_int64, P, P, P]
        lib.mpc_transpose.restype = ctypes.c_int
        lib.mpc_linear_share_grouped.argtypes = [L, ctypes.c_int, ctypes.POINTER(mpc_share_ptrs), P,
                                                 ctypes.c_size_t, P]
        lib.mpc_linear_share_grouped.restype = ctypes.c_int
        lib.mpc_linear_tag_grouped.argtypes = [L, ctypes.c_int, ctypes.c_int, ctypes.POINTER(mpc_tag_ptrs), P,
                                               ctypes.c_size_t, P]
        lib.mpc_linear_tag_grouped.restype = ctypes.c_int
        lib.mpc_workspace_size_grouped.argtypes = [L, ctypes.c_int, ctypes.c_int]
        lib.mpc_workspace_size_grouped.restype = ctypes.c_size_t
        lib.mpc_launch_count_grouped.argtypes = [L, ctypes.c_int, ctypes.c_int]
        lib.mpc_launch_count_grouped.restype = ctypes.c_int
        lib.mpc_autotune.argtypes = [L, ctypes.c_int, P]
        lib.mpc_autotune.restype = ctypes.c_int
        lib.mpc_autotune_set.argtypes = [L, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.mpc_autotune_set.restype = ctypes.c_int
        IP = ctypes.POINTER(ctypes.c_int)
        lib.mpc_autotune_choice.argtypes = [L, IP, IP, IP, IP]
        lib.mpc_autotune_choice.restype = ctypes.c_int
        lib.mpc_autotune_save.argtypes = [ctypes.c_char_p]
        lib.mpc_autotune_save.restype = ctypes.c_int
        lib.mpc_autotune_load.argtypes = [ctypes.c_char_p]
        lib.mpc_autotune_load.restype = ctypes.c_int
        lib.mpc_autotune_clear.argtypes = []
        lib.mpc_autotune_clear.restype = ctypes.c_int
        lib.mpc_launch_count.argtypes = [L, ctypes.c_int]
        lib.mpc_launch_count.restype = ctypes.c_int
        lib.mpc_selftest_wait.argtypes = [ctypes.c_longlong, P]
        lib.mpc_selftest_wait.restype = ctypes.c_int
        lib.mpc_device_status.argtypes = []
        lib.mpc_device_status.restype = ctypes.c_int
        lib.mpc_gemm_path.argtypes = [L]
        lib.mpc_gemm_path.restype = ctypes.c_int
        lib.mpc_version.argtypes = []
        lib.mpc_version.restype = ctypes.c_int
        _lib = lib
        return lib


def make_layer(M: int, K: int, N: int, k: int = 32, s: int = 32, party: int = 0,
               nparties: int = 2) -> mpc_layer:
    words = (k + s + 63) // 64
    return mpc_layer(int(M), int(K), int(N), mpc_ring(int(k), int(s), int(words)), int(party),
                     int(nparties))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr() if t.numel() > 0 else None


def _sized(fn, name, t, elems, words):
    """Address of a tensor argument that the call reads or writes as `elems`
    elements of `words` 64-bit words, after checking that the tensor is
    contiguous and holds at least that many bytes: a shorter tensor raises
    ValueError before anything is launched, instead of letting a kernel run
    past its end.  None and raw integer addresses pass through unchecked; the
    caller answers for those, as in C."""
    if t is None or isinstance(t, int):
        return t
    need = int(elems) * words * 8
    if t.nbytes < need or not t.is_contiguous():
        raise ValueError(f"{fn}: {name} must be a contiguous buffer of at least {need} bytes "
                         f"({int(elems)} elements of {words} word(s)); got {tuple(t.shape)} {t.dtype}"
                         + ("" if t.is_contiguous() else ", not contiguous"))
    return t.data_ptr() if t.numel() > 0 else None


def _share_elems(M, K, N):
    return dict(E=M * K, F=K * N, A_i=M * K, B_i=K * N, C_i=M * N, Z_i=M * N)


def _tag_elems(M, K, N, mode):
    e = dict(alpha_i=1, E=M * K, F=K * N, mA_i=M * K, mB_i=K * N, mC_i=M * N, mZ_i=M * N)
    if mode != MPC_TAG_FULL:
        e.update(mR_i=M * N, Dtilde=M * N, chi=N, mDc_i=M, Dc=M)
    return e


def _args(fn, layer, elems, given):
    """Sized addresses of `given` (name -> tensor), in the order of `given`;
    names without an element count (ignored by the call) pass through."""
    w = layer.ring.words
    return [_sized(fn, n, t, elems[n], w) if n in elems else _ptr(t) for n, t in given.items()]


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(fn: str, status: int):
    if status != 0:
        raise MpcError(fn, status, load().mpc_status_str(status).decode())


def mpc_status_str(status: int) -> str:
    return load().mpc_status_str(int(status)).decode()


def mpc_version() -> int:
    return load().mpc_version()


def mpc_gemm_path(layer: mpc_layer) -> int:
    return int(load().mpc_gemm_path(ctypes.byref(layer)))


def mpc_launch_count(layer: mpc_layer, which: int) -> int:
    return int(load().mpc_launch_count(ctypes.byref(layer), int(which)))


def mpc_selftest_wait(limit_cycles: int, stream=None) -> int:
    """Status of the bounded-wait self-test: MPC_E_TIMEOUT when the wait gave up as designed."""
    return int(load().mpc_selftest_wait(int(limit_cycles), _stream(stream)))


def mpc_device_status() -> int:
    """MPC_E_TIMEOUT (-9) if a kernel's bounded wait gave up since the last query."""
    return int(load().mpc_device_status())


def mpc_workspace_size(layer: mpc_layer, which: int) -> int:
    return int(load().mpc_workspace_size(ctypes.byref(layer), int(which)))


def _ws(layer, which, ws, stream=None):
    if ws is not None:
        return _ptr(ws), ws.numel() * ws.element_size()
    need = mpc_workspace_size(layer, which)
    if need == 0:
        return None, 0
    return _alloc_ws(need, stream)


def _alloc_ws(need, stream):
    """A workspace allocated on the call's stream, so that the caching
    allocator orders its reuse after the call; it lives until the next call
    that allocates one."""
    import torch
    if stream is None or isinstance(stream, int):
        buf = torch.empty(need, dtype=torch.uint8, device="cuda")
    else:
        with torch.cuda.stream(stream):
            buf = torch.empty(need, dtype=torch.uint8, device="cuda")
    _alloc_ws.keep = buf
    return buf.data_ptr(), need


def mpc_linear_share(layer, E, F, A_i, B_i, C_i, Z_i, ws=None, stream=None):
    a = _args("mpc_linear_share", layer, _share_elems(layer.M, layer.K, layer.N),
              dict(E=E, F=F, A_i=A_i, B_i=B_i, C_i=C_i, Z_i=Z_i))
    wp, wb = _ws(layer, MPC_WS_SHARE, ws, stream)
    _check("mpc_linear_share", load().mpc_linear_share(ctypes.byref(layer), *a, wp, wb, _stream(stream)))
    return Z_i


def mpc_linear_tag(layer, mode, alpha_i, E, F, mA_i, mB_i, mC_i, mZ_i, mR_i=None, Dtilde=None,
                   chi=None, mDc_i=None, Dc=None, ws=None, stream=None):
    which = MPC_WS_TAG_FULL if mode == MPC_TAG_FULL else MPC_WS_TAG_COMPACT
    a = _args("mpc_linear_tag", layer, _tag_elems(layer.M, layer.K, layer.N, mode),
              dict(alpha_i=alpha_i, E=E, F=F, mA_i=mA_i, mB_i=mB_i, mC_i=mC_i, mR_i=mR_i, Dtilde=Dtilde,
                   chi=chi, mZ_i=mZ_i, mDc_i=mDc_i, Dc=Dc))
    wp, wb = _ws(layer, which, ws, stream)
    _check("mpc_linear_tag", load().mpc_linear_tag(ctypes.byref(layer), int(mode), *a, wp, wb,
                                                   _stream(stream)))
    return mZ_i


def mpc_tag_check(layer, mode, alpha_i, chi_hat, opened, tag_i, cs_i, ws=None, stream=None):
    which = MPC_WS_CHECK_COMPACT if mode == MPC_CHECK_COMPACT else MPC_WS_CHECK_BATCHREC
    fn, w = "mpc_tag_check", layer.ring.words
    n = layer.M if mode == MPC_CHECK_COMPACT else layer.M * layer.N
    # the seeded BATCHREC check reads one 64-bit seed word, not ring elements
    ch = _sized(fn, "chi_hat", chi_hat, 1, 1) if mode == MPC_CHECK_BATCHREC_SEEDED \
        else _sized(fn, "chi_hat", chi_hat, n, w)
    a = [_sized(fn, "alpha_i", alpha_i, 1, w), ch, _sized(fn, "opened", opened, n, w),
         _sized(fn, "tag_i", tag_i, n, w), _sized(fn, "cs_i", cs_i, 1, w)]
    wp, wb = _ws(layer, which, ws, stream)
    _check(fn, load().mpc_tag_check(ctypes.byref(layer), int(mode), *a, wp, wb, _stream(stream)))
    return cs_i


def mpc_linear_tag_compact_noalloc(layer, alpha_i, E, F, mA_i, mB_i, mC_i, mR_i, Dtilde, chi,
                                   mZ_i, mDc_i, Dc, stream=None):
    """CompactTag tag without a workspace: scratch comes from the library's
    static device buffer (see include/mpclinear.h for the rules of use)."""
    fn = "mpc_linear_tag_compact_noalloc"
    a = _args(fn, layer, _tag_elems(layer.M, layer.K, layer.N, MPC_TAG_COMPACT),
              dict(alpha_i=alpha_i, E=E, F=F, mA_i=mA_i, mB_i=mB_i, mC_i=mC_i, mR_i=mR_i, Dtilde=Dtilde,
                   chi=chi, mZ_i=mZ_i, mDc_i=mDc_i, Dc=Dc))
    _check(fn, load().mpc_linear_tag_compact_noalloc(ctypes.byref(layer), *a, _stream(stream)))
    return mZ_i


def mpc_linear_share_trunc(layer, E, F, A_i, B_i, C_i, Z_i, ws=None, stream=None):
    """Truncated layer, step 2: Z_i = C_i + E.B_i + A_i.F for every party."""
    a = _args("mpc_linear_share_trunc", layer, _share_elems(layer.M, layer.K, layer.N),
              dict(E=E, F=F, A_i=A_i, B_i=B_i, C_i=C_i, Z_i=Z_i))
    wp, wb = _ws(layer, MPC_WS_SHARE_TRUNC, ws, stream)
    _check("mpc_linear_share_trunc", load().mpc_linear_share_trunc(ctypes.byref(layer), *a, wp, wb,
                                                                   _stream(stream)))
    return Z_i


def mpc_public_product(layer, E, F, P, ws=None, stream=None):
    """P = E.F (public)."""
    M, K, N = layer.M, layer.K, layer.N
    a = _args("mpc_public_product", layer, dict(E=M * K, F=K * N, P=M * N), dict(E=E, F=F, P=P))
    wp, wb = _ws(layer, MPC_WS_PUBLIC_PRODUCT, ws, stream)
    _check("mpc_public_product", load().mpc_public_product(ctypes.byref(layer), *a, wp, wb, _stream(stream)))
    return P


def mpc_optmac_trunc(layer, f, alpha_i, Rf_i, mRf_i, Dtilde, P, Zf_i, mZf_i, stream=None):
    """Truncated layer, steps 3-4 (OptMAC&Trunc plus the public product term)."""
    MN = layer.M * layer.N
    a = _args("mpc_optmac_trunc", layer, dict(alpha_i=1, Rf_i=MN, mRf_i=MN, Dtilde=MN, P=MN, Zf_i=MN, mZf_i=MN),
              dict(alpha_i=alpha_i, Rf_i=Rf_i, mRf_i=mRf_i, Dtilde=Dtilde, P=P, Zf_i=Zf_i, mZf_i=mZf_i))
    _check("mpc_optmac_trunc", load().mpc_optmac_trunc(ctypes.byref(layer), int(f), *a, _stream(stream)))
    return Zf_i, mZf_i


def mpc_batchrec_mask(k, s, rows, cols, X_i, A_i, R_i, mX_i, mA_i, mR_i, W_i, mW_i, stream=None):
    """Pi_BatchRec open phase step 1: W_i = X_i - A_i + R_i and the same for the tags."""
    ring = mpc_ring(int(k), int(s), (int(k) + int(s) + 63) // 64)
    fn, n = "mpc_batchrec_mask", int(rows) * int(cols)
    a = [_sized(fn, name, t, n, ring.words) for name, t in
         (("X_i", X_i), ("A_i", A_i), ("R_i", R_i), ("mX_i", mX_i), ("mA_i", mA_i), ("mR_i", mR_i),
          ("W_i", W_i), ("mW_i", mW_i))]
    _check(fn, load().mpc_batchrec_mask(ctypes.byref(ring), int(rows), int(cols), *a, _stream(stream)))
    return W_i, mW_i


def mpc_lincomb(k, s, coefs, ins, out, stream=None):
    """out = sum_j coefs[j] * ins[j] (elementwise, mod 2^(k+s)); ins are tensors of out's shape."""
    ring = mpc_ring(int(k), int(s), (int(k) + int(s) + 63) // 64)
    n = out.numel() // ring.words if out is not None and hasattr(out, "numel") else 0
    c = (ctypes.c_int64 * len(coefs))(*[int(x) for x in coefs])
    p = (ctypes.c_void_p * len(ins))(*[_sized("mpc_lincomb", f"ins[{j}]", t, n, ring.words)
                                       for j, t in enumerate(ins)])
    _check("mpc_lincomb", load().mpc_lincomb(ctypes.byref(ring), int(n), len(coefs), c, p,
                                             _sized("mpc_lincomb", "out", out, n, ring.words), _stream(stream)))
    return out


def mpc_lincomb_grouped(k, s, coefs, ins, outs, stream=None, n=None):
    """outs[g] = sum_j coefs[j] * ins[g][j] for every group g (one launch per 64 groups).
    n[g]: ring elements of group g; taken from outs[g] when omitted (tensors),
    required when the buffers are raw addresses."""
    ring = mpc_ring(int(k), int(s), (int(k) + int(s) + 63) // 64)
    G = len(outs)
    if G == 0:
        return outs
    cnt = len(coefs)
    ns = [int(x) for x in n] if n is not None else [o.numel() // ring.words for o in outs]
    nv = (ctypes.c_int64 * G)(*ns)
    c = (ctypes.c_int64 * cnt)(*[int(x) for x in coefs])
    fn = "mpc_lincomb_grouped"
    p = (ctypes.c_void_p * (G * cnt))(*[_sized(fn, f"ins[{g}][{j}]", t, ns[g], ring.words)
                                        for g in range(G) for j, t in enumerate(ins[g])])
    o = (ctypes.c_void_p * G)(*[_sized(fn, f"outs[{g}]", t, ns[g], ring.words) for g, t in enumerate(outs)])
    _check("mpc_lincomb_grouped", load().mpc_lincomb_grouped(ctypes.byref(ring), G, nv, cnt, c, p, o,
                                                             _stream(stream)))
    return outs


def mpc_tag_check_grouped(layers, ptrs, stream=None):
    """Compact check shares of many layers: ptrs[i] is a dict of CHECK_PTR_FIELDS tensors."""
    if not layers:
        return
    arr = (mpc_layer * len(layers))(*layers)
    pa = (mpc_check_ptrs * len(layers))()
    for i, d in enumerate(ptrs):
        L = layers[i]
        elems = dict(alpha_i=1, chi_hat=L.M, Dc=L.M, mDc_i=L.M, cs_i=1)
        for f in CHECK_PTR_FIELDS:
            setattr(pa[i], f, _sized("mpc_tag_check_grouped", f"layers[{i}].{f}", d[f], elems[f], L.ring.words))
    _check("mpc_tag_check_grouped", load().mpc_tag_check_grouped(arr, len(layers), pa, _stream(stream)))


def mpc_im2col(k, s, batch, channels, height, width, f, pad, stride, src, dst, stream=None):
    """dst = the im2col matrix of NCHW images src for an f x f filter (zero padding, stride)."""
    ring = mpc_ring(int(k), int(s), (int(k) + int(s) + 63) // 64)
    src_p, dst_p = _ptr(src), _ptr(dst)
    if f >= 1 and 0 <= pad < f and stride >= 1 and height + 2 * pad >= f and width + 2 * pad >= f:
        # sizes of a valid call (the library rejects the others with MPC_E_SHAPE)
        ho, wo = (height - f + 2 * pad) // stride + 1, (width - f + 2 * pad) // stride + 1
        src_p = _sized("mpc_im2col", "src", src, batch * channels * height * width, ring.words)
        dst_p = _sized("mpc_im2col", "dst", dst, batch * ho * wo * channels * f * f, ring.words)
    _check("mpc_im2col", load().mpc_im2col(ctypes.byref(ring), int(batch), int(channels), int(height), int(width),
                                           int(f), int(pad), int(stride), src_p, dst_p, _stream(stream)))
    return dst


def mpc_transpose(k, s, rows, cols, src, dst, stream=None):
    """dst (cols x rows) = src (rows x cols)^T, ring elements of Z_2^(k+s)."""
    ring = mpc_ring(int(k), int(s), (int(k) + int(s) + 63) // 64)
    n = int(rows) * int(cols)
    _check("mpc_transpose", load().mpc_transpose(ctypes.byref(ring), int(rows), int(cols),
                                                 _sized("mpc_transpose", "src", src, n, ring.words),
                                                 _sized("mpc_transpose", "dst", dst, n, ring.words),
                                                 _stream(stream)))
    return dst


# ---------------------------------------------------------------------------
# grouped calls: `layers` is a list of mpc_layer, `ptrs` a list of dicts keyed
# by the field names of mpc_share_ptrs / mpc_tag_ptrs (tensors or None)

def _layer_array(layers):
    arr = (mpc_layer * len(layers))(*layers)
    return arr


def _ptr_array(cls, fields, ptrs, fn, layers, elems_of):
    """ctypes array of pointer structs; elems_of(layer) gives each field's
    element count (fields it omits are not read by the call)."""
    arr = (cls * len(ptrs))()
    for i, d in enumerate(ptrs):
        L = layers[i]
        elems = elems_of(L)
        for f in fields:
            t = d.get(f)
            setattr(arr[i], f, _sized(fn, f"layers[{i}].{f}", t, elems[f], L.ring.words) if f in elems
                    else _ptr(t))
    return arr


def mpc_workspace_size_grouped(layers, which: int) -> int:
    return int(load().mpc_workspace_size_grouped(_layer_array(layers), len(layers), int(which)))


def mpc_launch_count_grouped(layers, which: int) -> int:
    return int(load().mpc_launch_count_grouped(_layer_array(layers), len(layers), int(which)))


def _ws_grouped(layers, which, ws, stream=None):
    if ws is not None:
        return _ptr(ws), ws.numel() * ws.element_size()
    need = mpc_workspace_size_grouped(layers, which)
    if need == 0:
        return None, 0
    return _alloc_ws(need, stream)


def mpc_linear_share_grouped(layers, ptrs, ws=None, stream=None):
    """Shares of many layers in one call (same results as one mpc_linear_share per layer)."""
    fn = "mpc_linear_share_grouped"
    pa = _ptr_array(mpc_share_ptrs, SHARE_PTR_FIELDS, ptrs, fn, layers, lambda L: _share_elems(L.M, L.K, L.N))
    wp, wb = _ws_grouped(layers, MPC_WS_SHARE, ws, stream)
    _check(fn, load().mpc_linear_share_grouped(_layer_array(layers), len(layers), pa, wp, wb, _stream(stream)))


def mpc_linear_tag_grouped(layers, mode, ptrs, ws=None, stream=None):
    """Tags of many layers in one call (same results as one mpc_linear_tag per layer)."""
    which = MPC_WS_TAG_FULL if mode == MPC_TAG_FULL else MPC_WS_TAG_COMPACT
    fn = "mpc_linear_tag_grouped"
    pa = _ptr_array(mpc_tag_ptrs, TAG_PTR_FIELDS, ptrs, fn, layers, lambda L: _tag_elems(L.M, L.K, L.N, mode))
    wp, wb = _ws_grouped(layers, which, ws, stream)
    _check(fn, load().mpc_linear_tag_grouped(_layer_array(layers), len(layers), int(mode), pa, wp, wb,
                                             _stream(stream)))


# ---------------------------------------------------------------------------
# launch table (autotuner)

def mpc_autotune(layers, stream=None) -> int:
    """Times the GEMM candidates of each distinct layer shape and stores the fastest."""
    if not layers:
        return 0
    n = load().mpc_autotune(_layer_array(layers), len(layers), _stream(stream))
    if n < 0:
        _check("mpc_autotune", n)
    return n


def mpc_autotune_set(layer, path: int, swizzle: int = 8, waves: int = 0, tile_rows: int = None):
    """tile_rows: 128 or 64 for the tensor cores (default 128); 64, 16 or 0 (by grid size) for the
    integer pipes (default 0)."""
    if tile_rows is None:
        tile_rows = 128 if path == 1 else 0
    _check("mpc_autotune_set", load().mpc_autotune_set(ctypes.byref(layer), int(path), int(tile_rows),
                                                       int(swizzle), int(waves)))


def mpc_autotune_choice(layer):
    """(path, swizzle, waves, tuned, tile_rows) the next call for this layer shape would use."""
    p, t, g, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    r = load().mpc_autotune_choice(ctypes.byref(layer), ctypes.byref(p), ctypes.byref(t), ctypes.byref(g),
                                   ctypes.byref(w))
    if r < 0:
        _check("mpc_autotune_choice", r)
    return p.value, g.value, w.value, bool(r), t.value


def mpc_autotune_save(path: str) -> int:
    n = load().mpc_autotune_save(os.fsencode(path))
    if n < 0:
        _check("mpc_autotune_save", n)
    return n


def mpc_autotune_load(path: str) -> int:
    n = load().mpc_autotune_load(os.fsencode(path))
    if n < 0:
        _check("mpc_autotune_load", n)
    return n


def mpc_autotune_clear() -> int:
    return int(load().mpc_autotune_clear())
