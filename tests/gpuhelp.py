"""Helpers for the GPU tests: move ring-element arrays between numpy (uint64
storage) and torch device tensors (int64 bit patterns), and run one party's
layer through the C ABI."""
from __future__ import annotations

import numpy as np

from paper_2311_04406_gb300 import abi


def dev(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def host(t) -> np.ndarray:
    return np.ascontiguousarray(t.cpu().numpy().view(np.uint64))


def empty_like_ring(shape, words):
    import torch
    full = tuple(shape) + ((2,) if words == 2 else ())
    return torch.empty(full, dtype=torch.int64, device="cuda")


def gpu_share(ring, party, E, F, A, B, C, nparties=2):
    M, K = E.shape[:2]
    N = F.shape[1]
    L = abi.make_layer(M, K, N, ring.k, ring.s, party, nparties)
    Z = empty_like_ring((M, N), ring.words)
    abi.mpc_linear_share(L, dev(E), dev(F), dev(A), dev(B), dev(C), Z)
    return host(Z)


def gpu_tag_full(ring, party, alpha, E, F, mA, mB, mC, nparties=2):
    M, K = E.shape[:2]
    N = F.shape[1]
    L = abi.make_layer(M, K, N, ring.k, ring.s, party, nparties)
    mZ = empty_like_ring((M, N), ring.words)
    abi.mpc_linear_tag(L, abi.MPC_TAG_FULL, dev(alpha), dev(E), dev(F), dev(mA), dev(mB), dev(mC), mZ)
    return host(mZ)


def gpu_tag_compact(ring, party, alpha, E, F, mA, mB, mC, mR, Dt, chi, nparties=2):
    M, K = E.shape[:2]
    N = F.shape[1]
    L = abi.make_layer(M, K, N, ring.k, ring.s, party, nparties)
    mZ = empty_like_ring((M, N), ring.words)
    mDc = empty_like_ring((M,), ring.words)
    Dc = empty_like_ring((M,), ring.words)
    abi.mpc_linear_tag(L, abi.MPC_TAG_COMPACT, dev(alpha), dev(E), dev(F), dev(mA), dev(mB), dev(mC),
                       mZ, mR_i=dev(mR), Dtilde=dev(Dt), chi=dev(chi), mDc_i=mDc, Dc=Dc)
    return host(mZ), host(mDc), host(Dc)


def gpu_check_compact(ring, alpha, chi_hat, Dc, mDc):
    M = Dc.shape[0]
    L = abi.make_layer(M, 1, 1, ring.k, ring.s)
    cs = empty_like_ring((1,), ring.words)
    abi.mpc_tag_check(L, abi.MPC_CHECK_COMPACT, dev(alpha), dev(chi_hat), dev(Dc), dev(mDc), cs)
    return host(cs)


def gpu_check_batchrec(ring, alpha, chi, W, mW):
    M, N = W.shape[:2]
    L = abi.make_layer(M, 1, N, ring.k, ring.s)
    cs = empty_like_ring((1,), ring.words)
    abi.mpc_tag_check(L, abi.MPC_CHECK_BATCHREC, dev(alpha), dev(chi), dev(W), dev(mW), cs)
    return host(cs)


def gpu_share_trunc(ring, party, E, F, A, B, C, nparties=2):
    M, K = E.shape[:2]
    N = F.shape[1]
    L = abi.make_layer(M, K, N, ring.k, ring.s, party, nparties)
    Z = empty_like_ring((M, N), ring.words)
    abi.mpc_linear_share_trunc(L, dev(E), dev(F), dev(A), dev(B), dev(C), Z)
    return host(Z)


def gpu_public_product(ring, E, F):
    M, K = E.shape[:2]
    N = F.shape[1]
    L = abi.make_layer(M, K, N, ring.k, ring.s)
    P = empty_like_ring((M, N), ring.words)
    abi.mpc_public_product(L, dev(E), dev(F), P)
    return host(P)


def gpu_optmac_trunc(ring, party, f, alpha, Rf, mRf, Dt, P, nparties=2):
    M, N = Rf.shape[:2]
    L = abi.make_layer(M, 1, N, ring.k, ring.s, party, nparties)
    Zf = empty_like_ring((M, N), ring.words)
    mZf = empty_like_ring((M, N), ring.words)
    abi.mpc_optmac_trunc(L, f, dev(alpha), dev(Rf), dev(mRf), dev(Dt), dev(P), Zf, mZf)
    return host(Zf), host(mZf)


def gpu_tag_compact_trunc(ring, party, alpha, E, F, mA, mB, mC, mR, Dt, chi, nparties=2):
    M, K = E.shape[:2]
    N = F.shape[1]
    L = abi.make_layer(M, K, N, ring.k, ring.s, party, nparties)
    mDc = empty_like_ring((M,), ring.words)
    Dc = empty_like_ring((M,), ring.words)
    abi.mpc_linear_tag(L, abi.MPC_TAG_COMPACT_TRUNC, dev(alpha), dev(E), dev(F), dev(mA), dev(mB),
                       dev(mC), None, mR_i=dev(mR), Dtilde=dev(Dt), chi=dev(chi), mDc_i=mDc, Dc=Dc)
    return host(mDc), host(Dc)
