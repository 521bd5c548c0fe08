"""Pins of training's backward linear layers through the oracle (§4 training
workloads): grad X = G . W^T and grad W = X^T . G as two more Beaver products,
with each party's transposed shares of the forward masks (mask reuse).

Independent routes: the gradients written out as index loops over Python
integers (W^T[n][k] read as W[k][n], X^T[k][m] as X[m][k], no transposed array
involved), the MAC relation of §2.4, the compact check's honest pass and its
tamper failure, and the relations the reused masks must satisfy.
"""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import dealer

RINGS = [synth.Z64, synth.Z128]


def ints(a, bits):
    return O.to_int(a, bits)


def grad_x(G, W, bits):
    M, N = G.shape
    K = W.shape[0]
    return np.array([[sum(int(G[m][n]) * int(W[k][n]) for n in range(N)) % (1 << bits)
                      for k in range(K)] for m in range(M)], dtype=object)


def grad_w(X, G, bits):
    M, K = X.shape
    N = G.shape[1]
    return np.array([[sum(int(X[m][k]) * int(G[m][n]) for m in range(M)) % (1 << bits)
                      for n in range(N)] for k in range(K)], dtype=object)


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}")
@pytest.mark.parametrize("n", [1, 2, 3])
def test_backward_shares_reconstruct_gradients(ring, n):
    bits = ring.bits
    d = dealer.deal(ring, 4, 6, 5, n=n, seed=70 + n)
    b = dealer.deal_backward(d, seed=70 + n)
    G, X, W = ints(b.G, bits), ints(d.X, bits), ints(d.Y, bits)
    out_x = dealer.run_layer(b.dX)
    out_w = dealer.run_layer(b.dW)
    assert np.array_equal(ints(dealer.total(bits, out_x["Z"]), bits), grad_x(G, W, bits))
    assert np.array_equal(ints(dealer.total(bits, out_w["Z"]), bits), grad_w(X, G, bits))


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: f"k{r.k}")
def test_backward_tags(ring):
    bits = ring.bits
    d = dealer.deal(ring, 5, 3, 4, n=2, seed=81)
    b = dealer.deal_backward(d, seed=81)
    a = ints(d.alpha, bits)[0]
    for layer in (b.dX, b.dW):
        out = dealer.run_layer(layer)
        Z = ints(dealer.total(bits, out["Z"]), bits)
        want = np.vectorize(lambda v: int(v) * int(a) % (1 << bits), otypes=[object])(Z)
        assert np.array_equal(ints(dealer.total(bits, out["mZ_full"]), bits), want)
        assert np.array_equal(ints(dealer.total(bits, out["mZ_opt"]), bits), want)
        assert not ints(out["cs_total"], bits).any()


def test_backward_masks_are_reused_consistently():
    ring = synth.Z64
    bits = ring.bits
    d = dealer.deal(ring, 3, 5, 4, n=3, seed=90)
    b = dealer.deal_backward(d, seed=90)
    # the public openings of the backward products are the forward ones
    # transposed and one new opening of G, shared by both products
    assert np.array_equal(b.dX.F, d.F.T)
    assert np.array_equal(b.dW.E, d.E.T)
    assert np.array_equal(b.dX.E, b.dW.F)
    # each opening is operand minus mask
    for L in (b.dX, b.dW):
        assert np.array_equal(L.E, O.sub(bits, L.X, L.A))
        assert np.array_equal(L.F, O.sub(bits, L.Y, L.B))
        assert np.array_equal(L.C, O.ring_gemm(bits, L.A, L.B))
        for i, p in enumerate(L.parties):
            assert p.A.shape[:2] == (L.M, L.K) and p.B.shape[:2] == (L.K, L.N)
    # the party's share of B^T is its forward share of B transposed
    for p, q in zip(d.parties, b.dX.parties):
        for kk in range(d.K):
            for nn in range(d.N):
                assert q.B[nn, kk] == p.B[kk, nn] and q.mB[nn, kk] == p.mB[kk, nn]


@pytest.mark.parametrize("which", ["dX", "dW"])
def test_backward_tamper_detected(which):
    ring = synth.Z64
    bits = ring.bits
    caught = 0
    for seed in range(8):
        d = dealer.deal(ring, 3, 4, 5, n=2, seed=200 + seed)
        layer = getattr(dealer.deal_backward(d, seed=200 + seed), which)
        out = dealer.run_layer(layer, tamper={"Dt": (seed % (layer.M * layer.N), 1 + seed)})
        caught += int(ints(out["cs_total"], bits).any())
    assert caught == 8


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 7, 3), (9, 2, 1)], ids=str)
def test_transpose_storage(shape):
    M, K, _ = shape
    for bits in (64, 128):
        a = synth.uniform(5, 1, 0, (M, K), bits)
        t = dealer.transpose(a)
        assert t.shape[:2] == (K, M) and t.flags.c_contiguous
        for m in range(M):
            for k in range(K):
                assert np.array_equal(t[k, m], a[m, k])
