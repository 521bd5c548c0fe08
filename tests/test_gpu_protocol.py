"""The whole per-layer protocol with every party simulated on the device:
openings by mpc_lincomb (E = sum_i (X_i - A_i), F = sum_i (Y_i - B_i),
D~ = sum_i (R_i - Z_i), the check sum), shares and both tags by the layer
calls.  The openings equal the trusted dealer's, the reconstructed share is
X.Y, the tags satisfy the MAC relation, an honest check sums to zero and a
tampered share fails it."""
import numpy as np
import pytest

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


def split(ring, V, n, seed, tid):
    """n additive shares of V (the last one fixes the sum)."""
    shares = [synth.uniform(seed, tid, i + 1, V.shape[:2], ring.bits) for i in range(n - 1)]
    last = V.copy()
    for s_ in shares:
        last = O.sub(ring.bits, last, s_)
    return shares + [last]


def run_device(ring, d, Xs, Ys, tamper=False):
    k, s, w = ring.k, ring.s, ring.words
    M, K, N, n = d.M, d.K, d.N, len(d.parties)
    P = d.parties
    E = empty_like_ring((M, K), w)
    F = empty_like_ring((K, N), w)
    abi.mpc_lincomb(k, s, [1, -1] * n, [t for i in range(n) for t in (dev(Xs[i]), dev(P[i].A))], E)
    abi.mpc_lincomb(k, s, [1, -1] * n, [t for i in range(n) for t in (dev(Ys[i]), dev(P[i].B))], F)
    Z, mZf = [], []
    for i, p in enumerate(P):
        L = abi.make_layer(M, K, N, k, s, i, n)
        z = empty_like_ring((M, N), w)
        abi.mpc_linear_share(L, E, F, dev(p.A), dev(p.B), dev(p.C), z)
        Z.append(z)
        t = empty_like_ring((M, N), w)
        abi.mpc_linear_tag(L, abi.MPC_TAG_FULL, dev(p.alpha), E, F, dev(p.mA), dev(p.mB), dev(p.mC), t)
        mZf.append(t)
    if tamper:
        z0 = host(Z[0])
        flat = z0.reshape(-1, w)
        flat[3] = O.from_int(O.to_int(flat[3], ring.bits) + 1, ring.bits)
        Z[0] = dev(z0)
    Dt = empty_like_ring((M, N), w)
    abi.mpc_lincomb(k, s, [1, -1] * n, [t for i in range(n) for t in (dev(P[i].R), Z[i])], Dt)
    cs = []
    for i, p in enumerate(P):
        L = abi.make_layer(M, K, N, k, s, i, n)
        mZ = empty_like_ring((M, N), w)
        mDc = empty_like_ring((M,), w)
        Dc = empty_like_ring((M,), w)
        abi.mpc_linear_tag(L, abi.MPC_TAG_COMPACT, dev(p.alpha), E, F, dev(p.mA), dev(p.mB), dev(p.mC), mZ,
                           mR_i=dev(p.mR), Dtilde=Dt, chi=dev(d.chi), mDc_i=mDc, Dc=Dc)
        c = empty_like_ring((1,), w)
        abi.mpc_tag_check(L, abi.MPC_CHECK_COMPACT, dev(p.alpha), dev(d.chi_hat), Dc, mDc, c)
        cs.append(c)
    total = empty_like_ring((1,), w)
    abi.mpc_lincomb(k, s, [1] * n, cs, total)
    return host(E), host(F), [host(z) for z in Z], [host(t) for t in mZf], host(Dt), host(total)


@pytest.mark.parametrize("ring,shape,n", [(synth.Z64, (128, 256, 96), 2), (synth.Z128, (64, 96, 48), 3),
                                          (synth.Z64, (5, 33, 7), 4)],
                         ids=lambda x: str(x) if isinstance(x, (tuple, int)) else None)
def test_protocol_on_device(ring, shape, n):
    M, K, N = shape
    bits = ring.bits
    d = dealer.deal(ring, M, K, N, n=n, seed=M + K + N + n)
    Xs = split(ring, d.X, n, 17, 900)
    Ys = split(ring, d.Y, n, 17, 901)
    E, F, Z, mZf, Dt, total = run_device(ring, d, Xs, Ys)
    assert np.array_equal(E, d.E) and np.array_equal(F, d.F)
    Zsum = dealer.total(bits, Z)
    assert np.array_equal(Zsum, O.ring_gemm(bits, d.X, d.Y))          # reconstruction I1
    assert np.array_equal(dealer.total(bits, mZf), O.smul(bits, d.alpha, Zsum))   # MAC relation I2
    ref = dealer.run_layer(d)
    assert np.array_equal(Dt, ref["Dt"])
    assert not O.to_int(total, bits).any()                              # honest check passes
    *_, bad = run_device(ring, d, Xs, Ys, tamper=True)
    assert O.to_int(bad, bits).any()                                    # tampered share caught
    assert abi.mpc_device_status() == 0


@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=["z64", "z128"])
@pytest.mark.parametrize("n_elems", [1, 7, 4096, 100001])
def test_lincomb_parity(ring, n_elems):
    bits = ring.bits
    ins = [synth.uniform(9, 30 + j, 0, (n_elems,), bits) for j in range(5)]
    coefs = [1, -1, 3, -7, 0]
    out = empty_like_ring((n_elems,), ring.words)
    abi.mpc_lincomb(ring.k, ring.s, coefs, [dev(x) for x in ins], out)
    want = ins[0]
    want = O.sub(bits, want, ins[1])
    want = O.add(bits, want, O.smul(bits, O.from_int(np.array([3], dtype=object), bits), ins[2]))
    want = O.sub(bits, want, O.smul(bits, O.from_int(np.array([7], dtype=object), bits), ins[3]))
    assert np.array_equal(host(out), want)
