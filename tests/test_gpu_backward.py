"""GPU parity of training's backward linear layers (grad X = G . W^T,
grad W = X^T . G, §4 training workloads): each party transposes its forward
mask shares and the public openings on the device (mpc_transpose), then runs
the forward layer kernels on the transposed shapes.  Every output equals the
oracle's bit for bit; the oracle transposes with numpy on the host."""
import numpy as np
import pytest

import synth
from oracle import dealer
from paper_2311_04406_gb300 import abi, build

from gpuhelp import dev, empty_like_ring, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    abi.load()


def dev_t(ring, a):
    """Upload a (rows x cols) ring matrix and transpose it on the device."""
    rows, cols = a.shape[:2]
    out = empty_like_ring((cols, rows), ring.words)
    abi.mpc_transpose(ring.k, ring.s, rows, cols, dev(a), out)
    return out


@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=lambda r: f"k{r.k}")
@pytest.mark.parametrize("shape", [(1, 1), (1, 77), (77, 1), (32, 32), (33, 65), (300, 7), (129, 257), (0, 5)],
                         ids=str)
def test_transpose_parity(ring, shape):
    a = synth.uniform(11, 1, 0, shape, ring.bits)
    got = host(dev_t(ring, a)) if a.size else np.empty((shape[1], 0), dtype=np.uint64)
    assert np.array_equal(got.reshape(dealer.transpose(a).shape), dealer.transpose(a))


def _run_layer_gpu(ring, L, i, E, F, A, B, C, mA, mB, mR, mC, ref):
    """One party's share, full tag and compact tag of layer L (operands given as
    device tensors), compared with the oracle's outputs."""
    p = L.parties[i]
    lay = abi.make_layer(L.M, L.K, L.N, ring.k, ring.s, i, len(L.parties))
    Z = empty_like_ring((L.M, L.N), ring.words)
    abi.mpc_linear_share(lay, E, F, A, B, C, Z)
    assert np.array_equal(host(Z), ref["Z"][i]), f"share party {i}"
    mZ = empty_like_ring((L.M, L.N), ring.words)
    abi.mpc_linear_tag(lay, abi.MPC_TAG_FULL, dev(p.alpha), E, F, mA, mB, mC, mZ)
    assert np.array_equal(host(mZ), ref["mZ_full"][i]), f"full tag party {i}"
    mDc = empty_like_ring((L.M,), ring.words)
    Dc = empty_like_ring((L.M,), ring.words)
    abi.mpc_linear_tag(lay, abi.MPC_TAG_COMPACT, dev(p.alpha), E, F, mA, mB, mC, mZ, mR_i=mR,
                       Dtilde=dev(ref["Dt"]), chi=dev(L.chi), mDc_i=mDc, Dc=Dc)
    assert np.array_equal(host(mZ), ref["mZ_opt"][i]), f"optimistic tag party {i}"
    assert np.array_equal(host(mDc), ref["mDc"][i]), f"compact tag party {i}"
    assert np.array_equal(host(Dc), ref["Dc"])


# forward (M, K, N); the backward products are (M, N, K) and (K, M, N).  The
# sizes take both products through the tensor-core kernel, the integer-pipe
# tile kernel and the skinny kernel, with ragged edges.
CASES = [(synth.Z64, (96, 200, 136)), (synth.Z64, (128, 256, 64)), (synth.Z64, (5, 70, 33)),
         (synth.Z64, (257, 33, 130)), (synth.Z128, (64, 96, 80)), (synth.Z128, (3, 17, 9))]


@pytest.mark.parametrize("ring,shape", CASES, ids=lambda x: str(x) if isinstance(x, tuple) else None)
def test_backward_layers_parity(ring, shape):
    M, K, N = shape
    d = dealer.deal(ring, M, K, N, n=2, seed=M * 7 + K + N)
    b = dealer.deal_backward(d, seed=M * 7 + K + N)
    ref_x = dealer.run_layer(b.dX)
    ref_w = dealer.run_layer(b.dW)
    Ft, Et = dev_t(ring, d.F), dev_t(ring, d.E)
    Eg = dev(b.dX.E)
    for i, p in enumerate(d.parties):
        qx, qw = b.dX.parties[i], b.dW.parties[i]
        # grad X: left G (mask A', fresh), right W^T (mask B^T: transposed on device)
        _run_layer_gpu(ring, b.dX, i, Eg, Ft, dev(qx.A), dev_t(ring, p.B), dev(qx.C), dev(qx.mA),
                       dev_t(ring, p.mB), dev(qx.mR), dev(qx.mC), ref_x)
        # grad W: left X^T (mask A^T: transposed on device), right G (mask A')
        _run_layer_gpu(ring, b.dW, i, Et, Eg, dev_t(ring, p.A), dev(qw.B), dev(qw.C), dev_t(ring, p.mA),
                       dev(qw.mB), dev(qw.mR), dev(qw.mC), ref_w)
    assert abi.mpc_device_status() == 0


def test_transpose_rejects_bad_arguments():
    import ctypes
    lib = abi.load()
    ring = abi.mpc_ring(32, 32, 1)
    assert lib.mpc_transpose(None, 2, 2, 0x1000, 0x2000, None) == abi.MPC_E_NULL
    assert lib.mpc_transpose(ctypes.byref(ring), -1, 2, 0x1000, 0x2000, None) == abi.MPC_E_SHAPE
    assert lib.mpc_transpose(ctypes.byref(ring), 2, 2, None, 0x2000, None) == abi.MPC_E_NULL
