"""GPU parity of the im2col view of a convolution (§2.6), and a convolution
layer's share computed as im2col + the share GEMM on the device, against the
oracle's im2col and product."""
import numpy as np
import pytest

import oracle as O
import synth
from paper_2311_04406_gb300 import abi, build

from gpuhelp import dev, empty_like_ring, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    abi.load()


def gpu_im2col(ring, x, f, pad, stride):
    B, C, H, W = x.shape[:4]
    Ho, Wo = (H - f + 2 * pad) // stride + 1, (W - f + 2 * pad) // stride + 1
    out = empty_like_ring((B * Ho * Wo, C * f * f), ring.words)
    abi.mpc_im2col(ring.k, ring.s, B, C, H, W, f, pad, stride, dev(x), out)
    return out


CASES = [(2, 3, 32, 32, 3, 1, 1), (1, 64, 32, 32, 3, 1, 1), (2, 64, 16, 16, 3, 1, 2), (3, 128, 8, 8, 1, 0, 2),
         (1, 5, 7, 9, 3, 2, 3), (1, 1, 3, 3, 3, 0, 1), (4, 16, 4, 4, 2, 1, 1)]


@pytest.mark.parametrize("ring", [synth.Z64, synth.Z128], ids=["z64", "z128"])
@pytest.mark.parametrize("cfg", CASES, ids=str)
def test_im2col_parity(ring, cfg):
    B, C, H, W, f, pad, stride = cfg
    x = synth.uniform(B + C, 1, 0, (B, C, H, W), ring.bits)
    got = host(gpu_im2col(ring, x, f, pad, stride))
    assert np.array_equal(got, O.im2col(x, f, pad, stride, ring.bits))


def test_conv_layer_share_on_device():
    """The first 3x3 conv of the CNN pair: im2col of the opened E image and of
    the party's A share on the device, then the share GEMM (1024 x 576 x 64)."""
    ring = synth.Z64
    bits = ring.bits
    C, H, W, Oc, f = 64, 32, 32, 64, 3
    u = lambda t, shape: synth.uniform(7, t, 0, shape, bits)
    Eimg, Aimg = u(1, (1, C, H, W)), u(2, (1, C, H, W))
    F, B, Cm = u(3, (C * f * f, Oc)), u(4, (C * f * f, Oc)), u(5, (H * W, Oc))
    E = gpu_im2col(ring, Eimg, f, 1, 1)
    A = gpu_im2col(ring, Aimg, f, 1, 1)
    L = abi.make_layer(H * W, C * f * f, Oc, ring.k, ring.s, 0, 2)
    Z = empty_like_ring((H * W, Oc), 1)
    abi.mpc_linear_share(L, E, dev(F), A, dev(B), dev(Cm), Z)
    want = O.linear_share(bits, 0, O.im2col(Eimg, f, 1, 1, bits), F, O.im2col(Aimg, f, 1, 1, bits), B, Cm)
    assert np.array_equal(host(Z), want)


def test_im2col_rejects_bad_shapes():
    import ctypes
    lib = abi.load()
    ring = abi.mpc_ring(32, 32, 1)
    R = ctypes.byref(ring)
    assert lib.mpc_im2col(R, 1, 1, 4, 4, 3, 3, 1, 0x1000, 0x2000, None) == abi.MPC_E_SHAPE   # pad >= f
    assert lib.mpc_im2col(R, 1, 1, 4, 4, 3, 1, 0, 0x1000, 0x2000, None) == abi.MPC_E_SHAPE   # stride 0
    assert lib.mpc_im2col(R, 1, 1, 1, 1, 5, 1, 1, 0x1000, 0x2000, None) == abi.MPC_E_SHAPE   # image < filter
