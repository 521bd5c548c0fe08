"""Pins of the oracle's im2col view of a convolution (§2.6): the im2col
matrix times the reshaped filter equals the convolution written out directly
(Python-integer loops, mod 2^64 and 2^128), the output size is the textbook
one, a 1x1 filter is a plain relayout, and the padding holds zeros."""
import numpy as np
import pytest

import oracle as O
import synth


def conv_direct(x, w, pad, stride, bits):
    """sum_{c, ky, kx} x[b][c][oy s + ky - p][ox s + kx - p] w[o][c][ky][kx] mod 2^bits."""
    B, C, H, W = x.shape[:4]
    Oc, _, f, _ = w.shape[:4]
    Ho, Wo = (H - f + 2 * pad) // stride + 1, (W - f + 2 * pad) // stride + 1
    xi, wi = O.to_int(x, bits), O.to_int(w, bits)
    out = np.zeros((B, Oc, Ho, Wo), dtype=object)
    for b in range(B):
        for o in range(Oc):
            for oy in range(Ho):
                for ox in range(Wo):
                    acc = 0
                    for c in range(C):
                        for ky in range(f):
                            for kx in range(f):
                                y, xx = oy * stride + ky - pad, ox * stride + kx - pad
                                if 0 <= y < H and 0 <= xx < W:
                                    acc += int(xi[b, c, y, xx]) * int(wi[o, c, ky, kx])
                    out[b, o, oy, ox] = acc % (1 << bits)
    return out


@pytest.mark.parametrize("bits", [64, 128])
@pytest.mark.parametrize("cfg", [(2, 3, 5, 6, 4, 3, 1, 1), (1, 2, 7, 7, 3, 3, 0, 2), (2, 1, 4, 5, 2, 1, 0, 1),
                                 (1, 2, 6, 6, 2, 3, 1, 2), (1, 1, 3, 3, 1, 3, 2, 1)], ids=str)
def test_im2col_gemm_is_convolution(bits, cfg):
    B, C, H, W, Oc, f, pad, stride = cfg
    x = synth.uniform(1, 1, 0, (B, C, H, W), bits)
    w = synth.uniform(1, 2, 0, (Oc, C, f, f), bits)
    cols = O.im2col(x, f, pad, stride, bits)
    Ho, Wo = (H - f + 2 * pad) // stride + 1, (W - f + 2 * pad) // stride + 1
    assert cols.shape[:2] == (B * Ho * Wo, C * f * f)
    wmat = np.ascontiguousarray(w.reshape((Oc, C * f * f) + w.shape[4:]).swapaxes(0, 1))
    Z = O.to_int(O.ring_gemm(bits, cols, wmat), bits)                  # (B Ho Wo) x Oc
    want = conv_direct(x, w, pad, stride, bits)                       # B x Oc x Ho x Wo
    assert np.array_equal(Z.reshape(B, Ho, Wo, Oc).transpose(0, 3, 1, 2), want)


def test_im2col_sizes_and_special_cases():
    bits = 64
    x = synth.uniform(2, 1, 0, (2, 64, 32, 32), bits)
    cols = O.im2col(x, 3, 1, 1, bits)
    assert cols.shape == (2 * 1024, 576) and 1024 == synth.conv_rows(32, 32, 3, 1, 1)
    assert O.im2col(x[:1, :4], 3, 1, 2, bits).shape == (16 * 16, 36)
    # 1x1 filter, no padding: the NCHW images as (B H W) x C
    one = O.im2col(x[:, :5, :4, :3], 1, 0, 1, bits)
    assert np.array_equal(one, np.ascontiguousarray(x[:, :5, :4, :3].transpose(0, 2, 3, 1).reshape(-1, 5)))
    # the padding ring of a 3x3 filter with pad 1: row (0, 0, 0) has zeros at (ky, kx) = (0, *) and (*, 0)
    first = cols[0].reshape(64, 3, 3)
    assert not first[:, 0, :].any() and not first[:, :, 0].any()
    assert np.array_equal(first[:, 1:, 1:], x[0, :, 0:2, 0:2])


def test_im2col_is_linear():
    bits = 128
    a = synth.uniform(3, 1, 0, (1, 3, 6, 6), bits)
    b = synth.uniform(3, 2, 0, (1, 3, 6, 6), bits)
    lhs = O.im2col(O.add(bits, a, b), 3, 1, 1, bits)
    rhs = O.add(bits, O.im2col(a, 3, 1, 1, bits), O.im2col(b, 3, 1, 1, bits))
    assert np.array_equal(lhs, rhs)
