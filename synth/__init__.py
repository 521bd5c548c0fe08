"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the protocol: it only draws uniform ring words
and lists layer shapes.  Secret shares, triple shares, tag shares and the public
opened matrices E, F, D~ of an SPDZ2k computation are uniformly distributed ring
elements by construction (§2.4: every share is masked by a fresh uniform share),
so uniform words have exactly the distribution of real protocol data; only the
shapes come from the paper's networks (§4.1).

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a counter-based generator.  The stream for
(seed, tensor_id, party) starts at state

    key = mix(mix(seed) + tensor_id * GAMMA + party * GAMMA2)

and word i is mix(key + (i + 1) * GAMMA), where mix is the SplitMix64 output
function.  All arithmetic is mod 2^64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
GAMMA2 = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (vectorised, wrapping uint64)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _key(seed: int, tensor_id: int, party: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        k = s + np.uint64(tensor_id & 0xFFFFFFFFFFFFFFFF) * GAMMA \
            + np.uint64(party & 0xFFFFFFFFFFFFFFFF) * GAMMA2
    return _mix(np.array([k], dtype=np.uint64))[0]


def words(seed: int, tensor_id: int, party: int, count: int) -> np.ndarray:
    """`count` uniform 64-bit words of the stream (seed, tensor_id, party)."""
    key = _key(seed, tensor_id, party)
    idx = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = key + idx * GAMMA
    return _mix(state)


def ring_words(bits: int) -> int:
    """Words per element of Z_{2^bits}: 1 up to 64 bits, else 2 (lo, hi)."""
    if not 1 <= bits <= 128:
        raise ValueError("ring width must be 1..128 bits")
    return 1 if bits <= 64 else 2


def uniform(seed: int, tensor_id: int, party: int, shape, bits: int) -> np.ndarray:
    """Uniform elements of Z_{2^bits} with the given logical shape.

    Storage is little-endian words: shape `shape` for one-word rings, shape
    `shape + (2,)` with (lo, hi) for two-word rings.  Values are reduced mod
    2^bits (high bits of the last word cleared).
    """
    shape = tuple(int(d) for d in shape)
    w = ring_words(bits)
    n = int(np.prod(shape, dtype=np.int64)) if shape else 1
    raw = words(seed, tensor_id, party, n * w)
    out = raw.reshape(shape + ((w,) if w == 2 else ()))
    top = bits - 64 * (w - 1)
    if top < 64:
        m = np.uint64((1 << top) - 1)
        if w == 1:
            out &= m
        else:
            out[..., 1] &= m
    return np.ascontiguousarray(out)


# ---------------------------------------------------------------------------
# Ring parameters (§4.1): (k, s) = (32, 32) gives shares in Z_{2^64}, (64, 64)
# gives shares in Z_{2^128}.

@dataclass(frozen=True)
class Ring:
    k: int
    s: int

    @property
    def bits(self) -> int:
        return self.k + self.s

    @property
    def words(self) -> int:
        return ring_words(self.bits)


Z64 = Ring(32, 32)
Z128 = Ring(64, 64)


# Tensor ids of the streams (one per operand; party index selects the share).
TID = dict(E=1, F=2, A=3, B=4, C=5, mA=6, mB=7, mC=8, R=9, mR=10, Dt=11,
           chi=12, chi_hat=13, alpha=14, X=15, Y=16, W=17, mW=18, chiW=19,
           Rf=20, mRf=21)


@dataclass(frozen=True)
class Layer:
    """One linear layer as a ring GEMM: Z (M x N) = X (M x K) . W (K x N)."""
    name: str
    M: int
    K: int
    N: int

    @property
    def macs(self) -> int:
        return self.M * self.K * self.N


def conv_rows(w: int, h: int, f: int, p: int, stride: int) -> int:
    """Output positions of an f x f convolution (im2col rows per image).

    The §2.6 formula omits the "+1" of the textbook output size; the textbook
    size floor((w - f + 2p) / stride) + 1 per axis is used (it gives 1024 rows
    for 32x32, 3x3, p=1, stride 1).
    """
    return ((w - f + 2 * p) // stride + 1) * ((h - f + 2 * p) // stride + 1)


def conv_layer(name, w, h, cin, cout, f=3, p=1, stride=1, batch=1) -> Layer:
    """im2col view of a convolution (§2.6): M = rows*batch, K = cin*f*f, N = cout."""
    return Layer(name, conv_rows(w, h, f, p, stride) * batch, cin * f * f, cout)


def vgg16_layers(batch: int = 1) -> list[Layer]:
    """VGG16 on a 32x32x3 input: 13 3x3 convolutions and a 512-4096-4096-10 head.

    Pooling and ReLU are not linear-layer work and are skipped; spatial size
    halves after each pooling stage (after conv 2, 4, 7, 10, 13).
    """
    plan = [(3, 64), (64, 64), "P", (64, 128), (128, 128), "P",
            (128, 256), (256, 256), (256, 256), "P",
            (256, 512), (512, 512), (512, 512), "P",
            (512, 512), (512, 512), (512, 512), "P"]
    out, side, i = [], 32, 0
    for step in plan:
        if step == "P":
            side //= 2
            continue
        i += 1
        cin, cout = step
        out.append(conv_layer(f"conv{i}", side, side, cin, cout, batch=batch))
    out += [Layer("fc1", batch, 512, 4096), Layer("fc2", batch, 4096, 4096),
            Layer("fc3", batch, 4096, 10)]
    return out


def resnet18_layers(batch: int = 1) -> list[Layer]:
    """CIFAR-style ResNet-18 on 32x32x3: conv1, four stages of two basic
    blocks (3x3 convs; stride-2 entry with a 1x1 downsample in stages 2-4),
    and the 512 -> 10 classifier."""
    out = [conv_layer("conv1", 32, 32, 3, 64, batch=batch)]
    side, cin = 32, 64
    for stage, cout in enumerate([64, 128, 256, 512]):
        for blk in range(2):
            stride = 2 if (stage > 0 and blk == 0) else 1
            nside = (side - 3 + 2) // stride + 1
            out.append(Layer(f"s{stage}b{blk}c1", nside * nside * batch, cin * 9, cout))
            out.append(Layer(f"s{stage}b{blk}c2", nside * nside * batch, cout * 9, cout))
            if stride == 2:
                out.append(Layer(f"s{stage}b{blk}ds", nside * nside * batch, cin, cout))
            side, cin = nside, cout
    out.append(Layer("fc", batch, 512, 10))
    return out


def cnn_pair() -> list[Layer]:
    """The two CNN-style layers: a 3x3 conv on 32x32x64 -> 64 (im2col
    1024 x 576 x 64) and a 4096 x 4096 dense layer at batch 128."""
    return [conv_layer("conv3x3_32x32x64", 32, 32, 64, 64),
            Layer("dense4096_b128", 128, 4096, 4096)]


def single_dense() -> Layer:
    """Single dense layer X 64x128, W 128x64 (two parties, Z_2^64)."""
    return Layer("dense_64x128x64", 64, 128, 64)


def transformer_layers(rows: int = 2048, hidden: int = 1024) -> list[Layer]:
    """Encoder projections at H=1024 with T1=2048 rows (§4.1, §4.3 example)."""
    return [Layer("qkv_or_out", rows, hidden, hidden),
            Layer("ffn_up", rows, hidden, 4 * hidden),
            Layer("ffn_down", rows, 4 * hidden, hidden)]


def transformer_block(rows: int = 2048, hidden: int = 1024, heads: int = 16) -> list[Layer]:
    """One encoder block at H = 1024, A = 16 heads, T1 = 2048 rows (§4.1):
    the Q, K, V and output projections, the two FFN products, and per head the
    attention-score product Q_h K_h^T (rows x d x rows) and the value product
    S_h V_h (rows x rows x d), d = H / A.  Softmax and the other nonlinear
    steps are not linear-layer work and are skipped."""
    d = hidden // heads
    out = [Layer(n, rows, hidden, hidden) for n in ("q_proj", "k_proj", "v_proj", "o_proj")]
    out += [Layer("ffn_up", rows, hidden, 4 * hidden), Layer("ffn_down", rows, 4 * hidden, hidden)]
    for h in range(heads):
        out.append(Layer(f"scores_h{h}", rows, d, rows))
        out.append(Layer(f"values_h{h}", rows, rows, d))
    return out


def uneven_layers(count: int = 256, seed: int = 0xC0FFEE03) -> list[Layer]:
    """`count` layers with M log-uniform in [1, 4096] and K, N drawn from
    {64, 128, ..., 4096} with a uniform exponent."""
    w = words(seed, 100, 0, 3 * count)
    out = []
    for i in range(count):
        u = (int(w[3 * i]) >> 11) / float(1 << 53)
        m = int(round(math.exp(u * math.log(4096.0))))
        m = min(max(m, 1), 4096)
        k = 64 << (int(w[3 * i + 1]) % 7)
        n = 64 << (int(w[3 * i + 2]) % 7)
        out.append(Layer(f"u{i}", m, k, n))
    return out


def backward_layers(forward: list) -> list:
    """The two gradient products of each forward layer Z (M x N) = X (M x K) . W:
    grad X = grad Z (M x N) . W^T (N x K)  -> (M, N, K), and
    grad W = X^T (K x M) . grad Z (M x N)  -> (K, M, N)."""
    out = []
    for L in forward:
        out.append(Layer(L.name + "_dX", L.M, L.N, L.K))
        out.append(Layer(L.name + "_dW", L.K, L.M, L.N))
    return out
