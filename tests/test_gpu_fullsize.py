"""Full-size layers of the benchmark workloads in the launch configuration the
benchmark times: sampled share and full-tag outputs (the oracle computes them
one by one) and the whole CompactTag tag, check included.  These shapes have
more tiles than CTAs, so they run the data-parallel waves of the tensor-core
schedule (whole tiles written directly as C + sum) as well as its stream-K
remainder; the samples include tile corners."""
import numpy as np
import pytest

import oracle as O
import synth
from paper_2311_04406_gb300 import abi, build

from gpuhelp import gpu_check_compact, gpu_share, gpu_tag_compact, gpu_tag_full
from test_gpu_parity import _uniform_layer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    abi.load()
    abi.mpc_autotune_clear()


CASES = [
    (synth.Z64, (2048, 1024, 4096)),     # Transformer ffn_up
    (synth.Z64, (2048, 4096, 1024)),     # Transformer ffn_down
    (synth.Z64, (4096, 128, 4096)),      # training grad W of the dense layer
    (synth.Z64, (65536, 576, 64)),       # VGG16 conv2 at batch 64
    (synth.Z128, (32768, 576, 64)),      # ResNet-18 stage-0 conv at batch 32, Z_2^128 (tall tile)
    (synth.Z128, (8192, 1152, 128)),     # ResNet-18 stage-1 conv at batch 32, Z_2^128 (tall tile, N = 128)
    (synth.Z128, (2048, 2304, 256)),     # ResNet-18 stage-2 conv at batch 32, Z_2^128
    (synth.Z64, (4096, 1152, 128)),      # VGG16 conv at 16x16 and batch 16, Z_2^64 (tall tile, N = 128)
]


def samples(M, N, n=384, seed=7):
    sw = synth.words(seed, 1, 0, 2 * n)
    rows = (sw[:n] % np.uint64(M)).astype(np.int64)
    cols = (sw[n:] % np.uint64(N)).astype(np.int64)
    # tile corners: rows 127/128, columns 15/16/31/32, the last row and column
    fixed = [(0, 0), (M - 1, N - 1), (min(127, M - 1), min(31, N - 1)), (min(128, M - 1), min(32, N - 1)),
             (min(255, M - 1), min(15, N - 1)), (min(256, M - 1), min(16, N - 1)), (M - 1, 0), (0, N - 1)]
    for i, (r, c) in enumerate(fixed):
        rows[i], cols[i] = r, c
    return rows, cols


@pytest.mark.parametrize("ring,shape", CASES, ids=lambda x: str(x) if isinstance(x, tuple) else None)
def test_full_size_layer(ring, shape):
    M, K, N = shape
    bits = ring.bits
    assert abi.mpc_gemm_path(abi.make_layer(M, K, N, ring.k, ring.s)) == 1
    x = _uniform_layer(ring, M, K, N, seed=M + K + N)
    rows, cols = samples(M, N)
    Z = gpu_share(ring, 0, x["E"], x["F"], x["A"], x["B"], x["C"])
    assert np.array_equal(Z[rows, cols], O.linear_share_at(bits, 0, x["E"], x["F"], x["A"], x["B"], x["C"],
                                                            rows, cols).reshape(Z[rows, cols].shape))
    del Z
    mZf = gpu_tag_full(ring, 1, x["alpha"], x["E"], x["F"], x["mA"], x["mB"], x["mC"])
    want = O.linear_tag_full_at(bits, x["alpha"], x["E"], x["F"], x["mA"], x["mB"], x["mC"], rows, cols)
    assert np.array_equal(mZf[rows, cols], want.reshape(mZf[rows, cols].shape))
    del mZf
    mZ, mDc, Dc = gpu_tag_compact(ring, 1, x["alpha"], x["E"], x["F"], x["mA"], x["mB"], x["mC"], x["mR"],
                                  x["Dt"], x["chi"])
    rmDc, rDc, _ = O.compact_tag(bits, x["alpha"], x["E"], x["F"], x["mA"], x["mB"], x["mC"], x["mR"], x["Dt"],
                                 x["chi"])
    assert np.array_equal(mDc, rmDc) and np.array_equal(Dc, rDc)
    assert np.array_equal(mZ, O.optmac(bits, x["alpha"], x["mR"], x["Dt"]))
    cs = gpu_check_compact(ring, x["alpha"], x["chi_hat"], Dc, mDc)
    assert np.array_equal(cs.reshape(-1), O.check_compact(bits, x["alpha"], x["chi_hat"], rDc, rmDc).reshape(-1))
    assert abi.mpc_device_status() == 0
