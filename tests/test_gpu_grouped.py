"""GPU parity of the grouped calls (many layers per call; the tensor-core
layers of a group share one persistent prologue + GEMM launch pair per 64
layers): every layer's share and tags equal the oracle's bit for bit, for
groups mixing the tensor-core, integer-pipe tile and skinny paths, several
parties, and more than one launch's worth of layers."""
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


def inputs(ring, shapes, seed, tags=True):
    bits = ring.bits
    out = []
    for li, (M, K, N) in enumerate(shapes):
        sd = seed + 7919 * li
        u = lambda name, shape: synth.uniform(sd, synth.TID[name], 1, shape, bits)
        key = lambda name, shape: synth.uniform(sd, synth.TID[name], 1, shape, ring.s).astype(np.uint64) \
            if ring.words == 1 else np.stack([synth.uniform(sd, synth.TID[name], 1, shape, ring.s),
                                               np.zeros(shape, np.uint64)], axis=-1)
        d = dict(M=M, K=K, N=N, E=u("E", (M, K)), F=u("F", (K, N)), A=u("A", (M, K)), B=u("B", (K, N)),
                 C=u("C", (M, N)), party=li % 3 % 2)
        if tags:
            d.update(mA=u("mA", (M, K)), mB=u("mB", (K, N)), mC=u("mC", (M, N)), mR=u("mR", (M, N)),
                     Dt=u("Dt", (M, N)), chi=key("chi", (N,)), alpha=key("alpha", (1,)))
        out.append(d)
    return out


def run_group(ring, data):
    w = ring.words
    layers = [abi.make_layer(d["M"], d["K"], d["N"], ring.k, ring.s, d["party"], 2) for d in data]
    dd = [{k: dev(v) for k, v in d.items() if isinstance(v, np.ndarray)} for d in data]
    for d, x in zip(data, dd):
        x["Z"] = empty_like_ring((d["M"], d["N"]), w)
        x["mZf"] = empty_like_ring((d["M"], d["N"]), w)
        x["mZ"] = empty_like_ring((d["M"], d["N"]), w)
        x["mDc"] = empty_like_ring((d["M"],), w)
        x["Dc"] = empty_like_ring((d["M"],), w)
    abi.mpc_linear_share_grouped(layers, [dict(E=x["E"], F=x["F"], A_i=x["A"], B_i=x["B"], C_i=x["C"],
                                               Z_i=x["Z"]) for x in dd])
    tag = lambda x, mz: dict(alpha_i=x["alpha"], E=x["E"], F=x["F"], mA_i=x["mA"], mB_i=x["mB"], mC_i=x["mC"],
                             mR_i=x["mR"], Dtilde=x["Dt"], chi=x["chi"], mZ_i=mz, mDc_i=x["mDc"], Dc=x["Dc"])
    abi.mpc_linear_tag_grouped(layers, abi.MPC_TAG_FULL, [tag(x, x["mZf"]) for x in dd])
    abi.mpc_linear_tag_grouped(layers, abi.MPC_TAG_COMPACT, [tag(x, x["mZ"]) for x in dd])
    return [{k: host(x[k]) for k in ("Z", "mZf", "mZ", "mDc", "Dc")} for x in dd]


def check(ring, data, got):
    bits = ring.bits
    for li, (d, g) in enumerate(zip(data, got)):
        Z = O.linear_share(bits, d["party"], d["E"], d["F"], d["A"], d["B"], d["C"])
        assert np.array_equal(g["Z"], Z), f"share of layer {li} {d['M'], d['K'], d['N']}"
        mZ = O.linear_tag_full(bits, d["alpha"], d["E"], d["F"], d["mA"], d["mB"], d["mC"])
        assert np.array_equal(g["mZf"], mZ), f"full tag of layer {li}"
        mDc, Dc, _ = O.compact_tag(bits, d["alpha"], d["E"], d["F"], d["mA"], d["mB"], d["mC"], d["mR"],
                                   d["Dt"], d["chi"])
        assert np.array_equal(g["mZ"], O.optmac(bits, d["alpha"], d["mR"], d["Dt"])), f"OptMAC tag {li}"
        assert np.array_equal(g["mDc"], mDc), f"compact tag of layer {li}"
        assert np.array_equal(g["Dc"], Dc), f"compressed D of layer {li}"


# tensor-core layers (small to large, ragged M, K, N), integer-pipe tiles
# (odd N, small products), skinny layers (M <= 8)
MIXED64 = [(128, 256, 64), (9, 700, 512), (300, 64, 130), (64, 128, 64), (4, 512, 300), (1, 1000, 1000),
           (200, 27, 1024), (33, 300, 31), (1024, 576, 64), (130, 129, 66), (16, 128, 1024)]
MIXED128 = [(64, 96, 80), (130, 256, 40), (5, 77, 9), (200, 64, 64), (1, 300, 200), (65, 128, 17)]


def test_grouped_mixed_z64():
    ring = synth.Z64
    data = inputs(ring, MIXED64, 11)
    check(ring, data, run_group(ring, data))
    assert abi.mpc_device_status() == 0


def test_grouped_mixed_z128():
    ring = synth.Z128
    data = inputs(ring, MIXED128, 12)
    check(ring, data, run_group(ring, data))
    assert abi.mpc_device_status() == 0


def test_grouped_more_than_one_launch():
    """70 tensor-core layers: two grouped launch pairs (64 + 6 layers)."""
    ring = synth.Z64
    shapes = [(16 + 8 * (i % 5), 144 + 16 * (i % 3), 1024 - 2 * (i % 4)) for i in range(70)]
    layers = [abi.make_layer(M, K, N) for M, K, N in shapes]
    assert all(abi.mpc_gemm_path(L) == 1 for L in layers)
    assert abi.mpc_launch_count_grouped(layers, abi.MPC_WS_SHARE) == 4
    data = inputs(ring, shapes, 13)
    got = run_group(ring, data)
    check(ring, data, got)


def test_grouped_uneven_chunk_sampled():
    """The first 64 layers of the seeded 256-layer uneven set at full size,
    checked on sampled outputs (the oracle computes them one by one)."""
    ring = synth.Z64
    bits = ring.bits
    shapes = [(L.M, L.K, L.N) for L in synth.uneven_layers(256)[:64]]
    data = inputs(ring, shapes, 14, tags=False)
    layers = [abi.make_layer(M, K, N, party=d["party"]) for (M, K, N), d in zip(shapes, data)]
    dd = [{k: dev(d[k]) for k in ("E", "F", "A", "B", "C")} for d in data]
    for d, x in zip(data, dd):
        x["Z"] = empty_like_ring((d["M"], d["N"]), 1)
    abi.mpc_linear_share_grouped(layers, [dict(E=x["E"], F=x["F"], A_i=x["A"], B_i=x["B"], C_i=x["C"],
                                               Z_i=x["Z"]) for x in dd])
    rng = np.random.default_rng(5)
    for d, x in zip(data, dd):
        M, N = d["M"], d["N"]
        rows = np.concatenate([[0, M - 1], rng.integers(0, M, 6)]).astype(np.int64)
        cols = np.concatenate([[0, N - 1], rng.integers(0, N, 6)]).astype(np.int64)
        want = O.linear_share_at(bits, d["party"], d["E"], d["F"], d["A"], d["B"], d["C"], rows, cols)
        Z = host(x["Z"])[rows, cols]
        assert np.array_equal(Z, want.reshape(Z.shape))
    assert abi.mpc_device_status() == 0


def test_grouped_empty_and_degenerate():
    ring = synth.Z64
    abi.mpc_linear_share_grouped([], [])
    data = inputs(ring, [(0, 16, 16), (16, 0, 16), (3, 5, 0), (64, 128, 64)], 15)
    got = run_group(ring, data)
    check(ring, data, got)


def test_grouped_rejects_mixed_rings():
    lib = abi.load()
    layers = [abi.make_layer(64, 64, 64), abi.make_layer(64, 64, 64, 64, 64)]
    assert abi.mpc_launch_count_grouped(layers, abi.MPC_WS_SHARE) == abi.MPC_E_RING
    arr = (abi.mpc_layer * 2)(*layers)
    ptrs = (abi.mpc_share_ptrs * 2)()
    assert lib.mpc_linear_share_grouped(arr, 2, ptrs, None, 0, None) == abi.MPC_E_RING
