"""The allocation-free CompactTag entry point against the workspace one.

mpc_linear_tag_compact_noalloc serves callers that cannot allocate device
memory (a host runtime using this library through a plain C FFI with no CUDA
allocator, or a process whose device memory is owned by another framework's
pool): its scratch is a static device buffer inside the library instead of a
caller workspace.  Its outputs must equal those of
mpc_linear_tag(MPC_TAG_COMPACT) bit for bit -- the tolerance of every integer
test here is zero -- on consecutive calls, where the second call starts with
the first call's leftovers in the shared buffer.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2311_04406_gb300 import abi, build

pytestmark = pytest.mark.gpu


def _inputs(ring, M, K, N, seed):
    g = lambda name, shape: synth.uniform(seed, synth.TID[name], 0, shape, ring.bits)

    def key(name, shape):
        # s-bit values (the MAC key share, the compression vector) stored as
        # ring elements: in Z_2^128 each takes two words, the high one zero
        v = synth.uniform(seed, synth.TID[name], 0, shape, ring.s)
        return v if ring.words == 1 else np.stack([v, np.zeros_like(v)], axis=-1)

    return dict(alpha=key("alpha", (1,)), E=g("E", (M, K)), F=g("F", (K, N)),
                mA=g("mA", (M, K)), mB=g("mB", (K, N)), mC=g("mC", (M, N)), mR=g("mR", (M, N)),
                Dt=g("Dt", (M, N)), chi=key("chi", (N,)))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _pad(words, ring):
    return words if ring.words == 1 else words + (2,)


def _both(ring, M, K, N, seed):
    host = _inputs(ring, M, K, N, seed)
    # every buffer holds exactly the ring elements the call reads
    elems = dict(alpha=1, E=M * K, F=K * N, mA=M * K, mB=K * N, mC=M * N, mR=M * N, Dt=M * N, chi=N)
    for name, n in elems.items():
        assert host[name].size == n * ring.words, name
    x = {k: _dev(v) for k, v in host.items()}
    lay = abi.make_layer(M, K, N, ring.k, ring.s, party=1, nparties=2)
    outs = []
    for noalloc in (False, True):
        mZ = torch.full(_pad((M, N), ring), -1, dtype=torch.int64, device="cuda")
        mDc = torch.full(_pad((M,), ring), -1, dtype=torch.int64, device="cuda")
        Dc = torch.full(_pad((M,), ring), -1, dtype=torch.int64, device="cuda")
        if noalloc:
            abi.mpc_linear_tag_compact_noalloc(lay, x["alpha"], x["E"], x["F"], x["mA"], x["mB"],
                                               x["mC"], x["mR"], x["Dt"], x["chi"], mZ, mDc, Dc)
        else:
            abi.mpc_linear_tag(lay, abi.MPC_TAG_COMPACT, x["alpha"], x["E"], x["F"], x["mA"],
                               x["mB"], x["mC"], mZ, mR_i=x["mR"], Dtilde=x["Dt"], chi=x["chi"],
                               mDc_i=mDc, Dc=Dc)
        torch.cuda.synchronize()
        outs.append((mZ.cpu(), mDc.cpu(), Dc.cpu()))
    return host, outs


def _as_ring(t, ring):
    return t.numpy().view(np.uint64)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    abi.load()


def test_noalloc_equals_workspace_entry_point_on_consecutive_calls():
    # first call uses split row chunks (large N), the second a small layer in
    # the other ring, then a third repeats the first shape with new values
    # (K < 64 takes the small-K vector kernel: covered in both rings)
    cases = [(synth.Z64, 96, 1500, 2600, 11), (synth.Z128, 65, 130, 70, 12),
             (synth.Z64, 96, 1500, 2600, 13), (synth.Z128, 65, 27, 70, 14), (synth.Z64, 33, 40, 50, 15),
             (synth.Z128, 65, 27, 70, 16)]
    for ring, M, K, N, seed in cases:
        lay = abi.make_layer(M, K, N, ring.k, ring.s)
        assert abi.mpc_workspace_size(lay, abi.MPC_WS_TAG_COMPACT) <= abi.MPC_NOALLOC_SCRATCH_BYTES
        host, (ref, got) = _both(ring, M, K, N, seed)
        for a, b, name in zip(ref, got, ("mZ", "mDc", "Dc")):
            assert torch.equal(a, b), f"{name} differs for {(M, K, N)} w={ring.words}"
        # and both equal the oracle
        h = host
        mDc, Dc, _ = O.compact_tag(ring.bits, h["alpha"], h["E"], h["F"], h["mA"], h["mB"], h["mC"],
                                   h["mR"], h["Dt"], h["chi"])
        assert np.array_equal(_as_ring(got[0], ring), O.optmac(ring.bits, h["alpha"], h["mR"], h["Dt"]))
        assert np.array_equal(_as_ring(got[1], ring), mDc), f"mDc vs oracle for {(M, K, N)}"
        assert np.array_equal(_as_ring(got[2], ring), Dc), f"Dc vs oracle for {(M, K, N)}"


@pytest.mark.hidden_gpu
def test_noalloc_rejects_layers_beyond_the_static_scratch():
    lib = abi.load()
    M, K, N = 1 << 20, 4096, 64       # needs far more than 4 MiB of scratch
    lay = abi.make_layer(M, K, N)
    assert abi.mpc_workspace_size(lay, abi.MPC_WS_TAG_COMPACT) > abi.MPC_NOALLOC_SCRATCH_BYTES
    fake = [0x1000] * 12
    st = lib.mpc_linear_tag_compact_noalloc(ctypes.byref(lay), *fake, None)
    assert st == abi.MPC_E_SCRATCH_LIMIT
    assert "MPC_NOALLOC_SCRATCH_BYTES" in abi.mpc_status_str(st)
