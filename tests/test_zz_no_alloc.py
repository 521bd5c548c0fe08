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

import synth
from paper_2311_04406_gb300 import abi, build

pytestmark = pytest.mark.gpu


def _inputs(ring, M, K, N, seed):
    b = ring.bits
    g = lambda name, shape, bits=b: synth.uniform(seed, synth.TID[name], 0, shape, bits)
    return dict(alpha=g("alpha", (1,), ring.s), E=g("E", (M, K)), F=g("F", (K, N)),
                mA=g("mA", (M, K)), mB=g("mB", (K, N)), mC=g("mC", (M, N)), mR=g("mR", (M, N)),
                Dt=g("Dt", (M, N)), chi=g("chi", (N,), ring.s))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _pad(words, ring):
    return words if ring.words == 1 else words + (2,)


def _both(ring, M, K, N, seed):
    x = {k: _dev(v) for k, v in _inputs(ring, M, K, N, seed).items()}
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
    return outs


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
        (ref, got) = _both(ring, M, K, N, seed)
        for a, b, name in zip(ref, got, ("mZ", "mDc", "Dc")):
            assert torch.equal(a, b), f"{name} differs for {(M, K, N)} w={ring.words}"


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
