"""GPU parity of the truncated layer (§3.4, Fig. Pi_OptMAC&Trunc and the
truncated Fig. Pi_CompactMatMul): every output equals the oracle bit for bit."""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import dealer
from paper_2311_04406_gb300 import abi, build

from gpuhelp import (gpu_check_compact, gpu_optmac_trunc, gpu_public_product, gpu_share_trunc,
                     gpu_tag_compact_trunc)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    abi.load()


CASES = [(synth.Z64, (64, 128, 64), 16), (synth.Z64, (300, 640, 96), 13), (synth.Z64, (3, 500, 70), 8),
         (synth.Z64, (65, 37, 67), 20), (synth.Z128, (130, 256, 40), 24), (synth.Z128, (5, 77, 9), 1),
         (synth.Z64, (40, 30, 20), 0)]


@pytest.mark.parametrize("ring,shape,f", CASES, ids=lambda x: str(x) if isinstance(x, tuple) else None)
def test_truncated_layer_parity(ring, shape, f):
    M, K, N = shape
    t = dealer.deal_trunc(ring, M, K, N, n=2, seed=M + K + N + f, f=f)
    d = t.base
    ref = dealer.run_layer_trunc(t)
    P = gpu_public_product(ring, d.E, d.F)
    assert np.array_equal(P, ref["P"]), "public product"
    for i, p in enumerate(d.parties):
        Z = gpu_share_trunc(ring, i, d.E, d.F, p.A, p.B, p.C)
        assert np.array_equal(Z, ref["Z"][i]), f"share party {i}"
        Zf, mZf = gpu_optmac_trunc(ring, i, f, p.alpha, t.Rf_shares[i], t.mRf_shares[i], ref["Dt"], P)
        assert np.array_equal(Zf, ref["Zf"][i]), f"truncated share party {i}"
        assert np.array_equal(mZf, ref["mZf"][i]), f"truncated tag party {i}"
        mDc, Dc = gpu_tag_compact_trunc(ring, i, p.alpha, d.E, d.F, p.mA, p.mB, p.mC, p.mR, ref["Dt"], d.chi)
        assert np.array_equal(mDc, ref["mDc"][i]), f"compact tag party {i}"
        assert np.array_equal(Dc, ref["Dc"])
        cs = gpu_check_compact(ring, p.alpha, d.chi_hat, Dc, mDc)
        assert np.array_equal(cs.reshape(-1), ref["cs"][i].reshape(-1))
    assert abi.mpc_device_status() == 0


def test_optmac_trunc_rejects_bad_f():
    import ctypes
    lib = abi.load()
    L = abi.make_layer(4, 4, 4)
    fake = [0x1000] * 7
    assert lib.mpc_optmac_trunc(ctypes.byref(L), 33, *fake, None) == -2
    assert lib.mpc_optmac_trunc(ctypes.byref(L), -1, *fake, None) == -2
