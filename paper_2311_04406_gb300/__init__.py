"""GB300-native SPDZ2k linear layers with CompactTag (arXiv 2311.04406).

One party's online computation of an actively secure linear layer Z = X . W
over Z_{2^{k+s}}: the Beaver-triple share, the CompactTag tag and check, and the
full SPDZ2k tag as the baseline, as CUDA kernels for sm_103a behind a C ABI
(include/mpclinear.h).  `abi` is the ctypes binding with the C names.
"""
from . import costmodel  # noqa: F401

__all__ = ["abi", "costmodel", "build"]


def __getattr__(name):
    if name in ("abi", "build"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
