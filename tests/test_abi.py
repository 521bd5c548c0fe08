"""The C ABI library builds, loads and exports every declared symbol; host-side
validation rejects bad arguments before any launch (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2311_04406_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abi.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mpclinear.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpc_[a-z_]+)\s*\(", src)))


def test_header_declares_abi():
    assert declared_functions() == sorted(abi.ABI_FUNCTIONS)


def test_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_layout_matches_header(lib):
    assert ctypes.sizeof(abi.mpc_ring) == 12
    assert abi.mpc_layer.M.offset == 0 and abi.mpc_layer.N.offset == 16
    assert abi.mpc_layer.ring.offset == 24 and abi.mpc_layer.party.offset == 36
    assert ctypes.sizeof(abi.mpc_layer) == 48


def test_status_strings(lib):
    assert abi.mpc_status_str(0) == "ok"
    for s in range(-9, 0):
        assert abi.mpc_status_str(s) != "unknown status"
    assert abi.mpc_version() >= 100


def test_workspace_sizes(lib):
    L = abi.make_layer(128, 4096, 4096)
    assert abi.mpc_workspace_size(L, abi.MPC_WS_TAG_COMPACT) > 0
    assert abi.mpc_workspace_size(L, abi.MPC_WS_CHECK_COMPACT) == 0
    assert abi.mpc_workspace_size(L, abi.MPC_WS_CHECK_BATCHREC) > 0
    bad = abi.make_layer(4, 4, 4, k=30, s=32)
    assert abi.mpc_workspace_size(bad, abi.MPC_WS_TAG_COMPACT) == 0
    L2 = abi.make_layer(64, 128, 64, k=64, s=64)
    assert abi.mpc_workspace_size(L2, abi.MPC_WS_TAG_COMPACT) >= \
        abi.mpc_workspace_size(abi.make_layer(64, 128, 64), abi.MPC_WS_TAG_COMPACT)


def _call_share(lib, layer, ptrs):
    return lib.mpc_linear_share(ctypes.byref(layer), *ptrs, None, 0, None)


def test_validation_rejects_before_launch(lib):
    good = [0x1000] * 6
    L = abi.make_layer(4, 4, 4)
    # NULL operand
    assert _call_share(lib, L, [None] + good[1:]) == -1
    # misaligned operand
    assert _call_share(lib, L, [0x1008] + good[1:]) == -4
    # unsupported ring
    assert _call_share(lib, abi.make_layer(4, 4, 4, k=16, s=32), good) == -3
    # negative shape
    assert _call_share(lib, abi.make_layer(-1, 4, 4), good) == -2
    # party outside [0, nparties)
    assert _call_share(lib, abi.make_layer(4, 4, 4, party=2, nparties=2), good) == -8
    # null layer
    assert lib.mpc_linear_share(None, *good, None, 0, None) == -1
    # unknown tag mode / check mode
    args = [0x1000] * 12
    assert lib.mpc_linear_tag(ctypes.byref(L), 7, *args, None, 0, None) == -7
    assert lib.mpc_tag_check(ctypes.byref(L), 9, *([0x1000] * 5), None, 0, None) == -7
    # compact tag without workspace
    assert lib.mpc_linear_tag(ctypes.byref(L), abi.MPC_TAG_COMPACT, *args, None, 0, None) == -5


def test_empty_layers_are_noops(lib):
    # zero-sized layers enqueue nothing, so they succeed without a GPU
    L = abi.make_layer(0, 5, 4)
    assert _call_share(lib, L, [None, 0x1000, None, 0x1000, None, None]) == 0
    L = abi.make_layer(5, 4, 0)
    assert _call_share(lib, L, [0x1000, None, 0x1000, None, None, None]) == 0
