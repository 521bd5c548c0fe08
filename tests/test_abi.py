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
    return sorted(set(re.findall(r"\b(mpc_[a-z0-9_]+)\s*\(", src)))


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


@pytest.mark.hidden_gpu
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


@pytest.mark.hidden_gpu
def test_empty_layers_are_noops(lib):
    # zero-sized layers enqueue nothing, so they succeed without a GPU
    L = abi.make_layer(0, 5, 4)
    assert _call_share(lib, L, [None, 0x1000, None, 0x1000, None, None]) == 0
    L = abi.make_layer(5, 4, 0)
    assert _call_share(lib, L, [0x1000, None, 0x1000, None, None, None]) == 0


@pytest.mark.hidden_gpu
def test_grouped_host_logic(lib):
    """Grouped calls: workspace and launch counts are the sums over the group;
    invalid groups are rejected before any launch."""
    layers = [abi.make_layer(128, 4096, 4096), abi.make_layer(4, 512, 300), abi.make_layer(1024, 576, 64),
              abi.make_layer(64, 256, 256)]
    tc = [abi.mpc_gemm_path(L) for L in layers]
    assert tc == [1, 0, 1, 1]
    ws = abi.mpc_workspace_size_grouped(layers, abi.MPC_WS_SHARE)
    assert ws == sum(-(-abi.mpc_workspace_size(L, abi.MPC_WS_SHARE) // 256) * 256 for L in layers)
    cws = abi.mpc_workspace_size_grouped(layers, abi.MPC_WS_TAG_COMPACT)
    assert cws == sum(-(-abi.mpc_workspace_size(L, abi.MPC_WS_TAG_COMPACT) // 256) * 256 for L in layers)
    # one prologue + GEMM pair per tile: the 128-row tile (128 x 4096 x 4096), the tall tile
    # (set for 1024 x 576 x 64: tall and narrow; the built-in rule takes it from 2048 rows), the
    # wide tile (M = 64: two of its 32-row tiles); one kernel for the integer-pipe layer
    assert [abi.mpc_autotune_choice(L)[4] for L in layers] == [128, 0, 128, 32]
    abi.mpc_autotune_set(layers[2], 1, 8, 0, tile_rows=-128)
    assert abi.mpc_launch_count_grouped(layers, abi.MPC_WS_SHARE) == 2 + 2 + 2 + 1
    # 30 layers of each tile: one launch pair per tile (at most 64 layers each)
    assert abi.mpc_launch_count_grouped(layers * 30, abi.MPC_WS_TAG_FULL) == 3 * 2 + 30
    assert abi.mpc_launch_count_grouped(layers[:1] * 65, abi.MPC_WS_TAG_FULL) == 2 * 2
    # a layer with units for >= 64 waves of the grid (2048 x 4096 x 4096: 131072 units) gets a
    # launch pair of its own
    long_ = abi.make_layer(2048, 4096, 4096)
    assert abi.mpc_launch_count_grouped([long_] + layers, abi.MPC_WS_SHARE) == 2 + 2 + 2 + 2 + 1
    abi.mpc_autotune_clear()
    # the CompactTag tags of a group: rows, finalize and vec passes, one launch each per 64 layers
    assert abi.mpc_launch_count_grouped(layers, abi.MPC_WS_TAG_COMPACT) == 3
    assert abi.mpc_launch_count_grouped(layers * 20, abi.MPC_WS_TAG_COMPACT) == 6
    assert abi.mpc_launch_count_grouped([abi.make_layer(0, 4, 4)], abi.MPC_WS_TAG_COMPACT) == 0
    mixed = [abi.make_layer(8, 8, 8), abi.make_layer(8, 8, 8, 64, 64)]
    assert abi.mpc_launch_count_grouped(mixed, abi.MPC_WS_SHARE) == abi.MPC_E_RING
    assert abi.mpc_workspace_size_grouped(mixed, abi.MPC_WS_SHARE) == 0
    arr = (abi.mpc_layer * 2)(*mixed)
    ptrs = (abi.mpc_share_ptrs * 2)()
    assert lib.mpc_linear_share_grouped(arr, 2, ptrs, None, 0, None) == abi.MPC_E_RING
    assert lib.mpc_linear_share_grouped(arr, -1, ptrs, None, 0, None) == abi.MPC_E_SHAPE
    assert lib.mpc_linear_share_grouped(None, 0, None, None, 0, None) == 0
    assert lib.mpc_linear_share_grouped(None, 2, ptrs, None, 0, None) == abi.MPC_E_NULL
    tptrs = (abi.mpc_tag_ptrs * 2)()
    same = (abi.mpc_layer * 2)(abi.make_layer(8, 8, 8), abi.make_layer(8, 8, 8))
    assert lib.mpc_linear_tag_grouped(same, 2, 9, tptrs, None, 0, None) == abi.MPC_E_MODE
    # NULL operands in a group are caught before any launch
    assert lib.mpc_linear_tag_grouped(same, 2, abi.MPC_TAG_FULL, tptrs, None, 0, None) == abi.MPC_E_NULL
    # a tensor-core group without its workspace
    big = (abi.mpc_layer * 1)(abi.make_layer(128, 256, 256))
    p1 = (abi.mpc_share_ptrs * 1)()
    for f in abi.SHARE_PTR_FIELDS:
        setattr(p1[0], f, 0x1000)
    assert lib.mpc_linear_share_grouped(big, 1, p1, None, 0, None) == abi.MPC_E_WORKSPACE
    assert lib.mpc_linear_share_grouped(big, 1, p1, 0x1010, 1 << 30, None) == abi.MPC_E_ALIGN


def test_launch_table_host_logic(lib, tmp_path):
    """The autotune table: set / query / save / load / clear, and rejection of
    choices the kernels cannot run (no GPU needed)."""
    abi.mpc_autotune_clear()
    big = abi.make_layer(128, 4096, 4096)
    small = abi.make_layer(64, 128, 64)
    skinny = abi.make_layer(4, 512, 512)
    assert abi.mpc_autotune_choice(big) == (1, 0, 0, False, 128)      # built-in rule
    assert abi.mpc_autotune_choice(small)[0] == 0
    assert abi.mpc_autotune_choice(abi.make_layer(64, 4608, 512)) == (1, 0, 0, False, 32)     # wide tile
    assert abi.mpc_autotune_choice(abi.make_layer(65, 4608, 512)) == (1, 0, 0, False, 128)
    assert abi.mpc_autotune_choice(abi.make_layer(32, 4608, 512, 64, 64)) == (1, 0, 0, False, 16)
    # the built-in tile rule's thresholds (host logic only)
    rows = lambda M, K, N, *ring: abi.mpc_autotune_choice(abi.make_layer(M, K, N, *ring))[4]
    assert rows(64, 2304, 256, 64, 64) == 16      # Z_2^128, 33-64 rows: wide once it has a unit per SM
    assert rows(64, 576, 128, 64, 64) == 64       # 72 wide units: 64-row tiles
    assert rows(2048, 576, 64) == -128 and rows(1024, 576, 64) == 128          # Z_2^64 tall from 2048 rows
    assert rows(1024, 576, 64, 64, 64) == -128 and rows(512, 576, 64, 64, 64) == 128   # Z_2^128 from 1024
    assert rows(4096, 1152, 128) == -128 and rows(2048, 1152, 128, 64, 64) == 128      # N = 128 from 4096
    assert rows(8192, 2304, 256, 64, 64) == 128   # N > 128: 128-row tiles
    assert rows(4096, 575, 64) == 128             # odd K in Z_2^64: no tall tile
    abi.mpc_autotune_set(small, 1, 4, 0, tile_rows=32)                 # the Z_2^64 wide tile
    with pytest.raises(abi.MpcError):
        abi.mpc_autotune_set(abi.make_layer(64, 128, 64, 64, 64), 1, 4, 0, tile_rows=32)   # Z_2^128: 16
    ws_before = abi.mpc_workspace_size(small, abi.MPC_WS_SHARE)
    abi.mpc_autotune_set(small, 1, 4, 0)
    assert abi.mpc_autotune_choice(small) == (1, 4, 0, True, 128)
    abi.mpc_autotune_set(small, 1, 4, 0, tile_rows=64)
    assert abi.mpc_autotune_choice(small) == (1, 4, 0, True, 64)
    assert abi.mpc_gemm_path(small) == 1
    assert abi.mpc_workspace_size(small, abi.MPC_WS_SHARE) == ws_before   # independent of the table
    abi.mpc_autotune_set(big, 0, 0, 8)
    assert abi.mpc_gemm_path(big) == 0
    # the tensor-core kernel cannot run M <= 8 or odd N in Z_2^64
    with pytest.raises(abi.MpcError):
        abi.mpc_autotune_set(skinny, 1, 8, 0)
    with pytest.raises(abi.MpcError):
        abi.mpc_autotune_set(abi.make_layer(64, 64, 63), 1, 8, 0)
    with pytest.raises(abi.MpcError):
        abi.mpc_autotune_set(small, 1, 0, 0)
    with pytest.raises(abi.MpcError):
        abi.mpc_autotune_set(small, 1, 4, 0, tile_rows=48)      # tensor-core tiles: 128, 64 or the wide tile
    with pytest.raises(abi.MpcError):
        abi.mpc_autotune_set(small, 0, 0, 2, tile_rows=128)     # integer pipes: 64, 16 or 0
    f = tmp_path / "table.txt"
    assert abi.mpc_autotune_save(str(f)) == 2
    lines = f.read_text().split("\n")
    assert lines[0] == "mpclinear-autotune 2" and "1 64 128 64 1 64 4 0" in lines
    assert abi.mpc_autotune_clear() == 2
    assert abi.mpc_autotune_choice(small)[3] is False
    assert abi.mpc_autotune_load(str(f)) == 2
    assert abi.mpc_autotune_choice(small) == (1, 4, 0, True, 64)
    old = tmp_path / "v1.txt"                                    # version 1: no tile height, 128 rows
    old.write_text("mpclinear-autotune 1\n1 64 128 64 1 8 0\n")
    assert abi.mpc_autotune_load(str(old)) == 1
    assert abi.mpc_autotune_choice(small) == (1, 8, 0, True, 128)
    bad = tmp_path / "bad.txt"
    bad.write_text("mpclinear-autotune 1\n1 4 512 512 1 8 0\n")   # tensor cores on M = 4
    with pytest.raises(abi.MpcError):
        abi.mpc_autotune_load(str(bad))
    bad.write_text("something else\n")
    with pytest.raises(abi.MpcError):
        abi.mpc_autotune_load(str(bad))
    with pytest.raises(abi.MpcError):
        abi.mpc_autotune_load(str(tmp_path / "missing.txt"))
    assert abi.mpc_autotune([]) == 0
    abi.mpc_autotune_clear()
    assert abi.mpc_gemm_path(big) == 1


@pytest.mark.hidden_gpu
def test_lincomb_validation(lib):
    import ctypes
    ring = abi.mpc_ring(32, 32, 1)
    c = (ctypes.c_int64 * 17)(*([1] * 17))
    p = (ctypes.c_void_p * 17)(*([0x1000] * 17))
    R = ctypes.byref(ring)
    assert lib.mpc_lincomb(R, 8, 0, c, p, 0x2000, None) == abi.MPC_E_SHAPE
    assert lib.mpc_lincomb(R, 8, 17, c, p, 0x2000, None) == abi.MPC_E_SHAPE
    assert lib.mpc_lincomb(R, -1, 2, c, p, 0x2000, None) == abi.MPC_E_SHAPE
    assert lib.mpc_lincomb(None, 8, 2, c, p, 0x2000, None) == abi.MPC_E_NULL
    assert lib.mpc_lincomb(R, 8, 2, c, p, 0x2008, None) == abi.MPC_E_ALIGN
    q = (ctypes.c_void_p * 2)(0x1000, None)
    assert lib.mpc_lincomb(R, 8, 2, c, q, 0x2000, None) == abi.MPC_E_NULL
    assert lib.mpc_lincomb(R, 0, 2, c, p, None, None) == 0          # nothing to do, nothing launched


@pytest.mark.hidden_gpu
def test_im2col_validation(lib):
    import ctypes
    ring = abi.mpc_ring(32, 32, 1)
    R = ctypes.byref(ring)
    assert lib.mpc_im2col(R, 1, 1, 4, 4, 3, 3, 1, 0x1000, 0x2000, None) == abi.MPC_E_SHAPE
    assert lib.mpc_im2col(R, 1, 1, 4, 4, 3, 1, 0, 0x1000, 0x2000, None) == abi.MPC_E_SHAPE
    assert lib.mpc_im2col(R, 1, 1, 1, 1, 5, 1, 1, 0x1000, 0x2000, None) == abi.MPC_E_SHAPE
    assert lib.mpc_im2col(R, 1, 1, 4, 4, 3, 1, 1, 0x1008, 0x2000, None) == abi.MPC_E_ALIGN
    assert lib.mpc_im2col(R, 0, 3, 4, 4, 3, 1, 1, None, None, None) == 0        # empty batch


def test_compact_launch_counts(lib):
    """CompactTag launches: rows + finalize + vec when a row is split into
    several chunks (the dense layer: M + K rows too few to fill the GPU, N >
    1024), rows + vec when every row is one chunk (the vec pass then reads the
    K-side partials in place)."""
    assert abi.mpc_launch_count(abi.make_layer(128, 4096, 4096), abi.MPC_WS_TAG_COMPACT) == 3
    assert abi.mpc_launch_count(abi.make_layer(1024, 576, 64), abi.MPC_WS_TAG_COMPACT) == 2
    assert abi.mpc_launch_count(abi.make_layer(8192, 1024, 4096), abi.MPC_WS_TAG_COMPACT) == 2
    assert abi.mpc_launch_count(abi.make_layer(0, 8, 8), abi.MPC_WS_TAG_COMPACT) == 0


@pytest.mark.hidden_gpu
def test_grouped_check_and_lincomb_validation(lib):
    """mpc_tag_check_grouped / mpc_lincomb_grouped reject bad groups before any launch."""
    layers = (abi.mpc_layer * 2)(abi.make_layer(8, 1, 1), abi.make_layer(8, 1, 1))
    ptrs = (abi.mpc_check_ptrs * 2)()
    for i in range(2):
        for f in abi.CHECK_PTR_FIELDS:
            setattr(ptrs[i], f, 0x1000)
    assert lib.mpc_tag_check_grouped(layers, 0, ptrs, None) == 0            # nothing to do
    assert lib.mpc_tag_check_grouped(layers, -1, ptrs, None) == abi.MPC_E_SHAPE
    assert lib.mpc_tag_check_grouped(None, 2, ptrs, None) == abi.MPC_E_NULL
    ptrs[1].Dc = 0x1008
    assert lib.mpc_tag_check_grouped(layers, 2, ptrs, None) == abi.MPC_E_ALIGN
    ptrs[1].Dc = None
    assert lib.mpc_tag_check_grouped(layers, 2, ptrs, None) == abi.MPC_E_NULL
    ptrs[1].Dc = 0x1000
    mixed = (abi.mpc_layer * 2)(abi.make_layer(8, 1, 1), abi.make_layer(8, 1, 1, 64, 64))
    assert lib.mpc_tag_check_grouped(mixed, 2, ptrs, None) == abi.MPC_E_RING
    ring = abi.mpc_ring(32, 32, 1)
    R = ctypes.byref(ring)
    n = (ctypes.c_int64 * 2)(8, 16)
    c = (ctypes.c_int64 * 3)(1, -1, 1)
    ins = (ctypes.c_void_p * 6)(*([0x1000] * 6))
    outs = (ctypes.c_void_p * 2)(0x2000, 0x3000)
    assert lib.mpc_lincomb_grouped(R, 0, n, 3, c, ins, outs, None) == 0
    assert lib.mpc_lincomb_grouped(R, 2, n, 5, c, ins, outs, None) == abi.MPC_E_SHAPE    # at most 4 terms
    assert lib.mpc_lincomb_grouped(R, -1, n, 3, c, ins, outs, None) == abi.MPC_E_SHAPE
    assert lib.mpc_lincomb_grouped(None, 2, n, 3, c, ins, outs, None) == abi.MPC_E_NULL
    bad = (ctypes.c_void_p * 6)(0x1000, 0x1000, 0x1000, 0x1000, 0x1008, 0x1000)
    assert lib.mpc_lincomb_grouped(R, 2, n, 3, c, bad, outs, None) == abi.MPC_E_ALIGN
    neg = (ctypes.c_int64 * 2)(8, -1)
    assert lib.mpc_lincomb_grouped(R, 2, neg, 3, c, ins, outs, None) == abi.MPC_E_SHAPE


def test_binding_rejects_short_tensors_before_the_call():
    """The binding checks every tensor argument against the element counts the
    header gives for the call, so a buffer that is too short (here: s-bit
    values stored one word each for Z_2^128, where the call reads ring
    elements of two words) raises before any kernel could read past its end."""
    import torch
    M, K, N = 5, 3, 7
    lay = abi.make_layer(M, K, N, 64, 64)
    full = lambda *shape: torch.zeros(shape + (2,), dtype=torch.int64)
    x = dict(alpha_i=full(1), E=full(M, K), F=full(K, N), mA_i=full(M, K), mB_i=full(K, N), mC_i=full(M, N),
             mR_i=full(M, N), Dtilde=full(M, N), chi=full(N), mZ_i=full(M, N), mDc_i=full(M), Dc=full(M))
    # the right sizes pass the check
    assert len(abi._args("f", lay, abi._tag_elems(M, K, N, abi.MPC_TAG_COMPACT), x)) == 12
    short = dict(x, chi=torch.zeros(N, dtype=torch.int64))
    with pytest.raises(ValueError, match="chi"):
        abi.mpc_linear_tag(lay, abi.MPC_TAG_COMPACT, **short)
    with pytest.raises(ValueError, match="alpha_i"):
        abi.mpc_linear_tag_compact_noalloc(lay, **dict(x, alpha_i=torch.zeros(1, dtype=torch.int64)))
    with pytest.raises(ValueError, match="not contiguous"):
        abi.mpc_linear_share(lay, x["E"], full(N, K).transpose(0, 1), x["mA_i"], x["mB_i"], x["mC_i"], x["mZ_i"])
    with pytest.raises(ValueError, match="Z_i"):
        abi.mpc_linear_share(lay, x["E"], x["F"], x["mA_i"], x["mB_i"], x["mC_i"], full(M, N - 1))
    # inputs the mode ignores are not checked; the ones it reads are
    assert abi._args("f", lay, abi._tag_elems(M, K, N, abi.MPC_TAG_FULL), dict(x, chi=full(1)))
    with pytest.raises(ValueError, match="tag_i"):
        abi.mpc_tag_check(lay, abi.MPC_CHECK_COMPACT, x["alpha_i"], x["Dc"], x["Dc"], full(M - 1), full(1))
    # the seeded check's chi_hat is one 64-bit seed word
    seed = torch.zeros(1, dtype=torch.int64)
    with pytest.raises(ValueError, match="opened"):
        abi.mpc_tag_check(lay, abi.MPC_CHECK_BATCHREC_SEEDED, x["alpha_i"], seed, full(M), x["mC_i"], full(1))
    # grouped calls name the layer
    lays = [abi.make_layer(M, K, N, 64, 64), abi.make_layer(M + 1, K, N, 64, 64)]
    with pytest.raises(ValueError, match=r"layers\[1\]\.E"):
        abi.mpc_linear_tag_grouped(lays, abi.MPC_TAG_COMPACT, [x, x])
    with pytest.raises(ValueError, match=r"layers\[1\]\.chi_hat"):
        abi.mpc_tag_check_grouped(lays, [dict(alpha_i=x["alpha_i"], chi_hat=x["Dc"], Dc=x["Dc"], mDc_i=x["Dc"],
                                              cs_i=x["alpha_i"])] * 2)
    with pytest.raises(ValueError, match=r"ins\[1\]\[0\]"):
        abi.mpc_lincomb_grouped(64, 64, [1], [[full(4)], [full(3)]], [full(4), full(4)])
    with pytest.raises(ValueError, match="dst"):
        abi.mpc_transpose(64, 64, 3, 4, full(3, 4), full(11))
    with pytest.raises(ValueError, match="dst"):
        abi.mpc_im2col(64, 64, 1, 2, 5, 5, 3, 1, 1, full(2, 5, 5), full(25, 17))
