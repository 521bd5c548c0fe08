"""The serving loop (continuous batching over grouped calls, memory-gated
admission): every request's outputs are the same bit for bit whether it is
served alone or in a mix, and they equal the oracle's."""
import numpy as np
import pytest

import oracle as O
import synth
from paper_2311_04406_gb300 import abi, build
from paper_2311_04406_gb300.serve import Server, make_requests, request_bytes

from gpuhelp import host

pytestmark = pytest.mark.gpu

OUT_KEYS = ("Z", "mZ", "mDc", "Dc", "cs")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    abi.load()


def fresh(reqs):
    """The same requests, not yet served."""
    from paper_2311_04406_gb300.serve import Request
    return [Request(r.rid, r.model, r.batch, r.arrival, r.seed, r.layers) for r in reqs]


def outputs(r):
    return [{k: host(d[k]) for k in OUT_KEYS} for d in r.bufs]


@pytest.mark.parametrize("graphs", [False, True], ids=["eager", "graphs"])
@pytest.mark.parametrize("budget_gb", [3, 24])
def test_alone_equals_mixed(budget_gb, graphs):
    reqs = make_requests(6, 1000.0, seed=3, max_batch=2)
    srv = Server(ring=synth.Z128, mem_budget=int(budget_gb * 2**30), ws_bytes=1 << 30, graphs=graphs)
    stats = srv.run(reqs, keep_outputs=True)
    assert stats["requests"] == 6
    mixed = {r.rid: outputs(r) for r in reqs}
    for r in fresh(reqs):
        srv.run([r], keep_outputs=True)
        alone = outputs(r)
        for li, (a, b) in enumerate(zip(alone, mixed[r.rid])):
            for k in OUT_KEYS:
                assert np.array_equal(a[k], b[k]), f"request {r.rid} layer {li} {k}"
    assert abi.mpc_device_status() == 0


def test_memory_gate_limits_residency():
    reqs = make_requests(5, 1e6, seed=4, max_batch=2)
    biggest = max(request_bytes(r.layers, 2) for r in reqs)
    srv = Server(ring=synth.Z128, mem_budget=biggest + 256, ws_bytes=1 << 30)
    stats = srv.run(reqs)
    assert stats["requests"] == 5
    assert stats["peak_resident_bytes"] <= biggest + 1


def test_served_layers_match_oracle():
    """One request's small layers against the oracle (full outputs)."""
    reqs = make_requests(3, 1e6, seed=5, max_batch=1, models=("resnet18",))
    Server(ring=synth.Z128, mem_budget=16 * 2**30, ws_bytes=1 << 30).run(reqs, keep_outputs=True)
    bits = 128
    r = reqs[1]
    checked = 0
    for L, d in zip(r.layers, r.bufs):
        if L.M * L.K * L.N > 3e7:
            continue
        g = {k: host(d[k]) for k in ("E", "F", "A", "B", "C", "mA", "mB", "mC", "mR", "Dt", "chi", "alpha",
                                      "chi_hat")}
        Z = O.linear_share(bits, 0, g["E"], g["F"], g["A"], g["B"], g["C"])
        assert np.array_equal(host(d["Z"]), Z), L
        mDc, Dc, _ = O.compact_tag(bits, g["alpha"], g["E"], g["F"], g["mA"], g["mB"], g["mC"], g["mR"], g["Dt"],
                                   g["chi"])
        assert np.array_equal(host(d["mDc"]), mDc) and np.array_equal(host(d["Dc"]), Dc), L
        assert np.array_equal(host(d["mZ"]), O.optmac(bits, g["alpha"], g["mR"], g["Dt"])), L
        cs = O.check_compact(bits, g["alpha"], g["chi_hat"], Dc, mDc)
        assert np.array_equal(host(d["cs"]).reshape(-1), cs.reshape(-1)), L
        checked += 1
    assert checked >= 3


def test_replayed_ticks_equal_eager_ticks():
    """Graphs on: three runs of same-shaped requests with different shares.
    Their ticks recur (same arena ranges, same layers): the first run issues
    them eagerly, the second captures them, the third replays them.  Every
    run's outputs equal those of an eager server on the same requests."""
    def wave(seed):
        return make_requests(4, 1e9, seed=seed, max_batch=1, models=("resnet18",), all_at_once=True)
    srv = Server(ring=synth.Z128, mem_budget=8 * 2**30, ws_bytes=1 << 30, graphs=True)
    ref = Server(ring=synth.Z128, mem_budget=8 * 2**30, ws_bytes=1 << 30, graphs=False)
    counts = []
    for run, seed in enumerate((11, 12, 13)):
        reqs = wave(seed)
        srv.run(reqs, keep_outputs=True)
        counts.append(dict(srv.tick_counts))
        got = {r.rid: outputs(r) for r in reqs}
        again = fresh(reqs)
        ref.run(again, keep_outputs=True)
        for r in again:
            for li, (a, b) in enumerate(zip(outputs(r), got[r.rid])):
                for k in OUT_KEYS:
                    assert np.array_equal(a[k], b[k]), f"run {run} request {r.rid} layer {li} {k}"
    assert counts[0]["replayed"] == 0 and counts[0]["eager"] > 0
    assert counts[1]["captured"] > 0
    assert counts[2]["replayed"] > 0 and counts[2]["captured"] == 0
    assert abi.mpc_device_status() == 0


def test_grouped_checks_and_openings_match_single_calls():
    """mpc_tag_check_grouped and mpc_lincomb_grouped against the one-layer calls."""
    import torch
    rng = np.random.default_rng(7)
    for ring in (synth.Z64, synth.Z128):
        w = ring.words
        shp = lambda *d: d + ((2,) if w == 2 else ())
        R = lambda *d: torch.from_numpy(rng.integers(0, 2**63, shp(*d), dtype=np.int64)).cuda()
        Ms = [1, 7, 64, 513, 3000, 0, 77]
        layers = [abi.make_layer(M, 1, 1, ring.k, ring.s) for M in Ms]
        ptrs = [dict(alpha_i=R(1), chi_hat=R(M), Dc=R(M), mDc_i=R(M), cs_i=R(1)) for M in Ms]
        abi.mpc_tag_check_grouped(layers * 10, ptrs * 10)   # 70 layers: two launches
        for L, d in zip(layers, ptrs):
            cs = torch.zeros_like(d["cs_i"]) - 1
            abi.mpc_tag_check(L, abi.MPC_CHECK_COMPACT, d["alpha_i"], d["chi_hat"], d["Dc"], d["mDc_i"], cs)
            assert torch.equal(cs, d["cs_i"]), (ring, L.M)
        ns = [5, 1, 4096, 0, 999, 70000] * 12          # 72 groups: two launches, empty ones skipped
        ins = [[R(n), R(n), R(n)] for n in ns]
        outs = [torch.zeros(shp(n), dtype=torch.int64, device="cuda") for n in ns]
        abi.mpc_lincomb_grouped(ring.k, ring.s, [1, -1, 3], ins, outs)
        for x, o in zip(ins, outs):
            ref = torch.zeros_like(o)
            abi.mpc_lincomb(ring.k, ring.s, [1, -1, 3], x, ref)
            assert torch.equal(ref, o)
    torch.cuda.synchronize()
    assert abi.mpc_device_status() == 0
