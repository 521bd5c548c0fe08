"""Continuous-batching serving loop over the grouped C ABI calls.

One party's online linear-layer work for a stream of inference requests
(ResNet-18 or VGG16 on 32x32x3 images, batch 1-32, shares in Z_2^128).  Each
request brings its own authenticated shares for every linear layer (fresh
triples per inference, §2.5), held resident in HBM from admission to
completion.  The scheduler

  * admits arrived requests first-come first-served while their shares fit a
    device-memory budget (memory-gated admission);
  * materialises an admitted request's shares on a side stream (device copies
    out of a seeded pool of uniform words standing in for the offline phase's
    output), so that input preparation overlaps the layers already running;
  * runs one "tick" at a time: the next linear layer of every admitted,
    ready request, as ONE grouped share call, ONE grouped tag call and the
    per-layer checks (continuous batching: a request joins at the next tick
    after admission and leaves after its last layer, whatever the others are
    doing);
  * keeps at most `max_inflight` ticks queued on the device, and releases a
    finished request's memory once its last tick has completed.

Latency is measured on the device clock: a start event is recorded when the
run begins, each tick records an event, and a request's completion time is
its last tick's event.  Arrival times are host times from the same start.

The grouped calls compute every layer exactly as the per-layer calls do, so a
request's outputs do not depend on which other requests share its ticks
(tests/test_gpu_serve.py checks alone against mixed).
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np

import synth

from . import abi

MODELS = {"resnet18": synth.resnet18_layers, "vgg16": synth.vgg16_layers}
KEYS_MK = ("E", "A", "mA")
KEYS_KN = ("F", "B", "mB")
KEYS_MN = ("C", "mC", "mR", "Dt")


@dataclass
class Request:
    rid: int
    model: str
    batch: int
    arrival: float                 # seconds after the run starts
    seed: int
    layers: list = field(default_factory=list)
    bufs: list = None              # per layer: dict of device tensors
    nxt: int = 0                   # next layer to run
    ready: object = None           # event: shares materialised
    done_ms: float = None          # device time of completion
    admit_s: float = None

    @property
    def units(self) -> int:
        """Ring MACs of the request's share products (2MKN per layer)."""
        return sum(2 * L.M * L.K * L.N for L in self.layers)


def request_bytes(layers, words: int) -> int:
    e = 8 * words
    tot = 0
    for L in layers:
        M, K, N = L.M, L.K, L.N
        tot += e * (3 * M * K + 3 * K * N + 4 * M * N + N)      # inputs
        tot += e * (2 * M * N + 2 * M + 1)                       # Z, mZ, mDc, Dc, cs
    return tot


def make_requests(n: int, rate: float, seed: int, max_batch: int = 32, models=("resnet18", "vgg16"),
                  all_at_once: bool = False) -> list:
    """n requests with Poisson arrivals at `rate` per second (all at t = 0 if
    all_at_once), model uniform over `models`, batch uniform in 1..max_batch."""
    g = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        if not all_at_once:
            t += float(g.exponential(1.0 / rate))
        m = models[int(g.integers(0, len(models)))]
        b = int(g.integers(1, max_batch + 1))
        out.append(Request(i, m, b, 0.0 if all_at_once else t, seed * 1000003 + i, MODELS[m](b)))
    return out


class Server:
    POOL_WORDS = 1 << 28          # 2 GiB of uniform words, larger than any one share tensor

    def __init__(self, ring=synth.Z128, party: int = 0, nparties: int = 2, mem_budget: int = 96 << 30,
                 tag: str = "compact", max_inflight: int = 2, max_group: int = 512, pool_seed: int = 0x5EED):
        import torch
        if tag not in ("compact", "full"):
            raise ValueError("tag must be 'compact' or 'full'")
        self.torch = torch
        self.ring, self.party, self.nparties = ring, party, nparties
        self.mem_budget, self.tag = mem_budget, tag
        self.max_inflight, self.max_group = max_inflight, max_group
        abi.load()
        gen = torch.Generator(device="cuda")
        gen.manual_seed(pool_seed)
        self.pool = torch.randint(-(1 << 63), (1 << 63) - 1, (self.POOL_WORDS,), dtype=torch.int64,
                                  device="cuda", generator=gen)

    # -- request shares -------------------------------------------------------
    def _materialise(self, req: Request, stream):
        """Allocate the request's shares and fill them on `stream` with copies
        of pool windows at offsets drawn from the request's seed (so the same
        request always gets the same shares)."""
        torch = self.torch
        w = self.ring.words
        shp = (lambda *d: d + ((2,) if w == 2 else ()))
        gen = torch.Generator(device="cuda")
        gen.manual_seed(req.seed)
        rng = np.random.default_rng(req.seed)
        bufs = []

        def window(shape):
            n = int(np.prod(shape))
            off = int(rng.integers(0, self.POOL_WORDS - n + 1))
            t = torch.empty(shape, dtype=torch.int64, device="cuda")
            t.view(-1).copy_(self.pool[off:off + n], non_blocking=True)
            return t

        with torch.cuda.stream(stream):
            for L in req.layers:
                M, K, N = L.M, L.K, L.N
                d = {}
                for k in KEYS_MK:
                    d[k] = window(shp(M, K))
                for k in KEYS_KN:
                    d[k] = window(shp(K, N))
                for k in KEYS_MN:
                    d[k] = window(shp(M, N))
                # key share and combiners: uniform in [0, 2^s) (s <= 63 here: 2^63 - 1 bound)
                smax = (1 << min(self.ring.s, 63)) - 1
                d["alpha"] = torch.zeros(shp(1), dtype=torch.int64, device="cuda")
                d["chi"] = torch.zeros(shp(N), dtype=torch.int64, device="cuda")
                d["chi_hat"] = torch.zeros(shp(M), dtype=torch.int64, device="cuda")
                for k, n_ in (("alpha", 1), ("chi", N), ("chi_hat", M)):
                    v = torch.randint(0, smax, (n_,), dtype=torch.int64, device="cuda", generator=gen)
                    if w == 2:
                        d[k][:, 0] = v
                    else:
                        d[k].copy_(v)
                d["Z"] = torch.empty(shp(M, N), dtype=torch.int64, device="cuda")
                d["mZ"] = torch.empty(shp(M, N), dtype=torch.int64, device="cuda")
                d["mDc"] = torch.empty(shp(M), dtype=torch.int64, device="cuda")
                d["Dc"] = torch.empty(shp(M), dtype=torch.int64, device="cuda")
                d["cs"] = torch.empty(shp(1), dtype=torch.int64, device="cuda")
                d["layer"] = abi.make_layer(M, K, N, self.ring.k, self.ring.s, self.party, self.nparties)
                bufs.append(d)
            ev = torch.cuda.Event()
            ev.record(stream)
        req.bufs = bufs
        req.ready = ev

    # -- one tick -------------------------------------------------------------
    def _tick(self, group, ws):
        a = abi
        layers = [r.bufs[r.nxt]["layer"] for r in group]
        bufs = [r.bufs[r.nxt] for r in group]
        a.mpc_linear_share_grouped(layers, [dict(E=d["E"], F=d["F"], A_i=d["A"], B_i=d["B"], C_i=d["C"],
                                                 Z_i=d["Z"]) for d in bufs], ws=ws)
        tp = [dict(alpha_i=d["alpha"], E=d["E"], F=d["F"], mA_i=d["mA"], mB_i=d["mB"], mC_i=d["mC"],
                   mR_i=d["mR"], Dtilde=d["Dt"], chi=d["chi"], mZ_i=d["mZ"], mDc_i=d["mDc"], Dc=d["Dc"])
              for d in bufs]
        if self.tag == "compact":
            a.mpc_linear_tag_grouped(layers, a.MPC_TAG_COMPACT, tp, ws=ws)
            for d in bufs:
                a.mpc_tag_check(d["layer"], a.MPC_CHECK_COMPACT, d["alpha"], d["chi_hat"], d["Dc"], d["mDc"],
                                d["cs"])
        else:
            a.mpc_linear_tag_grouped(layers, a.MPC_TAG_FULL, tp, ws=ws)

    def _workspace(self, group):
        torch = self.torch
        layers = [r.bufs[r.nxt]["layer"] for r in group]
        which = (abi.MPC_WS_SHARE, abi.MPC_WS_TAG_COMPACT if self.tag == "compact" else abi.MPC_WS_TAG_FULL)
        need = max(abi.mpc_workspace_size_grouped(layers, w) for w in which)
        check = max(abi.mpc_workspace_size(L, abi.MPC_WS_CHECK_COMPACT) for L in layers)
        need = max(need, check, 256)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(int(need * 1.25), dtype=torch.uint8, device="cuda")
        return self._ws

    # -- the loop -------------------------------------------------------------
    def run(self, requests, keep_outputs: bool = False) -> dict:
        torch = self.torch
        st = torch.cuda.current_stream()
        side = torch.cuda.Stream()
        self._ws = None
        words = self.ring.words
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting = collections.deque()
        active = []
        inflight = collections.deque()      # (event, finished requests)
        tick_ms = []
        mem_used = 0
        peak_mem = 0
        start = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(st)
        t0 = time.perf_counter()
        prev_ev = start
        finished_all = []

        def retire(block: bool):
            nonlocal mem_used
            while inflight and (block or inflight[0][0].query()):
                ev, fin = inflight.popleft()
                ev.synchronize()
                t = start.elapsed_time(ev)
                for r in fin:
                    r.done_ms = t
                    mem_used -= request_bytes(r.layers, words)
                    if not keep_outputs:
                        r.bufs = None
                    finished_all.append(r)
                block = False

        while pending or waiting or active or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while waiting:
                need = request_bytes(waiting[0].layers, words)
                if mem_used + need > self.mem_budget and (active or inflight):
                    break
                r = waiting.popleft()
                mem_used += need
                peak_mem = max(peak_mem, mem_used)
                r.admit_s = time.perf_counter() - t0
                self._materialise(r, side)
                active.append(r)
            retire(block=False)
            if active:
                group = active[: self.max_group]
                for r in group:
                    if r.ready is not None:
                        st.wait_event(r.ready)
                        r.ready = None
                self._tick(group, self._workspace(group))
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(st)
                tick_ms.append((prev_ev, ev))
                prev_ev = ev
                fin = []
                for r in group:
                    r.nxt += 1
                    if r.nxt == len(r.layers):
                        fin.append(r)
                active = [r for r in active if r.nxt < len(r.layers)]
                inflight.append((ev, fin))
                while len(inflight) > self.max_inflight:
                    retire(block=True)
            elif inflight:
                retire(block=True)
            elif pending:
                time.sleep(max(0.0, pending[0].arrival - (time.perf_counter() - t0)))
        torch.cuda.synchronize()
        makespan_ms = max((r.done_ms for r in finished_all), default=0.0)
        lat = sorted(r.done_ms - 1e3 * r.arrival for r in finished_all)
        ticks = sorted(a.elapsed_time(b) for a, b in tick_ms)
        units = sum(r.units for r in finished_all)

        def q(xs, p):
            if not xs:
                return None
            return xs[min(len(xs) - 1, max(0, int(math.ceil(p / 100.0 * len(xs))) - 1))]

        return {
            "requests": len(finished_all), "makespan_ms": makespan_ms,
            "requests_per_s": len(finished_all) / (makespan_ms / 1e3) if makespan_ms > 0 else None,
            "ring_gmacs": units / (makespan_ms / 1e3) / 1e9 if makespan_ms > 0 else None,
            "latency_ms_p50": q(lat, 50), "latency_ms_p99": q(lat, 99),
            "tick_ms_p50": q(ticks, 50), "tick_ms_p99": q(ticks, 99), "ticks": len(ticks),
            "peak_resident_bytes": peak_mem, "tag": self.tag,
        }
