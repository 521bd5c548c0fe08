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
    ready request, as ONE grouped share call, ONE grouped opening of D~ on the
    device (this party's R - Z plus the other parties' part, a resident input
    standing in for the network exchange), ONE grouped tag call and ONE
    grouped check call (continuous batching: a request joins at the next tick
    after admission and leaves after its last layer, whatever the others are
    doing);
  * with graphs on, captures a tick as a CUDA graph the second time the same
    tick recurs -- the same requests' arena ranges at the same layers, so
    the same device pointers -- and replays it from then on (a stream of
    same-shaped requests placed at the same offsets, e.g. repeated waves of
    one model and batch size); other ticks are issued eagerly;
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
KEYS_MN = ("C", "mC", "R", "mR", "Drest")     # Drest: the other parties' part of the opening of D


@dataclass
class Request:
    rid: int
    model: str
    batch: int
    arrival: float                 # seconds after the run starts
    seed: int
    layers: list = field(default_factory=list)
    bufs: list = None              # per layer: device addresses (tensors once kept)
    region: tuple = None           # (offset, bytes) in the server's arena
    plan: list = None              # per layer: key -> (shape, byte offset in the region, words)
    nxt: int = 0                   # next layer to run
    ready: object = None           # event: shares materialised
    done_ms: float = None          # device time of completion
    admit_s: float = None
    carve: tuple = None            # (words, _carve(layers, words)), made once per ring width

    @property
    def units(self) -> int:
        """Ring MACs of the request's share products (2MKN per layer)."""
        return sum(2 * L.M * L.K * L.N for L in self.layers)


OUT_MN = ("Z", "mZ", "Dt")
OUT_M = ("mDc", "Dc")


def _carve(layers, words: int):
    """The byte layout of a request's resident tensors, in three sections:
    the pool-filled inputs (256-byte aligned tensors), the keys and combiners
    (alpha, chi, chi^: 16-byte aligned, filled by one generator call) and the
    outputs.  Returns (plan, inputs_end, keys_end, total), plan[layer][key] =
    (shape, byte offset, words)."""
    shp = (lambda *d: d + ((2,) if words == 2 else ()))
    plan = [dict() for _ in layers]

    def put(li, k, shape, off, align):
        n = math.prod(shape)            # words (plain ints: this runs per admitted request)
        plan[li][k] = (shape, off, n)
        return off + (8 * n + align - 1) // align * align

    off = 0
    for li, L in enumerate(layers):
        for k in KEYS_MK:
            off = put(li, k, shp(L.M, L.K), off, 256)
        for k in KEYS_KN:
            off = put(li, k, shp(L.K, L.N), off, 256)
        for k in KEYS_MN:
            off = put(li, k, shp(L.M, L.N), off, 256)
    inputs_end = off
    for li, L in enumerate(layers):
        off = put(li, "alpha", shp(1), off, 16)
        off = put(li, "chi", shp(L.N), off, 16)
        off = put(li, "chi_hat", shp(L.M), off, 16)
    keys_end = off = (off + 255) // 256 * 256
    for li, L in enumerate(layers):
        for k in OUT_MN:
            off = put(li, k, shp(L.M, L.N), off, 256)
        for k in OUT_M:
            off = put(li, k, shp(L.M), off, 256)
        off = put(li, "cs", shp(1), off, 256)
    return plan, inputs_end, keys_end, off


def request_bytes(layers, words: int) -> int:
    """Device bytes a request holds from admission to completion."""
    return _carve(layers, words)[3]


class RangeAllocator:
    """First-fit allocator of byte ranges (256-byte granules) in [0, nbytes).
    Free ranges are kept sorted and coalesced."""

    def __init__(self, nbytes: int):
        self.size = nbytes
        self.free = [(0, nbytes)]
        self.used = 0

    def alloc(self, n: int):
        n = (n + 255) // 256 * 256
        for i, (o, sz) in enumerate(self.free):
            if sz >= n:
                if sz == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (o + n, sz - n)
                self.used += n
                return o
        return None

    def release(self, off: int, n: int):
        n = (n + 255) // 256 * 256
        self.used -= n
        import bisect
        i = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(i, (off, n))
        # coalesce with the neighbours
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (self.free[i][0], self.free[i][1] + self.free[i + 1][1])
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            self.free.pop(i)



class Arena(RangeAllocator):
    """A RangeAllocator over one device buffer, so that admitting and retiring
    requests never calls the CUDA allocator."""

    def __init__(self, torch, nbytes: int):
        super().__init__(nbytes)
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.words = self.buf.view(torch.int64)
        self.base = self.buf.data_ptr()     # device address of byte 0

    def view(self, off: int, shape, n: int = None):
        """int64 tensor of `shape` at byte offset `off` (a multiple of 8)."""
        n = math.prod(shape) if n is None else n
        return self.words[off // 8:off // 8 + n].view(shape)


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

    MAX_GRAPHS = 256              # captured ticks kept (least recently used evicted)

    def __init__(self, ring=synth.Z128, party: int = 0, nparties: int = 2, mem_budget: int = 96 << 30,
                 tag: str = "compact", max_inflight: int = 2, max_group: int = 512, pool_seed: int = 0x5EED,
                 ws_bytes: int = 8 << 30, graphs: bool = False):
        import torch
        if tag not in ("compact", "full"):
            raise ValueError("tag must be 'compact' or 'full'")
        self.torch = torch
        self.ring, self.party, self.nparties = ring, party, nparties
        self.mem_budget, self.tag = mem_budget, tag
        self.max_inflight, self.max_group = max_inflight, max_group
        self.graphs = graphs
        self._graphs = collections.OrderedDict()    # tick key -> (CUDAGraph, event of its last replay)
        self._seen = collections.OrderedDict()      # tick keys issued eagerly once
        self._cap_stream = None
        self.tick_counts = {"eager": 0, "captured": 0, "replayed": 0}
        self._ws_cache = {}
        abi.load()
        # every admitted request's shares live in this arena: its size is the
        # memory budget that gates admission
        self.arena = Arena(torch, mem_budget)
        # one workspace for every tick, allocated up front: a tick whose layers
        # need more runs as several grouped calls in turn
        self.ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        gen = torch.Generator(device="cuda")
        gen.manual_seed(pool_seed)
        self.pool = torch.randint(-(1 << 63), (1 << 63) - 1, (self.POOL_WORDS,), dtype=torch.int64,
                                  device="cuda", generator=gen)

    # -- request shares -------------------------------------------------------
    def _materialise(self, req: Request, stream):
        """Fill the request's arena range on `stream`: the inputs with copies
        of pool windows (chunks of at most the pool's size, at offsets drawn
        from the request's seed, so the same request always gets the same
        shares) and the keys and combiners with one generator call; tensor
        views are made when a layer runs."""
        torch = self.torch
        w = self.ring.words
        base = req.region[0]
        plan, inputs_end, keys_end, _ = req.carve[1]
        rng = np.random.default_rng(req.seed)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(req.seed)
        smax = (1 << min(self.ring.s, 63)) - 1      # keys and combiners: uniform in [0, 2^s)
        with torch.cuda.stream(stream):
            words = self.arena.buf[base:base + inputs_end].view(torch.int64)
            pos = 0
            while pos < words.numel():
                n = min(self.POOL_WORDS, words.numel() - pos)
                o = int(rng.integers(0, self.POOL_WORDS - n + 1))
                words[pos:pos + n].copy_(self.pool[o:o + n], non_blocking=True)
                pos += n
            keys = self.arena.buf[base + inputs_end:base + keys_end].view(torch.int64)
            if w == 2:
                kv = keys.view(-1, 2)
                kv[:, 0].copy_(torch.randint(0, smax, (kv.shape[0],), dtype=torch.int64, device="cuda",
                                             generator=gen))
                kv[:, 1].zero_()
            else:
                keys.copy_(torch.randint(0, smax, (keys.numel(),), dtype=torch.int64, device="cuda", generator=gen))
            ev = torch.cuda.Event()
            ev.record(stream)
        req.plan = plan
        req.bufs = [None] * len(req.layers)
        req.ready = ev

    def _layer_args(self, req: Request, li: int) -> dict:
        """The call arguments of layer li of a request: the device address of
        each of its tensors in the arena (plain ints: the library reads the
        layouts the plan gives them, and a tick builds no tensor objects), the
        mpc_layer and the workspace it needs."""
        d = req.bufs[li]
        if d is None:
            base = self.arena.base + req.region[0]
            d = {k: base + off for k, (_, off, _) in req.plan[li].items()}
            L = req.layers[li]
            d["layer"] = abi.make_layer(L.M, L.K, L.N, self.ring.k, self.ring.s, self.party, self.nparties)
            d["ws_need"] = self._layer_ws(L.M, L.K, L.N)
            req.bufs[li] = d
        return d

    def _views(self, req: Request, li: int) -> dict:
        """Tensor views of layer li of a request (for reading its outputs)."""
        base = req.region[0]
        return {k: self.arena.view(base + off, shape, n) for k, (shape, off, n) in req.plan[li].items()}

    def _layer_ws(self, M, K, N) -> int:
        key = (M, K, N, self.tag)
        need = self._ws_cache.get(key)
        if need is None:
            L = abi.make_layer(M, K, N, self.ring.k, self.ring.s, self.party, self.nparties)
            which = (abi.MPC_WS_SHARE, abi.MPC_WS_TAG_COMPACT if self.tag == "compact" else abi.MPC_WS_TAG_FULL)
            need = self._ws_cache[key] = (max(abi.mpc_workspace_size_grouped([L], w) for w in which)
                                          + 255) // 256 * 256
        return need

    def _parts(self, group):
        """`group` split into parts whose grouped calls fit the workspace; the
        last part may need a workspace of its own (returned size > 0)."""
        parts, part, used = [], [], 0
        for r in group:
            need = self._layer_args(r, r.nxt)["ws_need"]
            if part and used + need > self.ws.numel():
                parts.append(part)
                part, used = [], 0
            part.append(r)
            used += need
        extra = used if (part and used > self.ws.numel()) else 0
        if part:
            parts.append(part)
        return parts, extra

    def _tick_eager(self, parts, extra):
        for i, part in enumerate(parts):
            ws = self.ws
            if extra and i == len(parts) - 1:
                ws = self.torch.empty(extra, dtype=self.torch.uint8, device="cuda")
            self._tick_part(part, ws)

    def _tick(self, group):
        """The next layer of every request in `group`, in as few grouped calls
        as the workspace allows; replayed from a captured graph when this exact
        tick ran before (graphs on)."""
        parts, extra = self._parts(group)
        if not self.graphs or extra:
            self.tick_counts["eager"] += 1
            self._tick_eager(parts, extra)
            return
        torch = self.torch
        key = (tuple((r.region[0], r.model, r.batch, r.nxt) for r in group), self.tag)
        hit = self._graphs.get(key)
        if hit is None and key not in self._seen:
            self._seen[key] = True
            while len(self._seen) > 4 * self.MAX_GRAPHS:
                self._seen.popitem(last=False)
            self.tick_counts["eager"] += 1
            self._tick_eager(parts, extra)
            return
        st = torch.cuda.current_stream()
        if hit is None:
            # second time this tick occurs: capture it (recording only, on a
            # side stream; nothing runs until the replay below)
            if self._cap_stream is None:
                self._cap_stream = torch.cuda.Stream()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(self._cap_stream):
                g.capture_begin(capture_error_mode="thread_local")
                try:
                    self._tick_eager(parts, 0)
                finally:
                    g.capture_end()
            self._seen.pop(key, None)
            self.tick_counts["captured"] += 1
            while len(self._graphs) >= self.MAX_GRAPHS:
                _, (old, ev) = self._graphs.popitem(last=False)
                ev.synchronize()          # not destroyed while a replay may still run
                del old
        else:
            g = hit[0]
            self._graphs.move_to_end(key)
            self.tick_counts["replayed"] += 1
        g.replay()
        ev = torch.cuda.Event()
        ev.record(st)
        self._graphs[key] = (g, ev)

    def _tick_part(self, group, ws):
        a = abi
        bufs = [self._layer_args(r, r.nxt) for r in group]
        layers = [d["layer"] for d in bufs]
        a.mpc_linear_share_grouped(layers, [dict(E=d["E"], F=d["F"], A_i=d["A"], B_i=d["B"], C_i=d["C"],
                                                 Z_i=d["Z"]) for d in bufs], ws=ws)
        if self.tag == "compact":
            # the opening between the share and the tag (Fig. Pi_OptMAC): this
            # party's [D]_i = [R]_i - [Z]_i plus the other parties' part, for
            # every layer of the tick in one call
            k, s = self.ring.k, self.ring.s
            a.mpc_lincomb_grouped(k, s, [1, -1, 1], [[d["R"], d["Z"], d["Drest"]] for d in bufs],
                                  [d["Dt"] for d in bufs], n=[d["layer"].M * d["layer"].N for d in bufs])
        tp = [dict(alpha_i=d["alpha"], E=d["E"], F=d["F"], mA_i=d["mA"], mB_i=d["mB"], mC_i=d["mC"],
                   mR_i=d["mR"], Dtilde=d["Dt"], chi=d["chi"], mZ_i=d["mZ"], mDc_i=d["mDc"], Dc=d["Dc"])
              for d in bufs]
        if self.tag == "compact":
            a.mpc_linear_tag_grouped(layers, a.MPC_TAG_COMPACT, tp, ws=ws)
            a.mpc_tag_check_grouped(layers, [dict(alpha_i=d["alpha"], chi_hat=d["chi_hat"], Dc=d["Dc"],
                                                  mDc_i=d["mDc"], cs_i=d["cs"]) for d in bufs])
        else:
            a.mpc_linear_tag_grouped(layers, a.MPC_TAG_FULL, tp, ws=ws)

    @staticmethod
    def _check_device():
        st = abi.mpc_device_status()
        if st != 0:
            raise RuntimeError(f"serving: {abi.mpc_status_str(st)}; the outputs of the retired ticks are invalid")

    # -- the loop -------------------------------------------------------------
    def run(self, requests, keep_outputs: bool = False, tag: str = None) -> dict:
        """Serve `requests` to completion; `tag` overrides the server's tag path
        for this run."""
        if tag is not None:
            if tag not in ("compact", "full"):
                raise ValueError("tag must be 'compact' or 'full'")
            saved, self.tag = self.tag, tag
            try:
                return self.run(requests, keep_outputs)
            finally:
                self.tag = saved
        torch = self.torch
        self.tick_counts = {"eager": 0, "captured": 0, "replayed": 0}
        st = torch.cuda.current_stream()
        side = torch.cuda.Stream()
        words = self.ring.words
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting = collections.deque()
        active = []
        inflight = collections.deque()      # (event, finished requests)
        tick_ms = []
        peak_mem = 0
        start = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(st)
        t0 = time.perf_counter()
        prev_ev = start
        finished_all = []

        kept = []

        def retire(block: bool):
            retired = False
            while inflight and (block or inflight[0][0].query()):
                ev, fin = inflight.popleft()
                ev.synchronize()
                retired = True
                t = start.elapsed_time(ev)
                for r in fin:
                    r.done_ms = t
                    if keep_outputs:
                        # outputs stay readable: copy them out of the arena before
                        # the range is handed to the next request (whose shares
                        # are written on the side stream)
                        r.bufs = [{k: v.clone() for k, v in self._views(r, li).items()}
                                  for li in range(len(r.layers))]
                        st.synchronize()
                    else:
                        r.bufs = None
                    self.arena.release(*r.region)
                    r.region = None
                    finished_all.append(r)
                block = False
            if retired:
                # the retired ticks have completed: a bounded wait that gave up
                # in one of their kernels has set the library's device flag
                self._check_device()

        while pending or waiting or active or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while waiting:
                if waiting[0].carve is None or waiting[0].carve[0] != words:
                    waiting[0].carve = (words, _carve(waiting[0].layers, words))
                need = waiting[0].carve[1][3]
                off = self.arena.alloc(need)
                if off is None:
                    if not (active or inflight):
                        raise MemoryError(f"request {waiting[0].rid} needs {need} bytes, more than the "
                                          f"{self.mem_budget}-byte budget")
                    break
                r = waiting.popleft()
                r.region = (off, need)
                peak_mem = max(peak_mem, self.arena.used)
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
                self._tick(group)
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
        self._check_device()
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
            "tick_launch": ("CUDA graph replay of recurring ticks, eager otherwise" if self.graphs
                            else "eager grouped calls"),
            "ticks_by_launch": dict(self.tick_counts),
        }
