#!/usr/bin/env python3
"""Benchmark of one party's online SPDZ2k linear layers with CompactTag on GB300.

Workload (default): the two CNN-style linear layers as im2col ring GEMMs in
Z_2^64 (k = s = 32) -- a 3x3 conv on 32x32x64 -> 64 (M, K, N = 1024, 576, 64)
and a 4096 x 4096 dense layer at batch 128 (128, 4096, 4096) -- for two
simulated parties on one GPU.  One step runs, for each layer and each party:
the share (a1), the full SPDZ2k tag (a2, the baseline), the CompactTag tag
(a3-a5) and its check share (a6).  Inputs are uniform ring words (exactly the
distribution of real shares), resident in HBM before the timed region.

Metric: ring-GMAC/s over the step.  Ring multiply-accumulates per layer and
party: 2MKN for the share, 2MKN for the full tag (E.mB + (mA + alpha E).F; the
paper's count is 3MKN + MN), 4MN + 2KN + 3MK + M for the CompactTag tag
(§3.4.3) and M for the check.  Also reported: the tag-overhead ratio
t(CompactTag) / t(full tag) per layer and summed, p50/p99 step latency, the
roofline fraction of the dominant kernel and the oracle on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from paper_2311_04406_gb300 import costmodel  # noqa: E402

METRIC = "ring-GMAC/s and tag-overhead ratio (CompactTag vs full tag), bit-exact; p99"
PARTIES = 2
RING = synth.Z64          # set from --ring in main()
SEED = 0xC0FFEE01

WORKLOADS = {
    "cnn": ("cnn_im2col_conv3x3_32x32x64_and_dense4096_b128", lambda b: synth.cnn_pair()),
    "single": ("dense_64x128x64", lambda b: [synth.single_dense()]),
    "vgg16": ("vgg16_32x32x3_b{b}", lambda b: synth.vgg16_layers(b)),
    "resnet18": ("resnet18_32x32x3_b{b}", lambda b: synth.resnet18_layers(b)),
    "transformer": ("transformer_h1024_t2048", lambda b: synth.transformer_layers()),
    "transformer_block": ("transformer_block_h1024_a16_t2048", lambda b: synth.transformer_block()),
    "uneven": ("uneven256_seeded", lambda b: synth.uneven_layers(256)),
    "serve": ("serve_resnet18_vgg16_b1-32_z128_poisson", None),
    "layer": ("layer_{b}", None),          # one layer of the --shape given
}
L2_BYTES = 129 * 2**20


PROTOCOL = "plain"        # set from --protocol in main()
TRUNC_F = 16
PASS = "forward"          # set from --pass in main(); "train" adds the backward layers


def layer_units(L) -> dict:
    M, K, N = L.M, L.K, L.N
    u = dict(share=2 * M * K * N, full=2 * M * K * N,
             compact=costmodel.compact_tag_mults(M, K, N), check=M)
    if PROTOCOL == "trunc":
        u["public"] = M * K * N          # E.F, computed by every party
        u["optmac_trunc"] = M * N
    return u


def step_units(layers) -> int:
    return PARTIES * sum(sum(layer_units(L).values()) for L in layers)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get(
            "bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


# ---------------------------------------------------------------------------
# distributed plumbing (replicas: every rank runs the same workload)

def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("MPC_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return rank, ws


def job_throughput(units_per_step: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job ring-GMAC/s: every rank runs the same workload (replicas, weak
    scaling), so the job processes world x units per step; the time is the
    slowest rank's."""
    return world * units_per_step * steps / (max_ms / 1e3) / 1e9


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the GPU arm

def _uniform(seed, name, party, shape, bits):
    return synth.uniform(seed, synth.TID[name], party, shape, bits)


def _key(seed, name, party, shape):
    """Public coins and key shares: uniform in [0, 2^s), stored in ring words."""
    v = synth.uniform(seed, synth.TID[name], party, shape, RING.s)
    if RING.words == 1:
        return v
    out = np.zeros(tuple(shape) + (2,), dtype=np.uint64)
    out[..., 0] = v
    return out


def ring_shape(*dims):
    return tuple(dims) + ((2,) if RING.words == 2 else ())


_HOST_CACHE = {}


def host_inputs(layers, seed=SEED):
    """Uniform inputs per layer: public E, F, D~, chi, chi^ and per-party shares
    (generated once per layer list and seed)."""
    key = (tuple((L.name, L.M, L.K, L.N) for L in layers), seed, PROTOCOL, RING)
    if key not in _HOST_CACHE:
        _HOST_CACHE.clear()
        _HOST_CACHE[key] = _host_inputs(layers, seed)
    return _HOST_CACHE[key]


def _host_inputs(layers, seed):
    out = []
    b = RING.bits
    for li, L in enumerate(layers):
        M, K, N = L.M, L.K, L.N
        sd = seed + 1000 * li
        pub = dict(E=_uniform(sd, "E", 0, (M, K), b), F=_uniform(sd, "F", 0, (K, N), b),
                   Dt=_uniform(sd, "Dt", 0, (M, N), b), chi=_key(sd, "chi", 0, (N,)),
                   chi_hat=_key(sd, "chi_hat", 0, (M,)))
        parties = []
        for p in range(PARTIES):
            parties.append(dict(
                alpha=_key(sd, "alpha", p, (1,)),
                A=_uniform(sd, "A", p + 1, (M, K), b), B=_uniform(sd, "B", p + 1, (K, N), b),
                C=_uniform(sd, "C", p + 1, (M, N), b), mA=_uniform(sd, "mA", p + 1, (M, K), b),
                mB=_uniform(sd, "mB", p + 1, (K, N), b), mC=_uniform(sd, "mC", p + 1, (M, N), b),
                mR=_uniform(sd, "mR", p + 1, (M, N), b)))
            if PROTOCOL == "trunc":
                parties[-1].update(Rf=_uniform(sd, "Rf", p + 1, (M, N), b),
                                   mRf=_uniform(sd, "mRf", p + 1, (M, N), b))
        out.append((L, pub, parties))
    return out


def device_inputs(layers, torch, seed=SEED):
    """The same structure as host_inputs, generated on the device: uniform
    64-bit words (torch's seeded generator) and keys and combiners uniform in
    [0, 2^s).  For timing-only records of workloads too large to generate on
    the host quickly; the values are not those of host_inputs."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    smax = 1 << min(RING.s, 63)

    def words(*dims):
        return torch.randint(-(1 << 63), (1 << 63) - 1, ring_shape(*dims), dtype=torch.int64, device="cuda",
                             generator=g)

    def key(*dims):
        v = torch.zeros(ring_shape(*dims), dtype=torch.int64, device="cuda")
        lo = torch.randint(0, smax, dims, dtype=torch.int64, device="cuda", generator=g)
        if RING.words == 1:
            v.copy_(lo)
        else:
            v[..., 0] = lo
        return v

    out = []
    for L in layers:
        M, K, N = L.M, L.K, L.N
        pub = dict(E=words(M, K), F=words(K, N), Dt=words(M, N), chi=key(N), chi_hat=key(M))
        parties = [dict(alpha=key(1), A=words(M, K), B=words(K, N), C=words(M, N), mA=words(M, K),
                        mB=words(K, N), mC=words(M, N), mR=words(M, N)) for _ in range(PARTIES)]
        out.append((L, pub, parties))
    return out


class GpuWorkload:
    def __init__(self, layers, torch, abi, pinned_host=False, device_gen=False):
        self.torch, self.abi = torch, abi
        self.layers = layers
        self.stream = torch.cuda.current_stream()
        if device_gen and pinned_host:
            raise ValueError("device-generated inputs have no host copy")
        hi = device_inputs(layers, torch) if device_gen else host_inputs(layers)
        t = (lambda a: a) if device_gen else (lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)))
        self.items = []
        self.h2d_pairs = []   # (host pinned, device) for the e2e copy
        self.h2d_by = {}      # (layer, party or "pub") -> its pairs, for the pipelined e2e step
        # backward layers: operands that are transposes of forward operands
        # (index of the forward layer, public key, share key, tag key, forward dims)
        names = {L.name: i for i, L in enumerate(layers)}
        self.links = {}
        for i, L in enumerate(layers):
            for suf, keys in (("_dX", ("F", "B", "mB")), ("_dW", ("E", "A", "mA"))):
                if L.name.endswith(suf) and L.name[:-3] in names:
                    j = names[L.name[:-3]]
                    Lf = layers[j]
                    dims = (Lf.K, Lf.N) if suf == "_dX" else (Lf.M, Lf.K)
                    self.links[i] = (j,) + keys + (dims,)
        for li, (L, pub, parties) in enumerate(hi):
            derived = set(self.links[li][1:4]) if li in self.links else set()
            M, K, N = L.M, L.K, L.N
            dpub = {k: t(v).cuda() for k, v in pub.items()}
            if device_gen:
                pub.clear()
            dpar = []
            for p, sh in enumerate(parties):
                lay = abi.make_layer(M, K, N, RING.k, RING.s, p, PARTIES)
                d = {k: t(v).cuda() for k, v in sh.items()}
                if device_gen:
                    sh.clear()
                d["Z"] = torch.empty(ring_shape(M, N), dtype=torch.int64, device="cuda")
                d["mZfull"] = torch.empty(ring_shape(M, N), dtype=torch.int64, device="cuda")
                d["mZ"] = torch.empty(ring_shape(M, N), dtype=torch.int64, device="cuda")
                d["mDc"] = torch.empty(ring_shape(M), dtype=torch.int64, device="cuda")
                d["Dc"] = torch.empty(ring_shape(M), dtype=torch.int64, device="cuda")
                d["cs"] = torch.empty(ring_shape(1), dtype=torch.int64, device="cuda")
                if PROTOCOL == "trunc":
                    d["P"] = torch.empty(ring_shape(M, N), dtype=torch.int64, device="cuda")
                    d["Zf"] = torch.empty(ring_shape(M, N), dtype=torch.int64, device="cuda")
                    d["mZf_t"] = torch.empty(ring_shape(M, N), dtype=torch.int64, device="cuda")
                d["layer"] = lay
                nws = max(abi.mpc_workspace_size(lay, w) for w in range(5))
                d["ws"] = torch.empty(max(nws, 256), dtype=torch.uint8, device="cuda")
                dpar.append(d)
                if pinned_host:
                    for k, v in sh.items():
                        if k not in derived:
                            self.h2d_by.setdefault((li, p), []).append((t(v).pin_memory(), d[k]))
            if pinned_host:
                for k, v in pub.items():
                    if k not in derived:
                        self.h2d_by.setdefault((li, "pub"), []).append((t(v).pin_memory(), dpub[k]))
                for key in [(li, "pub")] + [(li, p) for p in range(len(parties))]:
                    self.h2d_pairs += self.h2d_by.get(key, [])
            self.items.append((L, dpub, dpar))
        out_keys = ("Z", "mZfull", "mZ", "mDc", "Dc", "cs") if PROTOCOL == "plain" else \
            ("Z", "mZfull", "Zf", "mZf_t", "mDc", "Dc", "cs")
        self.outputs = [d[k] for _, _, dpar in self.items for d in dpar for k in out_keys]
        self.h_outputs = [o.cpu().pin_memory() for o in self.outputs] if pinned_host else []
        nk = len(out_keys)
        self.d2h_by = {}
        if pinned_host:
            j = 0
            for li, (_, _, dpar) in enumerate(self.items):
                for p in range(len(dpar)):
                    self.d2h_by[(li, p)] = list(zip(self.h_outputs[j:j + nk], self.outputs[j:j + nk]))
                    j += nk

    def _transpose(self, src, dst, rows, cols):
        self.abi.mpc_transpose(RING.k, RING.s, rows, cols, src, dst)

    def _pre(self, i, p, tag):
        """A backward layer's party first transposes, locally, the forward
        operands it reuses: the public opening and its mask share before the
        share GEMM, its tag share before a tag."""
        if i not in self.links:
            return
        j, kpub, ksh, ktag, (rows, cols) = self.links[i]
        _, fpub, fpar = self.items[j]
        _, pub, par = self.items[i]
        if tag:
            self._transpose(fpar[p][ktag], par[p][ktag], rows, cols)
        else:
            self._transpose(fpub[kpub], pub[kpub], rows, cols)
            self._transpose(fpar[p][ksh], par[p][ksh], rows, cols)

    # one call of each kind
    def share(self, i, p):
        L, pub, par = self.items[i]
        d = par[p]
        self._pre(i, p, tag=False)
        if PROTOCOL == "trunc":
            # share without E.F, and the public E.F that both protocols add after truncation
            self.abi.mpc_linear_share_trunc(d["layer"], pub["E"], pub["F"], d["A"], d["B"], d["C"], d["Z"],
                                            ws=d["ws"])
            self.abi.mpc_public_product(d["layer"], pub["E"], pub["F"], d["P"], ws=d["ws"])
        else:
            self.abi.mpc_linear_share(d["layer"], pub["E"], pub["F"], d["A"], d["B"], d["C"], d["Z"],
                                      ws=d["ws"])

    def full(self, i, p):
        L, pub, par = self.items[i]
        d = par[p]
        self._pre(i, p, tag=True)
        self.abi.mpc_linear_tag(d["layer"], self.abi.MPC_TAG_FULL, d["alpha"], pub["E"], pub["F"],
                                d["mA"], d["mB"], d["mC"], d["mZfull"], ws=d["ws"])

    def compact(self, i, p):
        L, pub, par = self.items[i]
        d = par[p]
        self._pre(i, p, tag=True)
        if PROTOCOL == "trunc":
            # OptMAC&Trunc (share and tag), compact tag without the E.U term
            self.abi.mpc_optmac_trunc(d["layer"], TRUNC_F, d["alpha"], d["Rf"], d["mRf"], pub["Dt"], d["P"],
                                      d["Zf"], d["mZf_t"])
            self.abi.mpc_linear_tag(d["layer"], self.abi.MPC_TAG_COMPACT_TRUNC, d["alpha"], pub["E"],
                                    pub["F"], d["mA"], d["mB"], d["mC"], None, mR_i=d["mR"],
                                    Dtilde=pub["Dt"], chi=pub["chi"], mDc_i=d["mDc"], Dc=d["Dc"],
                                    ws=d["ws"])
        else:
            self.abi.mpc_linear_tag(d["layer"], self.abi.MPC_TAG_COMPACT, d["alpha"], pub["E"], pub["F"],
                                    d["mA"], d["mB"], d["mC"], d["mZ"], mR_i=d["mR"], Dtilde=pub["Dt"],
                                    chi=pub["chi"], mDc_i=d["mDc"], Dc=d["Dc"], ws=d["ws"])
        self.abi.mpc_tag_check(d["layer"], self.abi.MPC_CHECK_COMPACT, d["alpha"], pub["chi_hat"],
                               d["Dc"], d["mDc"], d["cs"], ws=d["ws"])

    def step(self):
        for i in range(len(self.items)):
            for p in range(PARTIES):
                self.share(i, p)
                self.full(i, p)
                self.compact(i, p)

    # grouped calls: every layer of one party in one call of each kind
    def setup_grouped(self):
        a, torch = self.abi, self.torch
        self.glayers, self.gshare, self.gtag_full, self.gtag_comp, self.gws = [], [], [], [], []
        self.gcheck = []
        for p in range(PARTIES):
            lays = [par[p]["layer"] for _, _, par in self.items]
            sh, tf, tc, ck = [], [], [], []
            for _, pub, par in self.items:
                d = par[p]
                ck.append(dict(alpha_i=d["alpha"], chi_hat=pub["chi_hat"], Dc=d["Dc"], mDc_i=d["mDc"], cs_i=d["cs"]))
                sh.append(dict(E=pub["E"], F=pub["F"], A_i=d["A"], B_i=d["B"], C_i=d["C"], Z_i=d["Z"]))
                base = dict(alpha_i=d["alpha"], E=pub["E"], F=pub["F"], mA_i=d["mA"], mB_i=d["mB"], mC_i=d["mC"],
                            mR_i=d["mR"], Dtilde=pub["Dt"], chi=pub["chi"], mDc_i=d["mDc"], Dc=d["Dc"])
                tf.append(dict(base, mZ_i=d["mZfull"]))
                tc.append(dict(base, mZ_i=d["mZ"]))
            need = max(a.mpc_workspace_size_grouped(lays, w)
                       for w in (a.MPC_WS_SHARE, a.MPC_WS_TAG_FULL, a.MPC_WS_TAG_COMPACT))
            self.glayers.append(lays)
            self.gshare.append(sh)
            self.gtag_full.append(tf)
            self.gtag_comp.append(tc)
            self.gcheck.append(ck)
            self.gws.append(torch.empty(max(need, 256), dtype=torch.uint8, device="cuda"))

    def share_group(self, p):
        for i in self.links:
            self._pre(i, p, tag=False)
        self.abi.mpc_linear_share_grouped(self.glayers[p], self.gshare[p], ws=self.gws[p])

    def full_group(self, p):
        for i in self.links:
            self._pre(i, p, tag=True)
        self.abi.mpc_linear_tag_grouped(self.glayers[p], self.abi.MPC_TAG_FULL, self.gtag_full[p], ws=self.gws[p])

    def compact_group(self, p):
        for i in self.links:
            self._pre(i, p, tag=True)
        self.abi.mpc_linear_tag_grouped(self.glayers[p], self.abi.MPC_TAG_COMPACT, self.gtag_comp[p],
                                        ws=self.gws[p])
        # every layer's check share in one launch per 64 layers
        self.abi.mpc_tag_check_grouped(self.glayers[p], self.gcheck[p])

    def step_grouped(self):
        for p in range(PARTIES):
            self.share_group(p)
            self.full_group(p)
            self.compact_group(p)

    def launches_per_step_grouped(self):
        a = self.abi
        n = 0
        for p in range(PARTIES):
            lays = self.glayers[p]
            n += sum(a.mpc_launch_count_grouped(lays, w)
                     for w in (a.MPC_WS_SHARE, a.MPC_WS_TAG_FULL, a.MPC_WS_TAG_COMPACT))
            n += (len(lays) + 63) // 64 + 3 * len(self.links)   # grouped checks; transposes
        return n

    def launches_per_step(self):
        """Kernels one step enqueues, as the library reports them."""
        a = self.abi
        which = (a.MPC_WS_SHARE, a.MPC_WS_TAG_FULL, a.MPC_WS_TAG_COMPACT, a.MPC_WS_CHECK_COMPACT)
        if PROTOCOL == "trunc":
            which = (a.MPC_WS_SHARE_TRUNC, a.MPC_WS_TAG_FULL, a.MPC_WS_PUBLIC_PRODUCT,
                     a.MPC_WS_OPTMAC_TRUNC, a.MPC_WS_TAG_COMPACT, a.MPC_WS_CHECK_COMPACT)
        n = 0
        for i, (L, _, par) in enumerate(self.items):
            for d in par:
                n += sum(a.mpc_launch_count(d["layer"], w) for w in which)
                if i in self.links:
                    n += 4   # two transposes before the share, one before each tag
        return n

    COPY_STREAMS = 4

    def _copy_streams(self):
        if not hasattr(self, "_cs"):
            self._cs = [self.torch.cuda.Stream() for _ in range(self.COPY_STREAMS)]
        return self._cs

    def _spread(self, pairs, fn):
        """Issue the copies round-robin on several streams (several copy
        engines), each ordered after the work already on the compute stream,
        and make the compute stream wait for all of them."""
        torch = self.torch
        st = torch.cuda.current_stream()
        cs = self._copy_streams()
        # largest copies first, dealt so that the streams carry similar bytes
        order = sorted(range(len(pairs)), key=lambda i: -pairs[i][0].numel())
        load = [0] * len(cs)
        for c in cs:
            c.wait_stream(st)
        for i in order:
            j = min(range(len(cs)), key=lambda k: load[k])
            load[j] += pairs[i][0].numel()
            with torch.cuda.stream(cs[j]):
                fn(*pairs[i])
        for c in cs:
            st.wait_stream(c)

    def e2e_step(self):
        """One step with its host copies pipelined: the inputs are copied in
        the order the step consumes them (layer by layer, party by party) on a
        copy stream, each call waits only for its own inputs, and each party's
        outputs are copied back on a second stream as soon as they exist.  A
        layer's inputs for the next step are copied as soon as this step's
        calls on that layer are done (not after the whole step), so the copies
        of one step overlap the calls of the one before.  Workloads whose
        layers read other layers' operands (training) wait for the whole
        previous step instead."""
        torch = self.torch
        st = torch.cuda.current_stream()
        if not hasattr(self, "_h2d_stream"):
            self._h2d_stream, self._d2h_stream = torch.cuda.Stream(), torch.cuda.Stream()
        cs, ds = self._h2d_stream, self._d2h_stream
        prev = getattr(self, "_consumed", None)
        cross = prev is not None and not self.links
        if not cross:
            cs.wait_stream(st)    # the previous step is done with the buffers
        ready = {}
        for i in range(len(self.items)):
            with torch.cuda.stream(cs):
                if cross:
                    for p in range(PARTIES):
                        cs.wait_event(prev[(i, p)])   # the previous step's calls on layer i are done
                for h, d in self.h2d_by.get((i, "pub"), []):
                    d.copy_(h, non_blocking=True)
                for p in range(PARTIES):
                    for h, d in self.h2d_by.get((i, p), []):
                        d.copy_(h, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(cs)
                    ready[(i, p)] = ev
        ds.wait_stream(st)
        consumed = {}
        for i in range(len(self.items)):
            for p in range(PARTIES):
                st.wait_event(ready[(i, p)])
                self.share(i, p)
                self.full(i, p)
                self.compact(i, p)
                done = torch.cuda.Event()
                done.record(st)
                consumed[(i, p)] = done
                ds.wait_event(done)
                with torch.cuda.stream(ds):
                    for h, d in self.d2h_by[(i, p)]:
                        h.copy_(d, non_blocking=True)
        # the next step's calls overwrite the outputs only after they are read back
        st.wait_stream(ds)
        self._consumed = consumed

    def h2d(self):
        self._spread(self.h2d_pairs, lambda h, d: d.copy_(h, non_blocking=True))

    def d2h(self):
        self._spread(list(zip(self.h_outputs, self.outputs)), lambda h, d: h.copy_(d, non_blocking=True))

    def h2d_bytes(self):
        return sum(h.numel() * 8 for h, _ in self.h2d_pairs)

    def d2h_bytes(self):
        return sum(h.numel() * 8 for h in self.h_outputs)


def time_calls(torch, fn, reps, graph=True, budget_s=None):
    """Per-call device durations (ms) with CUDA events on the launching stream;
    with graph=True the call is captured once and its graph replayed, so host
    launch overhead is not counted.  With budget_s, `reps` is a maximum: the
    count is cut so that the timed calls take about budget_s (at least 20)."""
    st = torch.cuda.current_stream()
    call = fn
    if graph:
        cap = torch.cuda.Stream()
        cap.wait_stream(st)
        with torch.cuda.stream(cap):
            fn()
        st.wait_stream(cap)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            fn()
        torch.cuda.synchronize()
        call = g.replay
        call()
    if budget_s is not None:
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(st)
        for _ in range(3):
            call()
        a1.record(st)
        torch.cuda.synchronize()
        per = max(a0.elapsed_time(a1) / 3e3, 1e-6)
        reps = int(min(reps, max(20, budget_s / per)))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    for a, b in evs:
        a.record(st)
        call()
        b.record(st)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    i = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[i]


def profile_traffic(kernel_tag: str):
    """Per-launch DRAM bytes of `kernel_tag` from the committed ncu summary,
    when it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(kernel_tag)
        if not rec:
            return None
        import hashlib
        src = os.path.join(ROOT, "paper_2311_04406_gb300", "csrc", rec["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != rec["source_sha"]:
            return None
        return rec["bytes_per_launch"]
    except Exception:
        return None


def capture(torch, fn):
    """One call of fn captured into a CUDA graph (after one eager run on the
    capture stream); returns the graph."""
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        fn()
    torch.cuda.current_stream().wait_stream(cap)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap):
        fn()
    torch.cuda.synchronize()
    return g


def timed_steps(torch, fn, steps):
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


PER_LAYER_TABLE_MAX = 24      # larger layer sets report per-group call timings


def run_ours(args):
    import torch
    from paper_2311_04406_gb300 import abi, build
    rank, ws = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    abi.load()
    layers, workload = workload_layers(args)
    tune = None
    if args.autotune:
        t0 = time.perf_counter()
        shapes = [abi.make_layer(L.M, L.K, L.N, RING.k, RING.s) for L in layers]
        n_tuned = abi.mpc_autotune(shapes)
        torch.cuda.synchronize()
        tc_after = sum(1 for L in shapes if abi.mpc_gemm_path(L) == 1)
        tune = {"shapes": n_tuned, "seconds": time.perf_counter() - t0, "tensor_core_layers": tc_after,
                "choices (path, tile rows, swizzle, K split)": sorted(
                    {(c[0], c[4], c[1], c[2]) for c in (abi.mpc_autotune_choice(L) for L in shapes)})}
    run = GpuWorkload(layers, torch, abi, pinned_host=not args.no_e2e)
    units = step_units(layers)
    if args.grouped:
        run.setup_grouped()
    step_eager = run.step_grouped if args.grouped else run.step

    # warm-up (eager), then capture one step into a CUDA graph
    for _ in range(args.warmup):
        step_eager()
    torch.cuda.synchronize()
    graph = None
    if not args.eager:
        graph = capture(torch, step_eager)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
    step_fn = graph.replay if graph is not None else step_eager

    # timed region: K steps, per-step events, barrier + sync on both sides
    barrier(ws)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with Clocks(local) as ck:
        ev[0].record(st)
        for k in range(args.steps):
            step_fn()
            ev[k + 1].record(st)
        torch.cuda.synchronize()
    barrier(ws)
    check_device(abi, "the timed steps")
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms = max_over_ranks(total_ms, ws)
    ms_per_step = total_ms / args.steps
    value = job_throughput(units, args.steps, ws, total_ms)
    # the same steps issued eagerly through the API (host launch overhead included)
    eager_ms = timed_steps(torch, step_eager, args.steps) if graph is not None else None
    # grouped runs: the same step as one call per layer, for comparison
    per_layer_calls_ms = None
    if args.grouped and not args.eager:
        g2 = capture(torch, run.step)
        g2.replay()
        per_layer_calls_ms = timed_steps(torch, g2.replay, args.steps)
        del g2

    reps = 200                    # at most; each call kind gets about 2 s
    graphs = not args.eager
    hbm, bf16, bf16s, src = peaks()
    digit = costmodel.digit_products(RING.bits)
    per_layer, per_group = [], None
    if args.grouped or len(layers) > PER_LAYER_TABLE_MAX:
        # per-call timings of one party's grouped calls (the group runs as one
        # call of each kind in the grouped step, as one call per layer otherwise)
        if not args.grouped:
            run.setup_grouped()
        sh = time_calls(torch, lambda: run.share_group(1), reps, graphs, budget_s=2.0)
        fu = time_calls(torch, lambda: run.full_group(1), reps, graphs, budget_s=2.0)
        co = time_calls(torch, lambda: run.compact_group(1), reps, graphs, budget_s=2.0)
        per_group = dict(layers=len(layers), timed_calls=len(sh), share_ms_p50=pct(sh, 50),
                         full_tag_ms_p50=pct(fu, 50),
                         compact_tag_ms_p50=pct(co, 50), compact_tag_ms_p99=pct(co, 99),
                         full_tag_ms_p99=pct(fu, 99))
        sum_co, sum_fu = pct(co, 50), pct(fu, 50)
        tc_layers = [L for L in layers if abi_path_is_tc(abi, L)]
        tc_macs = sum(2 * L.M * L.K * L.N for L in tc_layers)
        all_macs = sum(2 * L.M * L.K * L.N for L in layers)
        gemm_calls = sh + fu
        avg_ms = sum(gemm_calls) / len(gemm_calls)
        achieved = tc_macs * digit * 2 / (avg_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": bf16, "unit": "TFLOP/s",
                "frac": achieved / bf16, "kernel": "ring_gemm_tc (grouped persistent launches)",
                "launch": f"grouped share and full-tag calls of all {len(layers)} layers of one party "
                          f"({len(tc_layers)} on the tensor cores), {len(gemm_calls)} calls, CUDA events"
                          + (" around graph replays of the call" if graphs else "")
                          + "; the call time includes the integer-pipe layers' kernels",
                "ring_gmacs": all_macs / (avg_ms / 1e3) / 1e9,
                "per_unit": f"2MKN ring MACs of the tensor-core layers x {digit} fp16 digit products x 2 flop",
                "peak_source": f"{src} bf16 dense burst (fp16 has the same nominal rate), x1.0",
                "traffic": None}
        co_ms = pct(co, 50)
        co_bytes = sum(8 * RING.words * (4 * L.M * L.N + 2 * L.K * L.N + 2 * L.M * L.K) for L in layers)
        hbm_kernel = "CompactTag grouped tag call + per-layer checks, all layers of one party"
    else:
        gemm_ms_by_layer = []
        for i, L in enumerate(layers):
            sh = time_calls(torch, lambda: run.share(i, 1), reps, graphs, budget_s=1.0)
            fu = time_calls(torch, lambda: run.full(i, 1), reps, graphs, budget_s=1.0)
            co = time_calls(torch, lambda: run.compact(i, 1), reps, graphs, budget_s=1.0)
            per_layer.append(dict(layer=L.name, M=L.M, K=L.K, N=L.N,
                                  share_ms_p50=pct(sh, 50), full_tag_ms_p50=pct(fu, 50),
                                  compact_tag_ms_p50=pct(co, 50), compact_tag_ms_p99=pct(co, 99),
                                  full_tag_ms_p99=pct(fu, 99),
                                  tag_overhead_ratio=pct(co, 50) / pct(fu, 50),
                                  full_tag_over_share=pct(fu, 50) / pct(sh, 50),
                                  compact_tag_over_share=pct(co, 50) / pct(sh, 50),
                                  timed_calls=len(sh),
                                  share_ring_gmacs=2 * L.M * L.K * L.N / (pct(sh, 50) / 1e3) / 1e9,
                                  cost_model_tag_ratio=costmodel.tag_mult_ratio(L.M, L.K, L.N)))
            gemm_ms_by_layer.append(sh + fu)
        sum_co = sum(x["compact_tag_ms_p50"] for x in per_layer)
        sum_fu = sum(x["full_tag_ms_p50"] for x in per_layer)
        # dominant kernel: the ring GEMM of the largest layer (share and full-tag calls)
        big = max(range(len(layers)), key=lambda i: layers[i].M * layers[i].K * layers[i].N)
        Lb = layers[big]
        gemm_calls = gemm_ms_by_layer[big]
        avg_ms = sum(gemm_calls) / len(gemm_calls)
        ring_macs = 2 * Lb.M * Lb.K * Lb.N
        if abi_path_is_tc(abi, Lb):
            achieved = ring_macs * digit * 2 / (avg_ms / 1e3) / 1e12
            roof = {"bound": "tensor", "achieved": achieved, "peak": bf16, "unit": "TFLOP/s",
                    "frac": achieved / bf16, "kernel": "ring_gemm_tc",
                    "launch": f"share and full-tag calls of layer {Lb.M}x{Lb.K}x{Lb.N} "
                              f"(prologue + GEMM), {len(gemm_calls)} calls, CUDA events"
                              + (" around graph replays of the call" if graphs else ""),
                    "ring_gmacs": ring_macs / (avg_ms / 1e3) / 1e9,
                    "per_unit": f"2MKN ring MACs per call x {digit} fp16 digit products x 2 flop",
                    "peak_source": f"{src} bf16 dense burst (fp16 has the same nominal rate), x1.0",
                    "traffic": profile_traffic("ring_gemm_tc")}
        else:
            peak_gops = 152 * 64 * 2.07
            achieved = ring_macs * 3 / (avg_ms / 1e3) / 1e9
            roof = {"bound": "alu", "achieved": achieved, "peak": peak_gops, "unit": "Gop/s",
                    "frac": achieved / peak_gops, "kernel": "ring_gemm_simt",
                    "per_unit": "3 IMAD-class ops per 64-bit ring MAC",
                    "peak_source": "derived: 152 SMs x 64 int32 multiply-add/clk x 2070 MHz",
                    "traffic": profile_traffic("ring_gemm_simt")}
        co_ms = per_layer[big]["compact_tag_ms_p50"]
        co_bytes = 8 * RING.words * (4 * Lb.M * Lb.N + 2 * Lb.K * Lb.N + 2 * Lb.M * Lb.K)
        hbm_kernel = "CompactTag tag call (rows + finalize + vec + check kernels)"
    hbm_roof = {"bound": "hbm", "achieved": co_bytes / (co_ms / 1e3) / 1e9, "peak": hbm,
                "unit": "GB/s", "frac": co_bytes / (co_ms / 1e3) / 1e9 / hbm,
                "kernel": hbm_kernel,
                "per_unit": "8 w (4MN + 2KN + 2MK) bytes per call", "peak_source": f"{src} hbm_gbs",
                "traffic": profile_traffic("rows_kernel") if per_group is None else None}

    launches = run.launches_per_step_grouped() if args.grouped else run.launches_per_step()

    # end-to-end: the same step through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e_steps = max(3, args.steps // 2)
        pipelined = not args.grouped
        # two sets of device buffers taken in turn, so that one step's input
        # copies also overlap the last layers of the step before (same inputs,
        # same work per step)
        runs = [run, GpuWorkload(layers, torch, abi, pinned_host=True)] if pipelined and not run.links else [run]
        run.h2d(); step_eager(); run.d2h()
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        for s_ in range(e2e_steps):
            if pipelined:
                runs[s_ % len(runs)].e2e_step()
            else:
                run.h2d()
                step_eager()
                run.d2h()
        b.record(st)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        check_device(abi, "the end-to-end steps")
        e2e_ms = max_over_ranks(max(a.elapsed_time(b), wall * 1e3), ws) / e2e_steps
        e2e = {"value": ws * units / (e2e_ms / 1e3) / 1e9, "unit": "ring-GMAC/s",
               "ms_per_step": e2e_ms, "h2d_bytes_per_step": run.h2d_bytes(),
               "d2h_bytes_per_step": run.d2h_bytes(), "host_buffers": "pinned",
               "copies": "pipelined with the calls (inputs layer by layer and party by party on a copy "
                         "stream, a layer's next inputs as soon as its calls are done, two device buffer "
                         "sets taken in turn, outputs back as produced)" if pipelined else
                         "all inputs, then the step, then all outputs"}

    # the other configurations' records, on one GPU only
    extras = {}
    if ws == 1 and args.workload == "cnn" and PROTOCOL == "plain" and PASS == "forward" and not args.no_extras:
        # drop every reference to the main workload's buffers (bound methods and
        # the captured graph hold the workload too)
        run = runs = step_eager = step_fn = graph = None
        import gc
        gc.collect()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        extras["grouped_uneven"] = extra_grouped_uneven(torch, abi, args.warmup)
        extras["vgg16_grouped"] = extra_vgg16(torch, abi, args.warmup)
        extras["serving"] = extra_serving(torch, abi)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(layers, budget_s=args.cpu_seconds)
    dtype = "u64" if RING.words == 1 else "u128 (two u64 words)"

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "ring-GMAC/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "p50_ms_per_step": pct(step_ms, 50), "p99_ms_per_step": pct(step_ms, 99),
            "step_launch": "CUDA graph replay of one captured step" if graph is not None else "eager API calls",
            "ms_per_step_eager_api": eager_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (uniform ring words from seeded SplitMix64; shapes of the paper's layers)",
            "config": make_config(workload, layers, ws),
            "tag_overhead_ratio": sum_co / sum_fu,
            "per_layer": per_layer,
            "per_group_call": per_group,
            "grouped": bool(args.grouped),
            "autotune": tune,
            "ms_per_step_per_layer_calls": per_layer_calls_ms,
            "roofline": roof,
            "compact_hbm_roofline": hbm_roof,
            "gpu_launches": launches * args.steps,
            "clocks": ck.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "device_status": "ok",
        }
        line.update(extras)
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def make_config(workload, layers, ws) -> dict:
    """The workload description both arms print (the same keys and values)."""
    return {"workload": workload + ("" if PROTOCOL == "plain" else f"_truncated_f{TRUNC_F}"),
            "protocol": "CompactTag with OptMAC&Trunc (truncated layer)" if PROTOCOL == "trunc"
            else "CompactTag (untruncated layer) beside the SPDZ2k full tag",
            "layers": [[L.M, L.K, L.N] for L in layers],
            "pass": "forward" if PASS == "forward" else
            "training: forward + grad X (M,N,K) + grad W (K,M,N) per layer, with device transposes",
            "ring": f"Z_2^{RING.bits} (k={RING.k}, s={RING.s})",
            "parties": PARTIES, "parallelism": f"replicas x{ws}",
            "l2": (f"inputs larger than L2 ({run_bytes(layers) / 2**20:.0f} MiB per step > 129 MiB)"
                   if run_bytes(layers) > L2_BYTES else
                   f"inputs smaller than L2 ({run_bytes(layers) / 2**20:.1f} MiB per step): steps hit in L2")}


def check_device(abi, where: str):
    """A kernel whose bounded wait gave up returned early with wrong outputs
    and set the library's device flag: such a run reports nothing."""
    st = abi.mpc_device_status()
    if st != 0:
        raise SystemExit(f"bench: {abi.mpc_status_str(st)} during {where}; the results are invalid")


# ---------------------------------------------------------------------------
# records of the other configurations in the default run (one GPU)

EXTRA_STEPS = 10


def extra_grouped_uneven(torch, abi, warmup):
    """256 uneven layers (M in [1, 4096] log-uniform, K and N in {64 .. 4096}),
    Z_2^64, two parties: the launch table is filled for their shapes, then one
    step (per party: one grouped share call, one grouped full-tag call, one
    grouped CompactTag call and the checks) is captured as a CUDA graph and
    replayed.  Inputs are generated on the device (41 GiB)."""
    layers = synth.uneven_layers(256)
    t0 = time.perf_counter()
    shapes = [abi.make_layer(L.M, L.K, L.N, RING.k, RING.s) for L in layers]
    tuned = abi.mpc_autotune(shapes)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    tiles = {}
    for L in shapes:
        c = abi.mpc_autotune_choice(L)
        key = "integer pipes" if c[0] == 0 else f"tensor cores, {c[4]}-row tiles"
        tiles[key] = tiles.get(key, 0) + 1
    run = GpuWorkload(layers, torch, abi, device_gen=True)
    run.setup_grouped()
    for _ in range(warmup):
        run.step_grouped()
    torch.cuda.synchronize()
    g = capture(torch, run.step_grouped)
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    with Clocks(torch.cuda.current_device()) as ck:
        ms = timed_steps(torch, g.replay, EXTRA_STEPS)
    check_device(abi, "the grouped uneven steps")
    del g
    sh = time_calls(torch, lambda: run.share_group(1), 50, True, budget_s=0.5)
    fu = time_calls(torch, lambda: run.full_group(1), 50, True, budget_s=0.5)
    co = time_calls(torch, lambda: run.compact_group(1), 50, True, budget_s=0.5)
    check_device(abi, "the grouped uneven calls")
    units = step_units(layers)
    rec = {"workload": "uneven256_seeded", "layers": len(layers), "ring": f"Z_2^{RING.bits}",
           "parties": PARTIES, "steps": EXTRA_STEPS, "ms_per_step": ms,
           "ring_gmacs": units / (ms / 1e3) / 1e9,
           "step_launch": "CUDA graph replay of one captured step (grouped persistent launches)",
           "tag_overhead_ratio": pct(co, 50) / pct(fu, 50),
           "share_ms_p50": pct(sh, 50), "full_tag_ms_p50": pct(fu, 50), "compact_tag_ms_p50": pct(co, 50),
           "autotune": {"shapes": tuned, "seconds": tune_s, "choices": tiles},
           "gpu_launches_per_step": run.launches_per_step_grouped(),
           "inputs": "device-generated uniform words (41 GiB), resident", "clocks": ck.summary()}
    del run
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    abi.mpc_autotune_clear()
    return rec


def extra_vgg16(torch, abi, warmup, batches=(1, 16)):
    """VGG16 on 32x32x3 (13 convs as im2col GEMMs + 3 dense layers), Z_2^64, two
    parties, grouped calls with the launch table filled for the shapes; one
    captured step replayed per batch size."""
    out = {}
    for b in batches:
        layers = synth.vgg16_layers(b)
        abi.mpc_autotune([abi.make_layer(L.M, L.K, L.N, RING.k, RING.s) for L in layers])
        run = GpuWorkload(layers, torch, abi, device_gen=True)
        run.setup_grouped()
        for _ in range(warmup):
            run.step_grouped()
        g = capture(torch, run.step_grouped)
        for _ in range(warmup):
            g.replay()
        torch.cuda.synchronize()
        with Clocks(torch.cuda.current_device()) as ck:
            ms = timed_steps(torch, g.replay, 4 * EXTRA_STEPS)
        check_device(abi, f"the VGG16 b{b} steps")
        fu = time_calls(torch, lambda: run.full_group(1), 50, True, budget_s=0.3)
        co = time_calls(torch, lambda: run.compact_group(1), 50, True, budget_s=0.3)
        out[f"b{b}"] = {"ms_per_step": ms, "ring_gmacs": step_units(layers) / (ms / 1e3) / 1e9,
                        "tag_overhead_ratio": pct(co, 50) / pct(fu, 50), "clocks": ck.summary()}
        del g, run
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    abi.mpc_autotune_clear()
    out.update(workload="vgg16_32x32x3", ring=f"Z_2^{RING.bits}", parties=PARTIES,
               step_launch="CUDA graph replay of one captured step (grouped calls, launch table filled)",
               inputs="device-generated uniform words, resident")
    return out


def extra_serving(torch, abi, n_requests=200, load=0.7):
    """Serving (ResNet-18 / VGG16 requests, batch 1-32, Z_2^128): capacity from
    a closed-loop run of 48 requests, then n_requests Poisson arrivals at
    `load` of that capacity; request and tick latency percentiles from the
    open-loop run."""
    from paper_2311_04406_gb300.serve import Server, make_requests
    srv = Server(ring=synth.Z128, mem_budget=96 << 30)
    srv.run(make_requests(4, 1e9, seed=SEED + 1, all_at_once=True))
    cap = srv.run(make_requests(48, 1e9, seed=SEED, all_at_once=True))
    rate = load * cap["requests_per_s"]
    with Clocks(torch.cuda.current_device()) as ck:
        st = srv.run(make_requests(n_requests, rate, seed=SEED + 70))
    rec = {"workload": WORKLOADS["serve"][0], "ring": "Z_2^128 (k=64, s=64)", "party": 0,
           "capacity_requests_per_s": cap["requests_per_s"], "capacity_ring_gmacs": cap["ring_gmacs"],
           "offered_fraction": load, "offered_rate_per_s": rate, "requests": st["requests"],
           "requests_per_s": st["requests_per_s"], "ring_gmacs": st["ring_gmacs"],
           "latency_ms_p50": st["latency_ms_p50"], "latency_ms_p99": st["latency_ms_p99"],
           "tick_ms_p50": st["tick_ms_p50"], "tick_ms_p99": st["tick_ms_p99"], "ticks": st["ticks"],
           "tick_launch": st.get("tick_launch"),
           "scheduler": "memory-gated FCFS admission (96 GiB arena), one grouped share + tag call per tick "
                        "over every admitted request's next layer, 2 ticks in flight",
           "clocks": ck.summary()}
    del srv
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return rec


def abi_path_is_tc(abi, L) -> bool:
    """Whether the library routes this layer's GEMM to the tensor-core kernel."""
    lay = abi.make_layer(L.M, L.K, L.N, RING.k, RING.s)
    return abi.mpc_gemm_path(lay) == 1


def run_bytes(layers) -> int:
    tot = 0
    for L in layers:
        M, K, N = L.M, L.K, L.N
        per_party = 8 * (2 * M * K + 2 * K * N + 3 * M * N + 3 * M * N)
        tot += PARTIES * per_party + 8 * (M * K + K * N + M * N)
    return tot


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and the --impl reference arm)

def cpu_sample(layers, frac_rows):
    """A bounded sample of the step: share and full tag at the output rows
    [0, ceil(frac * M)) of each layer and party, and the whole CompactTag path
    (tag + check) of each layer and party.  Returns (callable, units)."""
    import oracle as O
    hi = host_inputs(layers)
    jobs, units = [], 0
    for L, pub, parties in hi:
        M, K, N = L.M, L.K, L.N
        m = max(1, int(np.ceil(frac_rows * M)))
        rows = np.repeat(np.arange(m, dtype=np.int64), N)
        cols = np.tile(np.arange(N, dtype=np.int64), m)
        for p, sh in enumerate(parties):
            bits = RING.bits
            jobs.append(lambda sh=sh, p=p, pub=pub, rows=rows, cols=cols, bits=bits: (
                O.linear_share_at(bits, p, pub["E"], pub["F"], sh["A"], sh["B"], sh["C"], rows, cols),
                O.linear_tag_full_at(bits, sh["alpha"], pub["E"], pub["F"], sh["mA"], sh["mB"],
                                     sh["mC"], rows, cols)))
            units += 2 * (2 * m * K * N)
            jobs.append(lambda sh=sh, pub=pub, bits=bits: O.check_compact(
                bits, sh["alpha"], pub["chi_hat"],
                *O.compact_tag(bits, sh["alpha"], pub["E"], pub["F"], sh["mA"], sh["mB"], sh["mC"],
                               sh["mR"], pub["Dt"], pub["chi"])[1::-1]))
            units += costmodel.compact_tag_mults(M, K, N) + M

    def run():
        for j in jobs:
            j()
    return run, units


def cpu_cores() -> int:
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def cpu_baseline(layers, budget_s=15.0):
    # calibrate on a small sample, then time a sample sized for ~budget_s
    run, units = cpu_sample(layers, 1.0 / 128)
    t0 = time.perf_counter(); run(); t1 = time.perf_counter()
    rate = units / max(t1 - t0, 1e-6)
    full_units = step_units(layers)
    frac = min(1.0, max(1.0 / 128, (budget_s * rate) / full_units))
    run, units = cpu_sample(layers, frac)
    t0 = time.perf_counter(); run(); t1 = time.perf_counter()
    # the same oracle on one core, on a sample a core count smaller
    import oracle as O
    cores = cpu_cores()
    old = O.set_threads(1)
    try:
        run1, units1 = cpu_sample(layers, max(1.0 / 4096, frac / max(1, cores)))
        s0 = time.perf_counter(); run1(); s1 = time.perf_counter()
    finally:
        O.set_threads(old)
    return {"value": units / (t1 - t0) / 1e9, "unit": "ring-GMAC/s", "cores": cores,
            "kind": "oracle", "seconds": t1 - t0,
            "single_thread": {"value": units1 / (s1 - s0) / 1e9, "seconds": s1 - s0, "cores": 1},
            "sample": (f"share + full tag at the first {frac:.4f} of output rows of both layers and "
                       f"both parties, plus the whole CompactTag tag and check of both layers and "
                       f"parties ({units:.3e} ring MACs)")}


def workload_layers(args):
    """(layers, workload name) of the command line."""
    wl_name, wl_fn = WORKLOADS[args.workload]
    if args.workload == "layer":
        M, K, N = args.shape
        layers = [synth.Layer(f"layer_{M}x{K}x{N}", M, K, N)]
        name = f"layer_{M}x{K}x{N}"
    elif wl_fn is None:
        # the serving mix: one ResNet-18 and one VGG16 request at the mean batch
        layers = synth.resnet18_layers(16) + synth.vgg16_layers(16)
        name = wl_name
    else:
        layers = wl_fn(args.batch)
        name = wl_name.format(b=args.batch)
    if PASS == "train":
        layers = layers + synth.backward_layers(layers)
        name += "_train"
    return layers, name


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    layers, workload = workload_layers(args)
    run, units = cpu_sample(layers, 1.0 / 64)
    for _ in range(args.warmup):
        run()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter(); run(); times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = units * args.steps / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ring-GMAC/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot / args.steps * 1e3, "p99_ms_per_step": pct([t * 1e3 for t in times], 99),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64" if RING.words == 1 else "u128 (two u64 words)",
        "data": "synthetic (uniform ring words from seeded SplitMix64)",
        "config": make_config(workload, layers, int(os.environ.get("WORLD_SIZE", "1"))),
        "runs_on": "host cores (the oracle), rank 0 alone",
        "cpu_baseline": {"value": value, "unit": "ring-GMAC/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": "per step: share + full tag at the first 1/64 of output rows and "
                                   "the whole CompactTag tag and check, both layers and parties"},
        "e2e": {"value": value, "unit": "ring-GMAC/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_serve(args):
    """Serving: ResNet-18 / VGG16 requests (batch 1-32, Z_2^128) through the
    continuous-batching loop.  A closed-loop run (all requests at t = 0)
    measures capacity; open-loop runs with Poisson arrivals at fractions of it
    give the latency percentiles.  value = ring-GMAC/s of the closed-loop run
    (share products + CompactTag tag and check of every layer)."""
    import torch
    from paper_2311_04406_gb300 import abi, build
    from paper_2311_04406_gb300.serve import Server, make_requests
    rank, ws = dist_init()
    if rank != 0:
        return
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    abi.load()
    ring = synth.Z128
    budget = int(args.serve_budget_gb * 2**30)

    def units_of(reqs):
        u = 0
        for r in reqs:
            for L in r.layers:
                u += 2 * L.M * L.K * L.N + costmodel.compact_tag_mults(L.M, L.K, L.N) + L.M
        return u

    srv = Server(ring=ring, mem_budget=budget)
    srv.run(make_requests(max(4, args.warmup), 1e9, seed=SEED + 1, all_at_once=True))
    n = args.serve_requests
    cap_reqs = make_requests(n, 1e9, seed=SEED, all_at_once=True)
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as ck:
        cap = srv.run(cap_reqs)
    cap_units = units_of(cap_reqs)
    value = cap_units / (cap["makespan_ms"] / 1e3) / 1e9
    runs = []
    for frac in (0.3, 0.5, 0.7, 0.9):
        rate = frac * cap["requests_per_s"]
        reqs = make_requests(n, rate, seed=SEED + int(frac * 100))
        st = srv.run(reqs)
        st.update(offered_fraction=frac, offered_rate_per_s=rate)
        runs.append(st)
    full = srv.run(make_requests(n, 1e9, seed=SEED, all_at_once=True), tag="full")
    line = {
        "metric": METRIC, "value": value, "unit": "ring-GMAC/s", "n_gpus": 1,
        "steps": n, "warmup": args.warmup, "ms_per_step": cap["makespan_ms"] / n,
        "step": "one request (closed loop, all requests resident as admitted)",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u128 (two u64 words)",
        "data": "synthetic (request shares from seeded device generators; shapes of ResNet-18 / VGG16 on 32x32x3)",
        "config": {"workload": WORKLOADS["serve"][0], "ring": "Z_2^128 (k=64, s=64)", "requests_per_run": n,
                   "memory_budget_gib": args.serve_budget_gb, "party": 0,
                   "scheduler": "memory-gated FCFS admission, one grouped share + tag call per tick over "
                                "every admitted request's next layer, 2 ticks in flight"},
        "capacity": cap, "open_loop": runs,
        "full_tag_capacity": full,
        "tag_overhead_ratio": None,
        "gpu_launches": None, "clocks": ck.summary(), "e2e": None, "cpu_baseline": None,
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--eager", action="store_true", help="time eager API calls instead of graph replay")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the grouped uneven-layer, VGG16 and serving records")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cnn",
                    help="layer set (default: the CNN pair, conv 1024x576x64 + dense 128x4096x4096)")
    ap.add_argument("--batch", type=int, default=1, help="batch size for vgg16 / resnet18")
    ap.add_argument("--shape", type=lambda v: tuple(int(x) for x in v.split(",")), default=None,
                    help="M,K,N of the one layer of --workload layer")
    ap.add_argument("--ring", type=int, choices=[64, 128], default=64,
                    help="share ring Z_2^64 (k=s=32) or Z_2^128 (k=s=64)")
    ap.add_argument("--protocol", choices=["plain", "trunc"], default="plain",
                    help="trunc: the truncated layer (share without E.F, public product, "
                         "OptMAC&Trunc, compact tag without the E.F term)")
    ap.add_argument("--serve-requests", type=int, default=48, help="requests per serving run")
    ap.add_argument("--serve-budget-gb", type=float, default=96.0, help="serving memory budget (GiB)")
    ap.add_argument("--autotune", action="store_true",
                    help="fill the launch table for the workload's shapes (timed candidates) before warm-up")
    ap.add_argument("--grouped", action="store_true",
                    help="one grouped call of each kind per party for all layers (persistent grouped "
                         "tensor-core launches) instead of one call per layer")
    ap.add_argument("--pass", dest="pass_", choices=["forward", "train"], default="forward",
                    help="train: each layer's forward product and its two gradient products "
                         "(grad X = G.W^T, grad W = X^T.G on transposed mask shares)")
    args = ap.parse_args()
    global RING, PROTOCOL, PASS
    PASS = args.pass_
    RING = synth.Z64 if args.ring == 64 else synth.Z128
    PROTOCOL = args.protocol
    if args.warmup < 3:
        args.warmup = 3
    if args.grouped and PROTOCOL != "plain":
        ap.error("--grouped runs the untruncated layer (--protocol plain)")
    if (args.workload == "layer") != (args.shape is not None) or (args.shape is not None and len(args.shape) != 3):
        ap.error("--workload layer takes --shape M,K,N (and --shape needs --workload layer)")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
