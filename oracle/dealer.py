"""Trusted dealer and party simulation for tests -- TEST INFRASTRUCTURE.

The offline phase (§3.5) and F_MAC (App. A.2) are replaced by a trusted dealer,
as in the simulator of the security proof (App. B): it knows the global key and
the triples and hands each party consistent authenticated shares.

  * alpha_i uniform in [0, 2^s) per party; alpha = sum_i alpha_i mod 2^{k+s}.
  * A~, B~ uniform; C~ = A~ . B~ mod 2^{k+s}; R~ uniform (Fig. Pi_MatMul and
    Fig. Pi_OptMAC preprocessing).
  * every secret V in {A, B, C, R} is additively shared: parties 0..n-2 draw
    uniform shares, the last party's share makes the sum V~; its tag
    m(V) = alpha . V~ (§2.4) is shared the same way.
  * X~, Y~ uniform; the opened E = X~ - A~ and F = Y~ - B~ (Fig. Pi_MatMul
    step 1) are public.  chi (N) and chi^ (M) are public coins in [0, 2^s)
    (F_Rand, App. A.1).

Randomness comes from `synth` (uniform words); all ring arithmetic goes
through `oracle`.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

import oracle as O
import synth


def _store(bits: int, a: np.ndarray) -> np.ndarray:
    """Values below 2^64 re-stored in the storage of Z_{2^bits} (hi word 0)."""
    if O.words(bits) == 1:
        return np.ascontiguousarray(a.astype(np.uint64))
    out = np.zeros(a.shape + (2,), dtype=np.uint64)
    out[..., 0] = a
    return out


def key_range(ring: synth.Ring, seed: int, tid: int, party: int, shape) -> np.ndarray:
    """Uniform elements of [0, 2^s) (s <= 64) stored in ring width k + s."""
    if ring.s > 64:
        raise ValueError("key ring wider than 64 bits is not used")
    return _store(ring.bits, synth.uniform(seed, tid, party, shape, ring.s))


@dataclass
class Party:
    """One party's authenticated shares for one layer."""
    index: int
    alpha: np.ndarray
    A: np.ndarray
    B: np.ndarray
    C: np.ndarray
    R: np.ndarray
    mA: np.ndarray
    mB: np.ndarray
    mC: np.ndarray
    mR: np.ndarray


@dataclass
class Deal:
    ring: synth.Ring
    M: int
    K: int
    N: int
    alpha: np.ndarray            # global key (one element)
    X: np.ndarray                # secret inputs (for invariants only)
    Y: np.ndarray
    A: np.ndarray                # reconstructed triple (for invariants only)
    B: np.ndarray
    C: np.ndarray
    R: np.ndarray
    E: np.ndarray                # public opened matrices
    F: np.ndarray
    chi: np.ndarray
    chi_hat: np.ndarray
    parties: list = field(default_factory=list)


def _share(bits, seed, tid, target, n, shape):
    """Additive shares of `target`: uniform for parties 0..n-2, last fixes the sum."""
    shares = [synth.uniform(seed, tid, i + 1, shape, bits) for i in range(n - 1)]
    last = target.copy()
    for s_ in shares:
        last = O.sub(bits, last, s_)
    return shares + [last]


def deal(ring: synth.Ring, M: int, K: int, N: int, n: int = 2, seed: int = 1,
         alpha_full_width: bool = False) -> Deal:
    bits = ring.bits
    T = synth.TID
    if alpha_full_width:
        alphas = [synth.uniform(seed, T["alpha"], i, (1,), bits) for i in range(n)]
    else:
        alphas = [key_range(ring, seed, T["alpha"], i, (1,)) for i in range(n)]
    alpha = alphas[0].copy()
    for a in alphas[1:]:
        alpha = O.add(bits, alpha, a)
    X = synth.uniform(seed, T["X"], 0, (M, K), bits)
    Y = synth.uniform(seed, T["Y"], 0, (K, N), bits)
    A = synth.uniform(seed, T["A"], 0, (M, K), bits)
    B = synth.uniform(seed, T["B"], 0, (K, N), bits)
    C = O.ring_gemm(bits, A, B)
    R = synth.uniform(seed, T["R"], 0, (M, N), bits)
    E = O.sub(bits, X, A)
    F = O.sub(bits, Y, B)
    chi = key_range(ring, seed, T["chi"], 0, (N,))
    chi_hat = key_range(ring, seed, T["chi_hat"], 0, (M,))
    sh = {}
    for name, V, shape in (("A", A, (M, K)), ("B", B, (K, N)), ("C", C, (M, N)), ("R", R, (M, N))):
        sh[name] = _share(bits, seed, T[name], V, n, shape)
        sh["m" + name] = _share(bits, seed, T["m" + name], O.smul(bits, alpha, V), n, shape)
    parties = [Party(i, alphas[i], sh["A"][i], sh["B"][i], sh["C"][i], sh["R"][i],
                     sh["mA"][i], sh["mB"][i], sh["mC"][i], sh["mR"][i]) for i in range(n)]
    return Deal(ring, M, K, N, alpha, X, Y, A, B, C, R, E, F, chi, chi_hat, parties)


def total(bits: int, arrays) -> np.ndarray:
    """Opening: sum of the parties' shares mod 2^{k+s}."""
    arrays = list(arrays)
    acc = arrays[0].copy()
    for a in arrays[1:]:
        acc = O.add(bits, acc, a)
    return acc


def run_layer(d: Deal, tamper=None):
    """Run the whole per-layer protocol for every party through the oracle.

    Returns a dict of per-party lists and public values.  `tamper` is an
    optional dict of host-side fault injections:
      "Z": (party, flat_index, e)   add e to one party's [Z]_i before opening D
      "Dt": (flat_index, e)         add e to the broadcast D~ seen by everyone
      "alpha": (party, e)           use alpha_i + e in that party's tag
    """
    tamper = tamper or {}
    bits = d.ring.bits
    Z = [O.linear_share(bits, p.index, d.E, d.F, p.A, p.B, p.C) for p in d.parties]
    if "Z" in tamper:
        i, j, e = tamper["Z"]
        flat = Z[i].reshape(-1, O.words(bits))
        flat[j] = O.from_int(O.to_int(flat[j], bits) + e, bits)
    mZ_full = [O.linear_tag_full(bits, p.alpha, d.E, d.F, p.mA, p.mB, p.mC) for p in d.parties]
    D = [O.sub(bits, p.R, z) for p, z in zip(d.parties, Z)]
    Dt = total(bits, D)
    if "Dt" in tamper:
        j, e = tamper["Dt"]
        flat = Dt.reshape(-1, O.words(bits))
        flat[j] = O.from_int(O.to_int(flat[j], bits) + e, bits)
    alphas = [p.alpha for p in d.parties]
    if "alpha" in tamper:
        i, e = tamper["alpha"]
        alphas[i] = O.from_int(O.to_int(alphas[i], bits).reshape(-1)[0] + e, bits).reshape(alphas[i].shape)
    mZ_opt = [O.optmac(bits, a, p.mR, Dt) for a, p in zip(alphas, d.parties)]
    comp = [O.compact_tag(bits, a, d.E, d.F, p.mA, p.mB, p.mC, p.mR, Dt, d.chi)
            for a, p in zip(alphas, d.parties)]
    mDc = [c[0] for c in comp]
    Dc = comp[0][1]
    mZc = [c[2] for c in comp]
    cs = [O.check_compact(bits, a, d.chi_hat, Dc, m) for a, m in zip(alphas, mDc)]
    return dict(Z=Z, mZ_full=mZ_full, D=D, Dt=Dt, mZ_opt=mZ_opt, mDc=mDc, Dc=Dc,
                mZc=mZc, cs=cs, cs_total=total(bits, cs))


# ---------------------------------------------------------------------------
# truncated layer: the preprocessing of Fig. Pi_OptMAC&Trunc adds shares of a
# random R~ in [0, 2^k) and of R~^f = R~ / 2^f (floor), both authenticated.

@dataclass
class TruncDeal:
    base: Deal
    f: int
    R: np.ndarray                 # R~ (k-bit)
    Rf: np.ndarray                # R~ >> f
    Rf_shares: list = field(default_factory=list)
    mRf_shares: list = field(default_factory=list)


def deal_trunc(ring: synth.Ring, M: int, K: int, N: int, n: int = 2, seed: int = 1,
               f: int = 16) -> TruncDeal:
    d = deal(ring, M, K, N, n=n, seed=seed)
    bits = ring.bits
    T = synth.TID
    Rk = _store(bits, synth.uniform(seed, T["R"], 99, (M, N), ring.k)) if ring.k <= 64 else None
    Rf = O.from_int(np.vectorize(lambda v: int(v) >> f, otypes=[object])(O.to_int(Rk, bits)), bits)
    # re-share R~ (k-bit) and R~^f with tags, replacing the dealer's R
    R_sh = _share(bits, seed, T["R"], Rk, n, (M, N))
    mR_sh = _share(bits, seed, T["mR"], O.smul(bits, d.alpha, Rk), n, (M, N))
    for p, r, mr in zip(d.parties, R_sh, mR_sh):
        p.R, p.mR = r, mr
    d.R = Rk
    Rf_sh = _share(bits, seed, T["Rf"], Rf, n, (M, N))
    mRf_sh = _share(bits, seed, T["mRf"], O.smul(bits, d.alpha, Rf), n, (M, N))
    return TruncDeal(d, f, Rk, Rf, Rf_sh, mRf_sh)


def run_layer_trunc(t: TruncDeal, tamper=None):
    """The truncated layer for every party through the oracle.  `tamper`:
    {"Dt": (flat_index, e)} adds e to the broadcast D~."""
    tamper = tamper or {}
    d = t.base
    bits = d.ring.bits
    Z = [O.linear_share_trunc(bits, d.E, d.F, p.A, p.B, p.C) for p in d.parties]
    Dt = total(bits, [O.sub(bits, p.R, z) for p, z in zip(d.parties, Z)])
    if "Dt" in tamper:
        j, e = tamper["Dt"]
        flat = Dt.reshape(-1, O.words(bits))
        flat[j] = O.from_int(O.to_int(flat[j], bits) + e, bits)
    P = O.public_product(bits, d.E, d.F)
    outs = [O.optmac_trunc(d.ring.k, d.ring.s, t.f, i, p.alpha, t.Rf_shares[i], t.mRf_shares[i], Dt, P)
            for i, p in enumerate(d.parties)]
    comp = [O.compact_tag_trunc(bits, p.alpha, d.E, d.F, p.mA, p.mB, p.mC, p.mR, Dt, d.chi)
            for p in d.parties]
    mDc = [c[0] for c in comp]
    Dc = comp[0][1]
    cs = [O.check_compact(bits, p.alpha, d.chi_hat, Dc, m) for p, m in zip(d.parties, mDc)]
    return dict(Z=Z, Dt=Dt, P=P, Zf=[o[0] for o in outs], mZf=[o[1] for o in outs], mDc=mDc,
                Dc=Dc, mZc=[c[2] for c in comp], cs=cs, cs_total=total(bits, cs))


# ---------------------------------------------------------------------------
# Pi_BatchRec: authenticated shares of a value V (as X - A) and of a mask R with
# R~ = 2^k r (so R~ = 0 mod 2^k), both with tags, for n parties.

@dataclass
class RecDeal:
    ring: synth.Ring
    alpha: np.ndarray
    alphas: list
    V: np.ndarray                 # reconstructed X - A
    X: list = field(default_factory=list)
    A: list = field(default_factory=list)
    R: list = field(default_factory=list)
    mX: list = field(default_factory=list)
    mA: list = field(default_factory=list)
    mR: list = field(default_factory=list)


def deal_batchrec(ring: synth.Ring, rows: int, cols: int, n: int = 2, seed: int = 1) -> RecDeal:
    bits = ring.bits
    T = synth.TID
    alphas = [key_range(ring, seed, T["alpha"], i, (1,)) for i in range(n)]
    alpha = total(bits, alphas)
    shape = (rows, cols)
    Xt = synth.uniform(seed, T["X"], 50, shape, bits)
    At = synth.uniform(seed, T["A"], 50, shape, bits)
    r = synth.uniform(seed, T["W"], 50, shape, ring.s)
    Rt = O.from_int(np.vectorize(lambda v: int(v) << ring.k, otypes=[object])(O.to_int(_store(bits, r), bits)), bits)
    d = RecDeal(ring, alpha, alphas, O.sub(bits, Xt, At))
    for name, V, lst, mlst in (("X", Xt, d.X, d.mX), ("A", At, d.A, d.mA), ("R", Rt, d.R, d.mR)):
        lst += _share(bits, seed, T[name] + 60, V, n, shape)
        mlst += _share(bits, seed, T[name] + 160, O.smul(bits, alpha, V), n, shape)
    return d


# ---------------------------------------------------------------------------
# Training's backward linear layers (§4 training workloads).  Given the forward
# layer Z = X . W (X = X~ is M x K, W = Y~ is K x N, masked by the triple's A, B
# as E = X - A, F = W - B), the gradients of a secret upstream gradient G (M x N)
# are two more Beaver products:
#   grad X = G . W^T   (M x N by N x K): a layer (M, N, K)
#   grad W = X^T . G   (K x M by M x N): a layer (K, M, N)
# The paper does not fix how the backward triples relate to the forward ones.
# Reading used here: every secret is masked once and the mask is reused in
# transposed form -- W^T by B^T (so F' = F^T is already public), X^T by A^T
# (E'' = E^T), and G by one fresh mask A' used on the left of grad X and on the
# right of grad W (E' = F'' = G - A').  Each party transposes its own shares and
# tags of A, B locally; only G - A' is opened, and the triples' C parts are
# fresh: C' = A' . B^T, C'' = A^T . A'.

def transpose(a: np.ndarray) -> np.ndarray:
    """Matrix transpose of ring-element storage ((rows, cols) or (rows, cols, 2))."""
    return np.ascontiguousarray(np.swapaxes(a, 0, 1))


@dataclass
class BackDeal:
    fwd: Deal
    G: np.ndarray                 # upstream gradient (secret, for invariants only)
    dX: Deal                      # grad X = G . W^T as a layer (M, N, K)
    dW: Deal                      # grad W = X^T . G as a layer (K, M, N)


def deal_backward(d: Deal, seed: int = 1) -> BackDeal:
    ring, bits, n = d.ring, d.ring.bits, len(d.parties)
    M, K, N = d.M, d.K, d.N
    alpha = d.alpha
    base = 400                     # tensor ids of the backward streams

    def fresh(tid, shape):
        return synth.uniform(seed, base + tid, 0, shape, bits)

    def shares(tid, V, shape):
        return (_share(bits, seed, base + tid, V, n, shape),
                _share(bits, seed, base + 100 + tid, O.smul(bits, alpha, V), n, shape))

    G = fresh(1, (M, N))
    Ag = fresh(2, (M, N))                       # mask of G
    Ag_sh, mAg_sh = shares(2, Ag, (M, N))
    Eg = O.sub(bits, G, Ag)                     # the one new opening
    layers = []
    # grad X = G . W^T: left operand G (mask A'), right operand W^T (mask B^T)
    Bt = transpose(d.B)
    Cx = O.ring_gemm(bits, Ag, Bt)
    Rx = fresh(3, (M, K))
    Cx_sh, mCx_sh = shares(3, Cx, (M, K))
    Rx_sh, mRx_sh = shares(4, Rx, (M, K))
    px = [Party(i, p.alpha, Ag_sh[i], transpose(p.B), Cx_sh[i], Rx_sh[i],
                mAg_sh[i], transpose(p.mB), mCx_sh[i], mRx_sh[i]) for i, p in enumerate(d.parties)]
    layers.append(Deal(ring, M, N, K, alpha, G, transpose(d.Y), Ag, Bt, Cx, Rx, Eg, transpose(d.F),
                       key_range(ring, seed, base + 5, 0, (K,)),
                       key_range(ring, seed, base + 6, 0, (M,)), px))
    # grad W = X^T . G: left operand X^T (mask A^T), right operand G (mask A')
    At = transpose(d.A)
    Cw = O.ring_gemm(bits, At, Ag)
    Rw = fresh(7, (K, N))
    Cw_sh, mCw_sh = shares(7, Cw, (K, N))
    Rw_sh, mRw_sh = shares(8, Rw, (K, N))
    pw = [Party(i, p.alpha, transpose(p.A), Ag_sh[i], Cw_sh[i], Rw_sh[i],
                transpose(p.mA), mAg_sh[i], mCw_sh[i], mRw_sh[i]) for i, p in enumerate(d.parties)]
    layers.append(Deal(ring, K, M, N, alpha, transpose(d.X), G, At, Ag, Cw, Rw, transpose(d.E), Eg,
                       key_range(ring, seed, base + 9, 0, (N,)),
                       key_range(ring, seed, base + 10, 0, (K,)), pw))
    return BackDeal(d, G, layers[0], layers[1])
