"""Host-side lowering of a quadratic-activation CNN to the library's program.

Offline model preparation (run once per model, before inference):

* parameter transforms -- batch norm folded into the preceding convolution
  (node fusing Case 2, Sec. 4.1) and forward weight redistribution (Sec. 4.2):
  each activation a x^2 + b x + c becomes monic x^2 + (b/a) x + (c/a), the
  average pool a plain sum, and the receivers absorb the updates;
* slot layouts (Sec. 5.1): the HW layout (a channel per ciphertext, its
  spatial values replicated into every free block of slots) or a
  channel-packed layout (one block of slots per channel); strided layers keep
  the gaps they leave (adaptive mapping);
* every linear layer as diagonals in baby-step / giant-step form:
  out = sum_g rot_g( sum_(i,b) d'_(i,g,b) (.) rot_b(in_i) ), with
  d'_(g,b) the diagonal of rotation g+b pre-rotated by -g; the giant step
  of a channel-packed convolution is k blocks of slots, k chosen per layer
  by a key-switch cost model (``bsgs_cost``: baby steps share one ModUp per
  input, giant steps share one ModDown per output);
* levels, scales and rescale points by the tower-reuse rule of Sec. 4.3
  (rescale when round(log_Delta scale) exceeds round(log_Delta q_level)).

The result is handed to ``fhe_model_load``; the homomorphic evaluation itself
runs in the CUDA library.  Expressions that decide encoded integers (folded
weights, plaintext scales, activation constants) use a fixed floating-point
operation order, documented at each.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import _lib as F


# =========================================================== transforms

def _by_input_channel(u, w: np.ndarray) -> np.ndarray:
    """w [cout, cin, ...] times u (a scalar, or one value per input channel)"""
    if np.ndim(u) == 0:
        return w * u
    return w * np.reshape(u, (1, -1) + (1,) * (w.ndim - 2))


def fuse_bn_act(b1, b0, c2, c1, c0):
    """Node fusing Case 1 (Sec. 4.1): P(B(x)) with B(x) = b1 x + b0 and
    P(x) = c2 x^2 + c1 x + c0 is p2 x^2 + p1 x + p0 with p2 = b1^2 c2,
    p1 = b1 (2 b0 c2 + c1), p0 = b0^2 c2 + b0 c1 + c0."""
    return b1 * b1 * c2, b1 * (2.0 * b0 * c2 + c1), b0 * b0 * c2 + b0 * c1 + c0


def prepare_params(net: List[Dict], raw: Dict) -> Dict[int, Dict]:
    """Folded, redistributed parameters per node.  Operation order:
    b1 = gamma/sigma; b0 = beta - b1*mu; w' = (w*b1[o])*u_in;
    bias' = bias*b1 + b0; activation c1 = b/a, c0 = c/a (u = a);
    pool u = u_in/float(k*k); dense w' = w*u_in; identity shortcut times u.
    A batch norm of its own (a "bn" node, not after a convolution) feeds one
    activation and fuses into it (Case 1, b1 times the u of its input):
    p2 x^2 + p1 x + p0 per channel, monic c1 = p1/p2, c0 = p0/p2, u = p2
    per channel (taken up by the next layer's input channels)."""
    u: Dict[int, float] = {}
    out: Dict[int, Dict] = {}
    for idx, node in enumerate(net):
        kind = node["op"]
        if kind == "input":
            u[idx] = 1.0
            continue
        if kind == "conv":
            p = raw[idx]
            b1 = p["gamma"] / p["sigma"]
            b0 = p["beta"] - b1 * p["mu"]
            out[idx] = dict(w=_by_input_channel(u[node["src"]], p["w"] * b1.reshape(-1, 1, 1, 1)),
                            bias=p["bias"] * b1 + b0)
            u[idx] = 1.0
        elif kind == "bn":
            users = [n["op"] for n in net if n.get("src") == idx or
                     (isinstance(n.get("src"), list) and idx in n["src"])]
            if users != ["act"]:
                raise ValueError("a batch norm of its own must feed one activation (node fusing Case 1)")
            u[idx] = None
        elif kind == "act" and net[node["src"]]["op"] == "bn":
            p, q = raw[idx], raw[node["src"]]
            b1 = q["gamma"] / q["sigma"]
            b0 = q["beta"] - b1 * q["mu"]
            p2, p1, p0 = fuse_bn_act(b1 * u[net[node["src"]]["src"]], b0, p["a"], p["b"], p["c"])
            out[idx] = dict(c1=p1 / p2, c0=p0 / p2)
            u[idx] = p2
        elif kind == "act":
            p = raw[idx]
            out[idx] = dict(c1=p["b"] / p["a"], c0=p["c"] / p["a"])
            u[idx] = p["a"]
        elif kind == "pool":
            u[idx] = u[node["src"]] / float(node["k"] * node["k"])
        elif kind == "dense":
            p = raw[idx]
            ud = u[node["src"]]
            if np.ndim(ud) != 0:
                ud = np.repeat(ud, p["w"].shape[1] // len(ud))   # inputs are channel-major
            out[idx] = dict(w=p["w"] * ud, bias=p["bias"])
            u[idx] = 1.0
        elif kind == "add":
            sc = node["src"][1]
            if net[sc]["op"] != "conv" and np.ndim(u[sc]) != 0:
                raise ValueError("an identity shortcut needs one upsilon for all channels")
            out[idx] = dict(shortcut=None if net[sc]["op"] == "conv" else u[sc])
            u[idx] = 1.0
    return out


# =========================================================== layouts

@dataclass
class SlotMap:
    """Channel c has copies at (ciphertext, base slot) pairs copies[c]; its
    logical position (h, w) is at base + h*st*row + w*st."""
    n_ct: int
    copies: List[List[Tuple[int, int]]]
    H: int
    W: int
    st: int
    row: int
    block: int

    def offsets(self) -> np.ndarray:
        h = np.arange(self.H).reshape(-1, 1)
        w = np.arange(self.W).reshape(1, -1)
        return (h * self.st * self.row + w * self.st).reshape(-1)


def map_hw(c, H, W, n_slots) -> SlotMap:
    blk = H * W
    bases = [b * blk for b in range(n_slots // blk)]
    return SlotMap(c, [[(ch, base) for base in bases] for ch in range(c)], H, W, 1, W, blk)


def map_hw_ensemble(c, H, W, n_slots, members: int) -> SlotMap:
    """HW layout of an ensemble (Sec. 5.3): channel c in ciphertext c, member
    m's values in block m (blocks >= members stay empty)."""
    blk = H * W
    if members * blk > n_slots:
        raise ValueError("the ensemble does not fit in the free blocks")
    return SlotMap(c, [[(ch, m * blk) for m in range(members)] for ch in range(c)], H, W, 1, W, blk)


def map_packed(c, H, W, st, row, blk, n_slots) -> SlotMap:
    nb = n_slots // blk
    if c <= nb:
        used = c * (nb // c)
        copies = [[(0, b * blk) for b in range(ch, used, c)] for ch in range(c)]
        return SlotMap(1, copies, H, W, st, row, blk)
    if c % nb:
        raise ValueError("channel count must be a multiple of the blocks per ciphertext")
    return SlotMap(c // nb, [[(ch // nb, (ch % nb) * blk)] for ch in range(c)], H, W, st, row, blk)


def map_single(c, blk, n_slots) -> SlotMap:
    nb = n_slots // blk
    return SlotMap(-(-c // nb), [[(k // nb, (k % nb) * blk)] for k in range(c)], 1, 1, 1, 1, blk)


def _pick_copy(copies, out_base, n_slots):
    best = None
    for ct, base in copies:
        key = ((base - out_base) % n_slots, ct)
        if best is None or key < best[0]:
            best = (key, ct, base)
    return best[1], best[2]


class SparseVec:
    """A slot vector given by its nonzero entries (slots ascending): the form
    in which weight vectors of a step encoded on demand are kept (a dense
    vector of a 512-channel packed convolution is N/2 doubles, of which a
    few hundred are nonzero)."""

    __slots__ = ("slots", "vals")

    def __init__(self, slots, vals):
        order = np.argsort(slots, kind="stable")
        self.slots = np.asarray(slots, dtype=np.int64)[order]
        self.vals = np.asarray(vals, dtype=np.float64)[order]

    def roll(self, g: int, n_slots: int) -> "SparseVec":
        """np.roll of the dense vector by g"""
        return SparseVec((self.slots + g) % n_slots, self.vals)

    def key(self) -> bytes:
        return self.slots.tobytes() + b"|" + self.vals.tobytes()

    def dense(self, n_slots: int) -> np.ndarray:
        v = np.zeros(n_slots)
        v[self.slots] = self.vals
        return v

    def __len__(self):
        return len(self.slots)


def diagonals(w: np.ndarray, stride: int, pad: int, src: SlotMap, dst: SlotMap, n_slots: int,
              sparse: bool = False):
    """{(out ct, in ct, r): vector} such that out[s] = sum_r vec[s]*in[s + r]
    (vectors as SparseVec with sparse=True)."""
    cout, cin, k, _ = w.shape
    oh = np.repeat(np.arange(dst.H), dst.W)
    ow = np.tile(np.arange(dst.W), dst.H)
    # kernel offsets: the valid output positions and their input offsets
    # (the same for every channel pair)
    offs = []
    for dh in range(k):
        ih = oh * stride + dh - pad
        for dw in range(k):
            iw = ow * stride + dw - pad
            ok = (ih >= 0) & (ih < src.H) & (iw >= 0) & (iw < src.W)
            if ok.any():
                offs.append((dh, dw, ok, ih[ok] * src.st * src.row + iw[ok] * src.st))
    rows = {"oc": [], "ic": [], "r": [], "so": [], "v": []}
    for o in range(cout):
        for oct_, obase in dst.copies[o]:
            so = obase + oh * dst.st * dst.row + ow * dst.st
            picks = [_pick_copy(src.copies[i], obase, n_slots) for i in range(cin)]
            ict = np.array([p_[0] for p_ in picks], dtype=np.int64)
            ibase = np.array([p_[1] for p_ in picks], dtype=np.int64)
            for dh, dw, ok, si_off in offs:
                so_ok = so[ok]
                n_ok = len(so_ok)
                # all input channels at once: [cin, n_ok]
                si = ibase[:, None] + si_off[None, :]
                rows["oc"].append(np.full(cin * n_ok, oct_))
                rows["ic"].append(np.repeat(ict, n_ok))
                rows["r"].append(((si - so_ok[None, :]) % n_slots).reshape(-1))
                rows["so"].append(np.tile(so_ok, cin))
                rows["v"].append(np.repeat(w[o, :, dh, dw], n_ok))
    oc = np.concatenate(rows["oc"])
    ic = np.concatenate(rows["ic"])
    r = np.concatenate(rows["r"])
    so = np.concatenate(rows["so"])
    v = np.concatenate(rows["v"])
    order = np.lexsort((so, r, ic, oc))
    oc, ic, r, so, v = oc[order], ic[order], r[order], so[order], v[order]
    key = np.stack([oc, ic, r], axis=1)
    cut = np.flatnonzero(np.any(key[1:] != key[:-1], axis=1)) + 1
    out = {}
    for lo, hi in zip(np.concatenate([[0], cut]), np.concatenate([cut, [len(oc)]])):
        seg_so = so[lo:hi]
        if np.any(seg_so[1:] == seg_so[:-1]):
            raise ValueError("two weights land on one diagonal slot")
        if sparse:
            vec = SparseVec(seg_so, v[lo:hi])
        else:
            vec = np.zeros(n_slots)
            vec[seg_so] = v[lo:hi]
        out[(int(oc[lo]), int(ic[lo]), int(r[lo]))] = vec
    return out


# =========================================================== program

@dataclass
class Terms:
    """The diagonals of a linear layer as arrays: term t adds vecs[vid[t]]
    (.) rot(in[ct[t]], r[t]) into output ciphertext out[t].  Equal vectors
    share one table entry (one encoded plaintext)."""
    out: np.ndarray
    ct: np.ndarray
    r: np.ndarray
    vid: np.ndarray
    vecs: List[np.ndarray]


def terms_of(diag: Dict) -> Terms:
    keys = sorted(diag)
    a = np.array(keys, dtype=np.int64).reshape(-1, 3)
    return Terms(a[:, 0], a[:, 1], a[:, 2], np.arange(len(keys)), [diag[k] for k in keys])


def diagonals_hw(ws: Sequence[np.ndarray], stride: int, pad: int, src: SlotMap, dst: SlotMap,
                 n_slots: int) -> Terms:
    """Convolution between HW layouts (channel c in ciphertext c): output
    replica k reads input replica k (same block), with weights ws[k]
    [cout, cin, k, k] (the replica's ensemble member).  For a kernel offset
    (dh, dw) every term reads rotation r = ((dh-pad) row + (dw-pad)) st_in,
    and its vector holds weight ws[k][o, i, dh, dw] on the valid output
    positions of replica k."""
    cout, cin, kh, kw = ws[0].shape
    oh = np.repeat(np.arange(dst.H), dst.W)
    ow = np.tile(np.arange(dst.W), dst.H)
    bases = [b for _, b in dst.copies[0]]
    if [b for _, b in src.copies[0]] != bases or len(ws) != len(bases):
        raise ValueError("HW convolution: replicas of input and output differ")
    o_idx, i_idx = np.meshgrid(np.arange(cout), np.arange(cin), indexing="ij")
    o_idx, i_idx = o_idx.reshape(-1), i_idx.reshape(-1)
    outs, cts, rs, vids, vecs = [], [], [], [], []
    for dh in range(kh):
        ih = oh * stride + dh - pad
        for dw in range(kw):
            iw = ow * stride + dw - pad
            ok = (ih >= 0) & (ih < src.H) & (iw >= 0) & (iw < src.W)
            if not ok.any():
                continue
            r = (((dh - pad) * src.st) * src.row + (dw - pad) * src.st) % n_slots
            so = oh[ok] * dst.st * dst.row + ow[ok] * dst.st
            tup = np.stack([w[:, :, dh, dw].reshape(-1) for w in ws], axis=1)
            uniq, inv = np.unique(tup, axis=0, return_inverse=True)
            base_vid = len(vecs)
            for u in uniq:
                v = np.zeros(n_slots)
                for k, b in enumerate(bases):
                    v[b + so] = u[k]
                vecs.append(v)
            outs.append(o_idx)
            cts.append(i_idx)
            rs.append(np.full(len(o_idx), r, dtype=np.int64))
            vids.append(base_vid + inv.reshape(-1))
    return Terms(np.concatenate(outs), np.concatenate(cts), np.concatenate(rs), np.concatenate(vids), vecs)


@dataclass
class TInfo:
    layout: SlotMap
    level: int
    scale: float


@dataclass
class Program:
    tensors: List[TInfo] = field(default_factory=list)
    steps: List[Dict] = field(default_factory=list)
    rotations: set = field(default_factory=set)
    input: int = 0
    output: int = 0


def _lam(x: float, log_delta: float) -> int:
    return int(math.floor(math.log2(x) / log_delta + 0.5))


def _round_int(v: float) -> float:
    """round half away from zero, as an integral double"""
    if abs(v) >= 2.0 ** 52:
        return float(v)
    return math.copysign(math.floor(abs(v) + 0.5), v)


def ks_cost(level: int, alpha: int) -> Tuple[float, float, float]:
    """Cost, in length-N limb transforms (8 modular products per coefficient),
    of the three parts of one hybrid key switch at `level`: ModUp (inverse NTT
    of the level+1 limbs; per digit a basis conversion of its d primes to the
    ext - d others, d products per output coefficient, and their forward
    NTT), the key inner product (two products per digit and extended limb),
    ModDown (inverse NTT of 2 alpha special limbs, conversion of both
    polynomials to the level+1 primes with alpha products each, forward NTT
    of 2 (level+1) limbs)."""
    nl = level + 1
    ext = nl + alpha
    digits = [min(alpha, nl - j) for j in range(0, nl, alpha)]
    modup = nl + sum((ext - d) * (1 + d / 8) for d in digits)
    ip = len(digits) * ext * 2 / 8
    moddown = 2 * alpha + 2 * nl * (1 + alpha / 8)
    return modup, ip, moddown


def bsgs_cost(terms: Terms, giant: int, level: int, alpha: int) -> float:
    """Key-switch cost of a linear layer whose diagonals are `terms`, split as
    r = g + b, b = r mod giant: every input with baby steps pays one ModUp,
    every baby step an inner product and a ModDown; every giant step a ModUp
    and an inner product, every output with giant steps one ModDown."""
    mu, ip, md = ks_cost(level, alpha)
    b = terms.r % giant
    g = terms.r - b
    babies = np.unique(np.stack([terms.ct[b != 0], b[b != 0]], axis=1), axis=0)
    giants = np.unique(np.stack([terms.out[g != 0], g[g != 0]], axis=1), axis=0)
    return (len(np.unique(babies[:, 0])) * mu + len(babies) * (ip + md) + len(giants) * (mu + ip)
            + len(np.unique(giants[:, 0])) * md)


# Relative cost of one plaintext product per coefficient against one modular
# product inside a key switch (measured on GB300 over ResNet-20: 0.72 us per
# MAC unit against 0.96 us per key-switch unit), for comparing schedules that
# trade key-switch work against MAC work.
MAC_WEIGHT = 0.75


def split_cost(terms: Terms, giant: int, level: int, alpha: int, hoist: int) -> float:
    """Cost, in the units of ks_cost, of a linear layer split as r = g + b
    (b = r mod giant) and evaluated with single (hoist 1) or double (hoist 2)
    hoisting, the plaintext MAC included (MAC_WEIGHT per product and
    coefficient, 1/8 of a limb transform).  Double hoisting keeps the baby
    rotations in Q_l u P: a baby step costs only its inner product, each
    output group (out, g) one ModDown, and the rotated terms' products run
    over the alpha extra limbs."""
    nl = level + 1
    mac_q = len(terms.r) * 2 * nl / 8 * MAC_WEIGHT
    if hoist == 1:
        return bsgs_cost(terms, giant, level, alpha) + mac_q
    mu, ip, md = ks_cost(level, alpha)
    b = terms.r % giant
    g = terms.r - b
    babies = np.unique(np.stack([terms.ct[b != 0], b[b != 0]], axis=1), axis=0)
    giants = np.unique(np.stack([terms.out[g != 0], g[g != 0]], axis=1), axis=0)
    rot_groups = np.unique(np.stack([terms.out[b != 0], g[b != 0]], axis=1), axis=0)
    mac = (len(terms.r) * 2 * nl + int(np.count_nonzero(b)) * 2 * alpha) / 8 * MAC_WEIGHT
    return (len(np.unique(babies[:, 0])) * mu + len(babies) * ip + len(rot_groups) * md
            + len(giants) * (mu + ip) + len(np.unique(giants[:, 0])) * md + mac)


def dh_group_bytes(terms: Terms, giant: int, level: int, alpha: int, log_n: int) -> int:
    """Device bytes per image that double hoisting holds for a step: one sum
    over Q_l u P (two polynomials) per output group with rotated terms,
    alive until the step's last chunk."""
    b = terms.r % giant
    g = terms.r - b
    n_groups = len(np.unique(np.stack([terms.out[b != 0], g[b != 0]], axis=1), axis=0)) if np.any(b) else 0
    return n_groups * 2 * (level + 1 + alpha) * (1 << log_n) * 8


def groups_of(st: Dict) -> Dict[Tuple[int, int], List]:
    """{(out ct, giant step): [(in ct, baby step, vector)]} of a linear step"""
    groups: Dict[Tuple[int, int], List] = {}
    for o, g, i, b, v in zip(st["t_out"], st["t_giant"], st["t_ct"], st["t_baby"], st["t_vid"]):
        groups.setdefault((int(o), int(g)), []).append((int(i), int(b), st["vecs"][v]))
    return groups


# The classifier (the network's last dense layer) has tiny, sparse weights
# once the pool divisor and the activation's leading coefficient are folded
# into it (about 1e-5 on a few slots), and an encoded plaintext's
# coefficients are of order Delta |w| sqrt(nonzero slots) / N: at Delta alone
# most of them would round to 0 and the weights would be attenuated.  Its
# plaintexts are encoded at Delta * 2^CLASSIFIER_EXTRA_BITS; the output keeps
# that factor in its (tracked) scale, which q_0 has room for.
CLASSIFIER_EXTRA_BITS = 6


class Planner:
    def __init__(self, primes_q: Sequence[int], log_n: int, log_scale: float, layout: str, alpha: int = 3,
                 max_giant_blocks: int = 8, members: int = 1, input_lambda: int = 1,
                 giants: Optional[Sequence[int]] = None, on_demand: bool = False, hoist="auto",
                 hoists: Optional[Sequence[int]] = None, dh_bytes: int = 1 << 30):
        self.on_demand = on_demand
        self.log_n = log_n
        self.dh_bytes = dh_bytes
        self.giants = None if giants is None else list(giants)
        if hoist not in ("auto", 1, 2):
            raise ValueError("hoist must be 'auto', 1 or 2")
        self.hoist = hoist
        self.hoists = None if hoists is None else list(hoists)
        self.n_linear = 0
        self.members = members
        self.input_lambda = input_lambda
        self.alpha = alpha
        self.max_giant_blocks = max_giant_blocks
        self.q = list(primes_q)
        self.L = len(self.q) - 1
        self.n = 1 << (log_n - 1)
        self.delta = 2.0 ** log_scale
        self.logd = math.log2(self.delta)
        self.layout = layout
        self.p = Program()

    # ---- bookkeeping
    def _t(self, layout, level, scale) -> int:
        self.p.tensors.append(TInfo(layout, level, scale))
        return len(self.p.tensors) - 1

    def _emit(self, **st) -> int:
        self.p.steps.append(st)
        return st["dst"]

    def _rule(self, t: int) -> int:
        """tower reuse: rescale when lambda(x) > lambda(q_level)"""
        info = self.p.tensors[t]
        ql = self.q[info.level]
        if info.level >= 1 and _lam(info.scale, self.logd) > _lam(ql, self.logd):
            return self._emit(kind=F.STEP_RESCALE, src=t, dst=self._t(info.layout, info.level - 1, info.scale / ql))
        return t

    def _hoist_options(self, terms: Optional[Terms] = None, giant: int = 0, level: int = 0) -> Tuple[int, ...]:
        """the admitted modes; "auto" admits double hoisting only while its
        group sums fit dh_bytes per image"""
        if self.hoist != "auto":
            return (self.hoist,)
        if terms is not None and dh_group_bytes(terms, giant, level, self.alpha, self.log_n) > self.dh_bytes:
            return (1,)
        return (1, 2)

    def _pick_giant(self, terms: Terms, block: int, level: int) -> int:
        """giant step = k blocks, k in 1, 2, 4, .. max_giant_blocks: the
        cheapest split by split_cost over the admitted hoisting modes (ties:
        the smaller k, then single hoisting)"""
        best = None
        k = 1
        while k <= self.max_giant_blocks and k * block <= self.n:
            for h in self._hoist_options(terms, k * block, level):
                c = split_cost(terms, k * block, level, self.alpha, h)
                if best is None or c < best[0]:
                    best = (c, k * block)
            k *= 2
        return best[1]

    def _pick_hoist(self, terms: Terms, giant: int, level: int) -> int:
        if self.hoists is not None:
            return int(self.hoists[self.n_linear])
        opts = self._hoist_options(terms, giant, level)
        costs = [split_cost(terms, giant, level, self.alpha, h) for h in opts]
        return opts[int(np.argmin(costs))]

    def _bias_vecs(self, biases: Sequence[np.ndarray], layout: SlotMap) -> Dict[int, np.ndarray]:
        """bias of channel ch, replica k (the member biases[k]), on the
        channel's positions"""
        out: Dict[int, np.ndarray] = {}
        offs = layout.offsets()
        for ch in range(len(layout.copies)):
            for k, (ct, base) in enumerate(layout.copies[ch]):
                out.setdefault(ct, np.zeros(self.n))[base + offs] = biases[min(k, len(biases) - 1)][ch]
        return out

    def _bsgs_step(self, src: int, terms: Terms, giant: int, dst_layout: SlotMap, w_scale: float,
                   bias_vecs: Dict[int, np.ndarray]) -> int:
        info = self.p.tensors[src]
        if self.giants is not None:
            giant = self.giants[self.n_linear]
        hoist = self._pick_hoist(terms, giant, info.level) if len(terms.r) else 1
        self.n_linear += 1
        prod = info.scale * w_scale
        dst = self._t(dst_layout, info.level, prod)
        b = terms.r % giant
        g = terms.r - b
        # each term's vector is pre-rotated by -g; equal results share an entry
        pairs, inv = np.unique(np.stack([terms.vid, g], axis=1), axis=0, return_inverse=True)
        table: Dict[bytes, int] = {}
        vecs: List[np.ndarray] = []
        remap = np.empty(len(pairs), dtype=np.int64)
        for j, (v, gg) in enumerate(pairs):
            vec = terms.vecs[v]
            if isinstance(vec, SparseVec):
                rolled = vec.roll(int(gg), self.n) if gg else vec
                key = rolled.key()
            else:
                rolled = np.roll(vec, gg) if gg else vec
                key = rolled.tobytes()
            if key not in table:
                table[key] = len(vecs)
                vecs.append(rolled)
            remap[j] = table[key]
        vid = remap[inv.reshape(-1)]
        order = np.lexsort((b, terms.ct, g, terms.out))
        self.p.rotations.update(int(x) for x in np.unique(b) if x)
        self.p.rotations.update(int(x) for x in np.unique(g) if x)
        return self._emit(kind=F.STEP_LINEAR, src=src, dst=dst, w_scale=w_scale, bias_scale=prod,
                          t_out=terms.out[order], t_giant=g[order], t_ct=terms.ct[order], t_baby=b[order],
                          t_vid=vid[order], vecs=vecs, bias=bias_vecs, giant=giant, hoist=hoist)

    def _shortcut_scale(self, info: TInfo, target: TInfo) -> float:
        ql = self.q[info.level]
        ws = target.scale * ql / info.scale
        if info.level >= 1 and _lam(info.scale * ws, self.logd) > _lam(ql, self.logd):
            return ws
        return target.scale / info.scale

    def _land_on(self, t: int, target: TInfo) -> int:
        info = self.p.tensors[t]
        if info.level < target.level:
            raise ValueError("shortcut arrives below the main branch's level")
        if info.level > target.level:
            return self._emit(kind=F.STEP_DROP, src=t, level=target.level,
                              dst=self._t(info.layout, target.level, target.scale))
        info.scale = target.scale
        return t

    # ---- layers (ps: the layer's parameters of every ensemble member)
    def conv(self, src: int, node: Dict, ps: List[Dict], target: Optional[TInfo] = None) -> int:
        info = self.p.tensors[src]
        lin = info.layout
        ho = (lin.H + 2 * node["pad"] - node["k"]) // node["stride"] + 1
        wo = (lin.W + 2 * node["pad"] - node["k"]) // node["stride"] + 1
        st = lin.st * node["stride"]
        if self.layout in ("hw", "hw_ens"):
            lout = SlotMap(node["cout"], [[(o, base) for (_, base) in lin.copies[0]] for o in range(node["cout"])],
                           ho, wo, st, lin.row, lin.block)
            reps = len(lin.copies[0])
            ws = [ps[k if self.layout == "hw_ens" else 0]["w"] for k in range(reps)]
            terms = diagonals_hw(ws, node["stride"], node["pad"], lin, lout, self.n)
            giant = self.n
            bias = self._bias_vecs([ps[k if self.layout == "hw_ens" else 0]["bias"] for k in range(reps)], lout)
        else:
            lout = map_packed(node["cout"], ho, wo, st, lin.row, lin.block, self.n)
            terms = terms_of(diagonals(ps[0]["w"], node["stride"], node["pad"], lin, lout, self.n,
                                       sparse=self.on_demand))
            giant = self._pick_giant(terms, lin.block, info.level)
            bias = self._bias_vecs([ps[0]["bias"]], lout)
        ws_scale = self.delta if target is None else self._shortcut_scale(info, target)
        t = self._bsgs_step(src, terms, giant, lout, ws_scale, bias)
        t = self._rule(t)
        return t if target is None else self._land_on(t, target)

    def act(self, src: int, ps: List[Dict]) -> int:
        prm = ps[0]
        if any(np.any(p["c1"] != prm["c1"]) or np.any(p["c0"] != prm["c0"]) for p in ps):
            raise ValueError("ensemble members must share the activation polynomial")
        info = self.p.tensors[src]
        s = info.scale
        s2 = s * s
        dst = self._t(info.layout, info.level, s2)
        if np.ndim(prm["c1"]):
            # per-channel coefficients (Case 1): slot vectors, c1 encoded at
            # scale s (so c1 (.) x is at s*s) and c0 at s*s
            self._emit(kind=F.STEP_ACT, src=src, dst=dst, c1=0.0, c0=0.0,
                       c1_vecs=self._channel_vecs(info.layout, prm["c1"]),
                       c0_vecs=self._channel_vecs(info.layout, prm["c0"]), c1_scale=s, c0_scale=s2)
        else:
            self._emit(kind=F.STEP_ACT, src=src, dst=dst, c1=_round_int(prm["c1"] * s),
                       c0=_round_int(prm["c0"] * s2))
        return self._rule(dst)

    def _channel_vecs(self, layout: SlotMap, values: np.ndarray) -> List[np.ndarray]:
        """one slot vector per ciphertext with values[c] at every position of
        every copy of channel c"""
        vecs = [np.zeros(self.n) for _ in range(layout.n_ct)]
        offs = layout.offsets()
        for ch, copies in enumerate(layout.copies):
            for ct, base in copies:
                vecs[ct][base + offs] = values[ch]
        return vecs

    def pool(self, src: int, k: int) -> int:
        info = self.p.tensors[src]
        L = info.layout
        lg = int(math.log2(k))
        steps = [L.st << m for m in range(lg)] + [(L.st * L.row) << m for m in range(lg)]
        lp = SlotMap(L.n_ct, L.copies, L.H // k, L.W // k, L.st * k, L.row, L.block)
        self.p.rotations.update(steps)
        return self._emit(kind=F.STEP_ROTSUM, src=src, dst=self._t(lp, info.level, info.scale), steps=steps)

    def shortcut_identity(self, src: int, ps: List[Dict], target: TInfo) -> int:
        value = ps[0]["shortcut"]
        if any(p["shortcut"] != value for p in ps):
            raise ValueError("ensemble members must share the shortcut multiplier")
        info = self.p.tensors[src]
        ws = self._shortcut_scale(info, target)
        dst = self._t(info.layout, info.level, info.scale * ws)
        self._emit(kind=F.STEP_CMUL, src=src, dst=dst, value=_round_int(value * ws))
        return self._land_on(self._rule(dst), target)

    def add(self, a: int, b: int) -> int:
        ia = self.p.tensors[a]
        return self._emit(kind=F.STEP_ADD, src=a, src2=b, dst=self._t(ia.layout, ia.level, ia.scale))

    def dense(self, src: int, node: Dict, ps: List[Dict], last: bool = False) -> int:
        info = self.p.tensors[src]
        lin = info.layout
        cout = node["cout"]
        wsc = self.delta * (2.0 ** CLASSIFIER_EXTRA_BITS if last else 1.0)
        if self.layout == "hw":
            # products in block k of ciphertext 0, then a sum over the block
            w = ps[0]["w"]
            offs = lin.offsets()
            diag = {}
            for c in range(len(lin.copies)):
                vec = diag.setdefault((0, lin.copies[c][0][0], 0), np.zeros(self.n))
                for k in range(cout):
                    ct, base = _pick_copy(lin.copies[c], k * lin.block, self.n)
                    vec[base + offs] = w[k, c * len(offs):(c + 1) * len(offs)]
            part = SlotMap(1, [[(0, k * lin.block)] for k in range(cout)], 1, 1, 1, 1, lin.block)
            t = self._bsgs_step(src, terms_of(diag), self.n, part, wsc, self._bias_vecs([ps[0]["bias"]], part))
            t = self._rule(t)
            ti = self.p.tensors[t]
            steps = [lin.st << m for m in range(int(math.log2(lin.W)))] + \
                    [(lin.st * lin.row) << m for m in range(int(math.log2(lin.H)))]
            self.p.rotations.update(steps)
            return self._emit(kind=F.STEP_ROTSUM, src=t, steps=steps,
                              dst=self._t(map_single(cout, lin.block, self.n), ti.level, ti.scale))
        if self.layout == "hw_ens":
            return self._dense_ensemble(src, node, ps, wsc)
        lout = map_single(cout, lin.block, self.n)
        terms = terms_of(diagonals(ps[0]["w"].reshape(cout, -1, 1, 1), 1, 0, lin, lout, self.n))
        t = self._bsgs_step(src, terms, 8 * lin.block, lout, wsc, self._bias_vecs([ps[0]["bias"]], lout))
        return self._rule(t)

    def _dense_ensemble(self, src: int, node: Dict, ps: List[Dict], wsc: float) -> int:
        """Dense layer of an ensemble in the HW layout, then the ensemble
        average (Sec. 5.3).  Input channel c (ciphertext c) holds member m's
        pooled feature at slot m*B; output k of member m goes to slot
        m*B + k, read at rotation r = -k, with weight w_m[k, c] / M; giant
        steps only (each partial sum sum_c d_(c,g) (.) in_c is rotated once).
        Then the M blocks are summed by rotations of B, 2B, 4B, .. (before
        the rescale): the averaged logit k ends in slot k of block 0."""
        info = self.p.tensors[src]
        lin = info.layout
        cout, M, B = node["cout"], self.members, lin.block
        if lin.H != 1 or lin.W != 1 or cout > B:
            raise ValueError("ensemble dense layer: expects one pooled feature per channel and cout <= block")
        cin = len(lin.copies)
        ws = [p["w"] / float(M) for p in ps]
        o_idx = np.zeros(cout * cin, dtype=np.int64)
        k_idx, c_idx = np.meshgrid(np.arange(cout), np.arange(cin), indexing="ij")
        k_idx, c_idx = k_idx.reshape(-1), c_idx.reshape(-1)
        tup = np.stack([w.reshape(cout, cin).reshape(-1) for w in ws], axis=1)
        # one vector per (member weights, k): values at slots m*B + k
        key = np.concatenate([tup, k_idx[:, None].astype(np.float64)], axis=1)
        uniq, inv = np.unique(key, axis=0, return_inverse=True)
        vecs = []
        for u in uniq:
            v = np.zeros(self.n)
            kk = int(u[-1])
            for m in range(M):
                v[m * B + kk] = u[m]
            vecs.append(v)
        terms = Terms(o_idx, c_idx, (-k_idx) % self.n, inv.reshape(-1), vecs)
        part = SlotMap(1, [[(0, m * B + k) for m in range(M)] for k in range(cout)], 1, 1, 1, 1, B)
        bias = self._bias_vecs([p["bias"] / float(M) for p in ps], part)
        t = self._bsgs_step(src, terms, 1, part, wsc, bias)
        # the block sum runs before the rescale, on the product at the
        # larger scale, where the rotations' noise is negligible
        ti = self.p.tensors[t]
        steps = [B << j for j in range(max(0, (M - 1).bit_length()))]
        self.p.rotations.update(steps)
        t = self._emit(kind=F.STEP_ROTSUM, src=t, steps=steps,
                       dst=self._t(SlotMap(1, [[(0, k)] for k in range(cout)], 1, 1, 1, 1, B), ti.level, ti.scale))
        return self._rule(t)

    def compile(self, net: List[Dict], prms: List[Dict]) -> Program:
        node_t: Dict[int, int] = {}
        later = {n["src"][1] for n in net if n["op"] == "add" and net[n["src"][1]]["op"] == "conv"}
        for idx, node in enumerate(net):
            kind = node["op"]
            ps = [p.get(idx) for p in prms]
            if kind == "input":
                if self.layout == "hw":
                    lay = map_hw(node["c"], node["h"], node["w"], self.n)
                elif self.layout == "hw_ens":
                    lay = map_hw_ensemble(node["c"], node["h"], node["w"], self.n, self.members)
                else:
                    lay = map_packed(node["c"], node["h"], node["w"], 1, node["w"], node["h"] * node["w"], self.n)
                node_t[idx] = self.p.input = self._t(lay, self.L, self.delta ** self.input_lambda)
            elif kind == "conv":
                if idx not in later:
                    node_t[idx] = self.conv(node_t[node["src"]], node, ps)
            elif kind == "bn":
                node_t[idx] = node_t[node["src"]]     # fused into the activation that follows
            elif kind == "act":
                node_t[idx] = self.act(node_t[node["src"]], ps)
            elif kind == "pool":
                node_t[idx] = self.pool(node_t[node["src"]], node["k"])
            elif kind == "add":
                a, b = node["src"]
                main = self.p.tensors[node_t[a]]
                if net[b]["op"] == "conv":
                    sc = self.conv(node_t[net[b]["src"]], net[b], [p[b] for p in prms], target=main)
                else:
                    sc = self.shortcut_identity(node_t[b], ps, main)
                node_t[idx] = self.add(node_t[a], sc)
            elif kind == "dense":
                node_t[idx] = self.dense(node_t[node["src"]], node, ps, last=idx == len(net) - 1)
        self.p.output = node_t[len(net) - 1]
        return self.p


def compile_network(net, raw, primes_q, log_n, log_scale, layout, alpha: int = 3,
                    max_giant_blocks: int = 8, input_lambda: int = 1,
                    giants: Optional[Sequence[int]] = None, on_demand: bool = False, hoist="auto",
                    hoists: Optional[Sequence[int]] = None, dh_bytes: int = 1 << 30) -> Program:
    """raw: one model's raw parameters, or a list of them (an ensemble, laid
    out with layout "hw_ens": member m in block m of every ciphertext).
    alpha: digit width of key switching (for the baby-step / giant-step
    cost model); max_giant_blocks = 1 keeps the giant step at one block.
    input_lambda: the client encodes the image at scale Delta^input_lambda
    (the program's input tensor scale; 2 keeps every key switch of the
    first layer at scale Delta^2).  giants: the giant-step size of every
    linear step in program order, in place of the planner's choice (any
    split evaluates the same diagonals).  on_demand: the weight vectors of
    the packed convolutions are kept sparse and encoded on the device each
    time their step runs, instead of being encoded once and held in HBM
    (for layers whose plaintexts do not fit).  hoist: 1 (every baby-step
    rotation brought back to Q_l by its own ModDown), 2 (double hoisting:
    rotations kept in Q_l u P, one ModDown per output group) or "auto" (per
    linear step, the cheaper by split_cost, double hoisting admitted only
    where its group sums over Q_l u P take at most dh_bytes per image);
    hoists: one mode per linear step in place of that choice."""
    raws = raw if isinstance(raw, (list, tuple)) else [raw]
    if len(raws) > 1 and layout != "hw_ens":
        raise ValueError("an ensemble needs the hw_ens layout")
    prms = [prepare_params(net, r) for r in raws]
    return Planner(primes_q, log_n, log_scale, layout, alpha, max_giant_blocks, len(raws),
                   input_lambda, giants, on_demand, hoist, hoists, dh_bytes).compile(net, prms)


def input_scale(prog: Program) -> float:
    """the scale at which the client encodes the program's input"""
    return prog.tensors[prog.input].scale


def giant_steps(prog: Program) -> List[int]:
    """the giant-step size of every linear step, in program order"""
    return [st["giant"] for st in prog.steps if st["kind"] == F.STEP_LINEAR]


def hoists(prog: Program) -> List[int]:
    """the hoisting mode (1 single, 2 double) of every linear step, in
    program order"""
    return [int(st.get("hoist", 1)) for st in prog.steps if st["kind"] == F.STEP_LINEAR]


def keyswitches_of_step(prog: Program, st: dict) -> int:
    """Hybrid key switches one image's step performs, all at the level of its
    source: the distinct baby rotations (input ciphertext, step) and giant
    rotations (output, step) of a linear step, one relinearisation per
    ciphertext of an activation, one rotation per ciphertext and step of a
    rotate-and-sum."""
    t_in = prog.tensors[st["src"]]
    if st["kind"] == F.STEP_LINEAR:
        babies = {(i, b) for i, b in zip(st["t_ct"], st["t_baby"]) if b}
        giants = {(o, g) for o, g in zip(st["t_out"], st["t_giant"]) if g}
        return len(babies) + len(giants)
    if st["kind"] == F.STEP_ACT:
        return t_in.layout.n_ct
    if st["kind"] == F.STEP_ROTSUM:
        return t_in.layout.n_ct * len(st["steps"])
    return 0


def keyswitch_census(prog: Program) -> Dict[int, int]:
    """level -> number of hybrid key switches one image performs there"""
    out: Dict[int, int] = {}
    for st in prog.steps:
        k = keyswitches_of_step(prog, st)
        if k:
            lv = prog.tensors[st["src"]].level
            out[lv] = out.get(lv, 0) + k
    return out


# =========================================================== to the C ABI

class ModelDesc:
    """Owns the arrays behind an FheModelDesc."""

    def __init__(self, prog: Program, n_slots: int):
        keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(np.asarray(x, dtype=dt))
            keep.append(a)
            return a

        def p32(a):
            return a.ctypes.data_as(F.P_I32)

        def pd(a):
            return a.ctypes.data_as(F.P_DBL)

        T = prog.tensors
        n_ct = arr([t.layout.n_ct for t in T], np.int32)
        lev = arr([t.level for t in T], np.int32)
        sc = arr([t.scale for t in T], np.float64)
        steps = (F.FheStepDesc * max(len(prog.steps), 1))()
        for i, st in enumerate(prog.steps):
            d = steps[i]
            d.kind = st["kind"]
            d.src = st["src"]
            d.src2 = st.get("src2", -1)
            d.dst = st["dst"]
            if st["kind"] == F.STEP_LINEAR:
                t_out, t_g = st["t_out"], st["t_giant"]
                n_t = len(t_out)
                if n_t:
                    cut = np.flatnonzero((t_out[1:] != t_out[:-1]) | (t_g[1:] != t_g[:-1])) + 1
                    starts = np.concatenate([[0], cut])
                else:
                    starts = np.zeros(0, dtype=np.int64)
                d.w_scale = st["w_scale"]
                d.bias_scale = st["bias_scale"]
                d.double_hoist = 1 if st.get("hoist", 1) == 2 else 0
                d.n_groups = len(starts)
                d.group_out = p32(arr(t_out[starts] if n_t else [0], np.int32))
                d.group_giant = p32(arr(t_g[starts] if n_t else [0], np.int32))
                d.group_term_begin = p32(arr(np.concatenate([starts, [n_t]]), np.int32))
                d.term_ct = p32(arr(st["t_ct"] if n_t else [0], np.int32))
                d.term_baby = p32(arr(st["t_baby"] if n_t else [0], np.int32))
                d.term_vec_id = p32(arr(st["t_vid"] if n_t else [0], np.int32))
                d.n_vecs = len(st["vecs"])
                if st["vecs"] and isinstance(st["vecs"][0], SparseVec):
                    # encoded on the device when the step runs
                    lens = np.array([len(v) for v in st["vecs"]], dtype=np.int64)
                    d.vecs = None
                    d.sparse_vec_begin = arr(np.concatenate([[0], np.cumsum(lens)]), np.int64).ctypes.data_as(
                        F.P_I64)
                    d.sparse_slot = p32(arr(np.concatenate([v.slots for v in st["vecs"]]), np.int32))
                    d.sparse_val = pd(arr(np.concatenate([v.vals for v in st["vecs"]]), np.float64))
                else:
                    d.vecs = pd(arr(np.stack(st["vecs"]) if st["vecs"] else np.zeros((1, n_slots)), np.float64))
                bo = sorted(st["bias"])
                d.n_bias = len(bo)
                d.bias_out = p32(arr(bo or [0], np.int32))
                d.bias_vec = pd(arr(np.stack([st["bias"][o] for o in bo]) if bo else np.zeros((1, n_slots)),
                                    np.float64))
            elif st["kind"] == F.STEP_ACT:
                d.c1 = st["c1"]
                d.c0 = st["c0"]
                if "c1_vecs" in st:
                    d.act_c1_vecs = pd(arr(np.stack(st["c1_vecs"]), np.float64))
                    d.act_c0_vecs = pd(arr(np.stack(st["c0_vecs"]), np.float64))
                    d.act_c1_scale = st["c1_scale"]
                    d.act_c0_scale = st["c0_scale"]
            elif st["kind"] == F.STEP_CMUL:
                d.value = st["value"]
            elif st["kind"] == F.STEP_ROTSUM:
                d.n_steps = len(st["steps"])
                d.steps = p32(arr(st["steps"], np.int32))
            elif st["kind"] == F.STEP_DROP:
                d.level = st["level"]
        self.desc = F.FheModelDesc(len(T), p32(n_ct), p32(lev), pd(sc), prog.input, prog.output, len(prog.steps),
                                   steps)
        self._keep = keep
        self._steps = steps
        # the struct holds raw pointers into these arrays: it keeps its owner
        # alive, so `ModelDesc(...).desc` may be passed on by itself
        self.desc._owner = self


def input_slots(prog: Program, img: np.ndarray, n_slots: int) -> List[np.ndarray]:
    """The client's slot vectors of an image in the program's input layout."""
    lay = prog.tensors[prog.input].layout
    offs = lay.offsets()
    out = [np.zeros(n_slots) for _ in range(lay.n_ct)]
    for c, copies in enumerate(lay.copies):
        flat = img[c].reshape(-1)
        for ct, base in copies:
            out[ct][base + offs] = flat
    return out


def logit_slots(prog: Program) -> List[Tuple[int, int]]:
    lay = prog.tensors[prog.output].layout
    return [cp[0] for cp in lay.copies]
