"""Quadratic-activation CNNs in float64 and under CKKS (test infrastructure only).

Three pieces, each written as plainly as possible:

1. ``forward_plain``: the network with its original parameters (batch norm
   gamma*(x-mu)/sigma + beta, activation a*x^2 + b*x + c, average pooling).
2. ``transform``: the structural optimisations that keep the function --
   node fusing Case 2 (batch norm folded into the preceding convolution,
   Sec. 4.1: omega = b1*w, alpha = b1*beta_c + b0, b1 = gamma/sigma,
   b0 = beta - b1*mu) and forward weight redistribution (Sec. 4.2: the
   activation becomes monic x^2 + (b/a) x + c/a with update upsilon = a, the
   average pool becomes a plain sum with upsilon = 1/k^2, and each receiver
   kernel multiplies its weights by the incoming upsilon; an identity shortcut
   carrying upsilon is multiplied by it).  ``forward_transformed`` evaluates
   the transformed network in float64.
3. ``compile_he`` / ``run_he``: the homomorphic evaluation.  Slot layouts
   follow Sec. 5.1: the HW layout (one channel per ciphertext, spatial values
   in the slots, replicated into every free block) or a channel-packed layout
   (the CHW alternative: one block of slots per channel).  Strided operations
   leave gaps that later layers follow (adaptive / lazy mapping).  A linear
   layer is written as sum over diagonals: out = sum_r d_r (.) rot(in, r),
   split into baby steps b = r mod G (rotations of the input) and giant steps
   g = r - b (rotations of partial sums), with d_r pre-rotated by -g.  The
   baby-step rotations of one input share one ModUp and the giant-step
   rotations of one output share one ModDown (``rotate_hoisted`` and
   ``rotate_sum_lazy`` in ckks.py).  Rescales follow the tower-reuse rule of
   Sec. 4.3.

Floating-point expressions that feed integers (weights after folding, the
scales of encoded plaintexts and constants) are written out once here, in a
fixed operation order; see the comments at each.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import ckks as C


# =================================================================== float64

def conv2d(x: np.ndarray, w: np.ndarray, stride: int, pad: int) -> np.ndarray:
    """Cross-correlation as in deep-learning convolutions: x [cin,H,W],
    w [cout,cin,k,k] -> [cout, Ho, Wo]."""
    cin, H, W = x.shape
    cout, _, k, _ = w.shape
    xp = np.zeros((cin, H + 2 * pad, W + 2 * pad))
    xp[:, pad:pad + H, pad:pad + W] = x
    Ho = (H + 2 * pad - k) // stride + 1
    Wo = (W + 2 * pad - k) // stride + 1
    out = np.zeros((cout, Ho, Wo))
    for dh in range(k):
        for dw in range(k):
            patch = xp[:, dh:dh + stride * (Ho - 1) + 1:stride, dw:dw + stride * (Wo - 1) + 1:stride]
            out += np.einsum("oi,ihw->ohw", w[:, :, dh, dw], patch)
    return out


def avgpool(x: np.ndarray, k: int) -> np.ndarray:
    c, H, W = x.shape
    return x.reshape(c, H // k, k, W // k, k).mean(axis=(2, 4))


def forward_plain(net: List[Dict], raw: Dict, img: np.ndarray) -> np.ndarray:
    vals: Dict[int, np.ndarray] = {}
    for i, nd in enumerate(net):
        op = nd["op"]
        if op == "input":
            vals[i] = img
        elif op == "conv":
            p = raw[i]
            y = conv2d(vals[nd["src"]], p["w"], nd["stride"], nd["pad"]) + p["bias"][:, None, None]
            y = p["gamma"][:, None, None] * (y - p["mu"][:, None, None]) / p["sigma"][:, None, None] \
                + p["beta"][:, None, None]
            vals[i] = y
        elif op == "bn":
            p = raw[i]
            x = vals[nd["src"]]
            vals[i] = p["gamma"][:, None, None] * (x - p["mu"][:, None, None]) / p["sigma"][:, None, None] \
                + p["beta"][:, None, None]
        elif op == "act":
            p = raw[i]
            x = vals[nd["src"]]
            vals[i] = p["a"] * x * x + p["b"] * x + p["c"]
        elif op == "pool":
            vals[i] = avgpool(vals[nd["src"]], nd["k"])
        elif op == "add":
            vals[i] = vals[nd["src"][0]] + vals[nd["src"][1]]
        elif op == "dense":
            p = raw[i]
            vals[i] = p["w"] @ vals[nd["src"]].reshape(-1) + p["bias"]
    return vals[len(net) - 1]


# ------------------------------------------------------------ node fusing
# Sec. 4.1, with batch norm written B(x) = b1 x + b0 (b1 = gamma / sigma,
# b0 = beta - b1 mu) and the activation P(x) = c2 x^2 + c1 x + c0.

def bn_linear(p: Dict) -> Tuple[np.ndarray, np.ndarray]:
    """(b1, b0) of a batch norm"""
    b1 = p["gamma"] / p["sigma"]
    return b1, p["beta"] - b1 * p["mu"]


def fuse_bn_act(b1, b0, c2, c1, c0):
    """Case 1, P(B(x)) = p2 x^2 + p1 x + p0 (the appendix's derivation):
    p2 = b1^2 c2, p1 = b1 (2 b0 c2 + c1), p0 = b0^2 c2 + b0 c1 + c0."""
    return b1 * b1 * c2, b1 * (2.0 * b0 * c2 + c1), b0 * b0 * c2 + b0 * c1 + c0


def fuse_bn_bn_add_act(bx1, bx0, by1, by0, c2, c1, c0):
    """Case 3, P(B_X(x) + B_Y(y)) = S(x, y) = dx2 x^2 + dy2 y^2 + dxy x y +
    dx x + dy y + d0, with s = bx0 + by0: dx2 = c2 bx1^2, dy2 = c2 by1^2,
    dxy = 2 c2 bx1 by1, dx = bx1 (2 c2 s + c1), dy = by1 (2 c2 s + c1),
    d0 = c2 s^2 + c1 s + c0.  Returns (dx2, dy2, dxy, dx, dy, d0)."""
    s = bx0 + by0
    return (c2 * bx1 * bx1, c2 * by1 * by1, 2.0 * c2 * bx1 * by1, bx1 * (2.0 * c2 * s + c1),
            by1 * (2.0 * c2 * s + c1), c2 * s * s + c1 * s + c0)


def fuse_bn_add_act(bx1, bx0, c2, c1, c0):
    """Case 4 (identity shortcut), P(B_X(x) + y) = S(x, y): dx2 = c2 bx1^2,
    dy2 = c2, dxy = 2 c2 bx1, dx = bx1 (2 c2 bx0 + c1), dy = 2 c2 bx0 + c1,
    d0 = c2 bx0^2 + c1 bx0 + c0.  Returns (dx2, dy2, dxy, dx, dy, d0)."""
    return (c2 * bx1 * bx1, c2 * np.ones_like(bx1), 2.0 * c2 * bx1, bx1 * (2.0 * c2 * bx0 + c1),
            2.0 * c2 * bx0 + c1, c2 * bx0 * bx0 + c1 * bx0 + c0)


def _scale_in(u, w: np.ndarray) -> np.ndarray:
    """multiply the input channels of weights w [cout, cin, ...] by u (a
    scalar or one value per input channel)"""
    if np.ndim(u) == 0:
        return w * u
    return w * np.reshape(u, (1, -1) + (1,) * (w.ndim - 2))


def transform(net: List[Dict], raw: Dict) -> Dict:
    """Folded and redistributed parameters.  Operation order (fixed):
    b1 = gamma / sigma; b0 = beta - b1 * mu; omega = (w * b1[o]) * u_in;
    alpha = bias * b1 + b0; act: c1 = b / a, c0 = c / a, u = a;
    pool: u = u_in / float(k*k); dense: w = w * u_in; identity shortcut:
    multiply by u of the shortcut's source.  A batch norm that is a node of
    its own (not after a convolution) must feed an activation: the two fuse
    (Case 1, with b1 taken times the u of the batch norm's input) into
    p2 x^2 + p1 x + p0 per channel, made monic: c1 = p1 / p2, c0 = p0 / p2,
    u = p2 (one value per channel, taken up by the next convolution's or
    dense layer's input channels)."""
    t: Dict = {}
    ups: Dict[int, float] = {}
    for i, nd in enumerate(net):
        op = nd["op"]
        if op == "input":
            ups[i] = 1.0
        elif op == "conv":
            p = raw[i]
            b1 = p["gamma"] / p["sigma"]
            b0 = p["beta"] - b1 * p["mu"]
            omega = _scale_in(ups[nd["src"]], p["w"] * b1[:, None, None, None])
            alpha = p["bias"] * b1 + b0
            t[i] = {"w": omega, "bias": alpha}
            ups[i] = 1.0
        elif op == "bn":
            users = [j for j, m in enumerate(net) if m.get("src") == i or (isinstance(m.get("src"), list)
                                                                            and i in m["src"])]
            if [net[j]["op"] for j in users] != ["act"]:
                raise ValueError("a batch norm of its own must feed one activation (node fusing Case 1)")
            t[i] = {"fused_into": users[0]}
            ups[i] = None
        elif op == "act" and net[nd["src"]]["op"] == "bn":
            # Case 1 on the batch norm's computed input x' = x / u: B(x) =
            # (b1 u) x' + b0
            p = raw[i]
            bn_node = net[nd["src"]]
            b1, b0 = bn_linear(raw[nd["src"]])
            p2, p1, p0 = fuse_bn_act(b1 * ups[bn_node["src"]], b0, p["a"], p["b"], p["c"])
            t[i] = {"c1": p1 / p2, "c0": p0 / p2}
            ups[i] = p2
        elif op == "act":
            p = raw[i]
            t[i] = {"c1": p["b"] / p["a"], "c0": p["c"] / p["a"]}
            ups[i] = p["a"]
        elif op == "pool":
            ups[i] = ups[nd["src"]] / float(nd["k"] * nd["k"])
        elif op == "dense":
            p = raw[i]
            u = ups[nd["src"]]
            if np.ndim(u) != 0:
                u = np.repeat(u, p["w"].shape[1] // len(u))   # inputs are channel-major
            t[i] = {"w": p["w"] * u, "bias": p["bias"]}
            ups[i] = 1.0
        elif op == "add":
            a, b = nd["src"]
            # the main branch is a convolution (upsilon 1); an identity
            # shortcut from an activation carries that activation's upsilon
            if net[b]["op"] != "conv" and np.ndim(ups[b]) != 0:
                raise ValueError("an identity shortcut needs one upsilon for all channels")
            t[i] = {"shortcut_const": ups[b] if net[b]["op"] != "conv" else None}
            ups[i] = 1.0
    return t


def forward_transformed(net: List[Dict], t: Dict, img: np.ndarray) -> np.ndarray:
    vals: Dict[int, np.ndarray] = {}
    for i, nd in enumerate(net):
        op = nd["op"]
        if op == "input":
            vals[i] = img
        elif op == "conv":
            vals[i] = conv2d(vals[nd["src"]], t[i]["w"], nd["stride"], nd["pad"]) \
                + t[i]["bias"][:, None, None]
        elif op == "bn":
            vals[i] = vals[nd["src"]]          # fused into the activation that follows
        elif op == "act":
            x = vals[nd["src"]]
            c1, c0 = t[i]["c1"], t[i]["c0"]
            if np.ndim(c1):
                c1, c0 = c1[:, None, None], c0[:, None, None]
            vals[i] = x * x + c1 * x + c0
        elif op == "pool":
            c, H, W = vals[nd["src"]].shape
            k = nd["k"]
            vals[i] = vals[nd["src"]].reshape(c, H // k, k, W // k, k).sum(axis=(2, 4))
        elif op == "add":
            a, b = nd["src"]
            sc = vals[b]
            if t[i]["shortcut_const"] is not None:
                sc = sc * t[i]["shortcut_const"]
            vals[i] = vals[a] + sc
        elif op == "dense":
            vals[i] = t[i]["w"] @ vals[nd["src"]].reshape(-1) + t[i]["bias"]
    return vals[len(net) - 1]


# =================================================================== layouts

@dataclass
class Layout:
    """Where each channel's logical (h, w) values sit: channel c has replicas
    rep[c] = [(ciphertext index, base slot)], and value (h, w) of a replica is
    at slot base + (h*st)*Wp + w*st."""
    n_ct: int
    rep: List[List[Tuple[int, int]]]
    H: int
    W: int
    st: int
    Wp: int
    B: int          # slots per block

    def slot(self, base: int, h: int, w: int) -> int:
        return base + (h * self.st) * self.Wp + w * self.st


def hw_layout(c: int, H: int, W: int, n_slots: int) -> Layout:
    """HW layout: channel c alone in ciphertext c, replicated into every
    block of H*W slots."""
    B = H * W
    rep = [[(ch, b * B) for b in range(n_slots // B)] for ch in range(c)]
    return Layout(c, rep, H, W, 1, W, B)


def packed_layout(c: int, H: int, W: int, st: int, Wp: int, B: int, n_slots: int) -> Layout:
    """Channel-packed: one block of B slots per channel.  With c <= blocks per
    ciphertext, a single ciphertext holds channel (b mod c) in block b for
    every b < c*floor(blocks/c); otherwise channel ch sits in ciphertext
    ch // blocks, block ch mod blocks."""
    nb = n_slots // B
    if c <= nb:
        rep = [[(0, b * B) for b in range(c * (nb // c)) if b % c == ch] for ch in range(c)]
        return Layout(1, rep, H, W, st, Wp, B)
    assert c % nb == 0
    rep = [[(ch // nb, (ch % nb) * B)] for ch in range(c)]
    return Layout(c // nb, rep, H, W, st, Wp, B)


def hw_ensemble_layout(c: int, H: int, W: int, n_slots: int, members: int) -> Layout:
    """HW layout shared by an ensemble of `members` networks (Sec. 5.3):
    channel c alone in ciphertext c, member m's copy in block m; the other
    blocks stay zero."""
    B = H * W
    assert members * B <= n_slots
    return Layout(c, [[(ch, m * B) for m in range(members)] for ch in range(c)], H, W, 1, W, B)


def forward_ensemble(net: List[Dict], raws: List[Dict], img: np.ndarray) -> np.ndarray:
    """Averaged logits of the ensemble members (float64)."""
    return sum(forward_plain(net, r, img) for r in raws) / float(len(raws))


def single_layout(c: int, B: int, n_slots: int) -> Layout:
    """One value per channel, channel k at block k (no replicas)."""
    nb = n_slots // B
    rep = [[(k // nb, (k % nb) * B)] for k in range(c)]
    return Layout((c + nb - 1) // nb, rep, 1, 1, 1, 1, B)


# =================================================================== program

def channel_vectors(L: Layout, values: np.ndarray, n_slots: int) -> List[np.ndarray]:
    """One slot vector per ciphertext of layout L holding values[c] at every
    position of every replica of channel c (zero elsewhere)."""
    vecs = [np.zeros(n_slots) for _ in range(L.n_ct)]
    for ch, reps in enumerate(L.rep):
        for ct, base in reps:
            for h in range(L.H):
                for w in range(L.W):
                    vecs[ct][L.slot(base, h, w)] = values[ch]
    return vecs


def round_exact(v: float) -> int:
    """round half away from zero, exactly, for any finite double."""
    if abs(v) >= 2.0 ** 52:
        return int(v)
    return int(math.copysign(math.floor(abs(v) + 0.5), v))


def lam_of(scale: float, log_delta: float) -> int:
    """sublevel lambda = round(log_Delta scale) (Sec. 4.3)."""
    return int(math.floor(math.log2(scale) / log_delta + 0.5))


@dataclass
class TensorInfo:
    layout: Layout
    level: int
    scale: float


class Program:
    """A straight-line homomorphic program over tensors (lists of ciphertexts).
    steps are dicts; see compile_he."""

    def __init__(self):
        self.steps: List[Dict] = []
        self.tensors: Dict[int, TensorInfo] = {}
        self.input_tensor = 0
        self.output_tensor = -1
        self.rot_steps: set = set()

    def new(self, info: TensorInfo) -> int:
        k = len(self.tensors)
        self.tensors[k] = info
        return k


def _lower_conv(w, stride: int, pad: int, Lin: Layout, Lout: Layout,
                n_slots: int) -> Dict[Tuple[int, int, int], np.ndarray]:
    """Diagonals {(out ct, in ct, r): vector} of a convolution between
    layouts: out slot so reads in slot si = so + r (mod n).  For each output
    replica, each input channel is read from its replica whose base is the
    smallest distance (base_in - base_out) mod n after it (ties: lower ct).
    w is one weight tensor, or a list: replica k of every output channel
    uses w[k] (an ensemble member per block)."""
    wl = w if isinstance(w, list) else None
    w0 = wl[0] if wl is not None else w
    cout, cin, k, _ = w0.shape
    diags: Dict[Tuple[int, int, int], np.ndarray] = {}
    hs = np.arange(Lout.H)
    ws = np.arange(Lout.W)
    for o in range(cout):
        for rk, (oct_, obase) in enumerate(Lout.rep[o]):
            w = wl[rk] if wl is not None else w0
            so = obase + (hs[:, None] * Lout.st) * Lout.Wp + ws[None, :] * Lout.st
            for i in range(cin):
                ict, ibase = min(Lin.rep[i], key=lambda cb: ((cb[1] - obase) % n_slots, cb[0]))
                for dh in range(k):
                    for dw in range(k):
                        hi = hs[:, None] * stride + dh - pad
                        wi = ws[None, :] * stride + dw - pad
                        ok = (hi >= 0) & (hi < Lin.H) & (wi >= 0) & (wi < Lin.W)
                        ok = np.broadcast_to(ok, so.shape)
                        if not ok.any():
                            continue
                        hi_b = np.broadcast_to(hi, so.shape)[ok]
                        wi_b = np.broadcast_to(wi, so.shape)[ok]
                        si = ibase + (hi_b * Lin.st) * Lin.Wp + wi_b * Lin.st
                        so_b = so[ok]
                        r_all = (si - so_b) % n_slots
                        for r in np.unique(r_all):
                            sel = r_all == r
                            key = (oct_, ict, int(r))
                            if key not in diags:
                                diags[key] = np.zeros(n_slots)
                            d = diags[key]
                            assert not d[so_b[sel]].any(), "two weights on one diagonal slot"
                            d[so_b[sel]] = w[o, i, dh, dw]
    return diags


def _bsgs(diags, G: int, n_slots: int):
    """Split r = g + b with b = r mod G; pre-rotate each diagonal by -g
    (vector v'[s] = v[s - g]) so that rot_g(v' . rot_b(x)) = v . rot_r(x)."""
    baby = set()
    groups: Dict[int, Dict[int, List]] = {}
    for (o, i, r) in sorted(diags):
        b = r % G
        g = r - b
        if b:
            baby.add((i, b))
        groups.setdefault(o, {}).setdefault(g, []).append((i, b, np.roll(diags[(o, i, r)], g)))
    return sorted(baby), groups


def _bias_vector(bias, Lout: Layout, n_slots: int) -> Dict[int, np.ndarray]:
    """bias: one vector over channels, or a list (replica k uses bias[k])"""
    bl = bias if isinstance(bias, list) else None
    vecs: Dict[int, np.ndarray] = {}
    for o in range(len(bl[0] if bl is not None else bias)):
        for rk, (ct, base) in enumerate(Lout.rep[o]):
            b = bl[rk] if bl is not None else bias
            v = vecs.setdefault(ct, np.zeros(n_slots))
            for h in range(Lout.H):
                for w in range(Lout.W):
                    v[Lout.slot(base, h, w)] = b[o]
    return vecs


# Scale of the classifier's plaintexts: Delta * 2^6.  Its folded weights
# (pool divisor and activation coefficient included) are ~1e-5 on a few
# slots, and a plaintext's coefficients are of order Delta |w|
# sqrt(nonzero slots) / N; at Delta they would mostly round to zero.
CLASSIFIER_SCALE_BITS = 6


class Compiler:
    """Builds the homomorphic program of a transformed network: layouts,
    diagonals, levels, scales and rescale points."""

    def __init__(self, prm: C.Params, layout_kind: str, giants: Optional[List[int]] = None, members: int = 1,
                 input_lambda: int = 1, hoists: Optional[List[int]] = None):
        """giants: the giant-step size of each linear step in program order
        (any split r = g + b with b = r mod G is a valid evaluation of the
        same diagonals; the choice only moves work between baby and giant
        rotations).  Default: one block for convolutions, 8 blocks for the
        packed dense layer, the whole slot vector in the HW layout.
        hoists: per linear step, 1 (each baby-step rotation brought back to
        Q_l by its own ModDown) or 2 (double hoisting: the rotations stay in
        Q_l u P, their plaintext products are summed there and each output
        group takes one ModDown); default 1."""
        self.prm = prm
        self.n = prm.N // 2
        self.log_delta = math.log2(prm.scale)
        self.kind = layout_kind
        self.prog = Program()
        self.giants = giants
        self.hoists = hoists
        self.n_linear = 0
        self.members = members
        # the client encrypts the image at scale Delta^input_lambda
        self.input_lambda = input_lambda

    # -- tower reuse
    def _maybe_rescale(self, t: int) -> int:
        info = self.prog.tensors[t]
        q = self.prm.q[info.level]
        if info.level >= 1 and lam_of(info.scale, self.log_delta) > lam_of(q, self.log_delta):
            out = self.prog.new(TensorInfo(info.layout, info.level - 1, info.scale / q))
            self.prog.steps.append({"op": "rescale", "src": t, "dst": out})
            return out
        return t

    def _linear(self, src: int, diags, G: int, Lout: Layout, w_scale: float,
                bias_vecs: Optional[Dict[int, np.ndarray]], out_scale: Optional[float] = None) -> int:
        info = self.prog.tensors[src]
        if self.giants is not None:
            G = self.giants[self.n_linear]
        hoist = self.hoists[self.n_linear] if self.hoists is not None else 1
        self.n_linear += 1
        baby, groups = _bsgs(diags, G, self.n)
        prod_scale = info.scale * w_scale
        out = self.prog.new(TensorInfo(Lout, info.level, prod_scale if out_scale is None else out_scale))
        for (_, b) in baby:
            self.prog.rot_steps.add(b)
        for o in groups:
            for g in groups[o]:
                if g:
                    self.prog.rot_steps.add(g)
        self.prog.steps.append({"op": "linear", "src": src, "dst": out, "w_scale": w_scale, "giant": G,
                                "bias_scale": prod_scale, "baby": baby, "groups": groups,
                                "bias": bias_vecs or {}, "n_out": Lout.n_ct, "hoist": hoist})
        return out

    def compile(self, net: List[Dict], t) -> Program:
        """t: one model's transformed parameters, or a list of them (an
        ensemble in the hw_ens layout; the members share activation
        polynomials and shortcut multipliers)."""
        ts = t if isinstance(t, list) else [t]
        t = ts[0]
        for i, nd in enumerate(net):
            if nd["op"] in ("act", "add"):
                assert all(x[i] == t[i] for x in ts), "members must share activations and shortcuts"
        prm, n = self.prm, self.n
        node_t: Dict[int, int] = {}
        shortcut_convs = {nd["src"][1] for nd in net if nd["op"] == "add"
                          and net[nd["src"][1]]["op"] == "conv"}
        for i, nd in enumerate(net):
            op = nd["op"]
            if op == "input":
                if self.kind == "hw":
                    L0 = hw_layout(nd["c"], nd["h"], nd["w"], n)
                elif self.kind == "hw_ens":
                    L0 = hw_ensemble_layout(nd["c"], nd["h"], nd["w"], n, self.members)
                else:
                    L0 = packed_layout(nd["c"], nd["h"], nd["w"], 1, nd["w"], nd["h"] * nd["w"], n)
                node_t[i] = self.prog.new(TensorInfo(L0, prm.L, prm.scale ** self.input_lambda))
                self.prog.input_tensor = node_t[i]
            elif op == "conv":
                if i in shortcut_convs:
                    continue
                node_t[i] = self._conv(node_t[nd["src"]], nd, [x[i] for x in ts], None)
            elif op == "bn":
                node_t[i] = node_t[nd["src"]]      # fused into the activation (Case 1)
            elif op == "act":
                src = node_t[nd["src"]]
                info = self.prog.tensors[src]
                s = info.scale
                s2 = s * s
                out = self.prog.new(TensorInfo(info.layout, info.level, s2))
                if np.ndim(t[i]["c1"]):
                    # per-channel coefficients (Case 1): slot vectors, c1
                    # encoded at scale s (c1 (.) x is at s*s), c0 at s*s
                    self.prog.steps.append({"op": "act", "src": src, "dst": out,
                                            "c1_vecs": channel_vectors(info.layout, t[i]["c1"], n),
                                            "c0_vecs": channel_vectors(info.layout, t[i]["c0"], n),
                                            "c1_scale": s, "c0_scale": s2})
                else:
                    # constants: c1 at scale s (so c1*x is at s*s), c0 at scale s*s
                    self.prog.steps.append({"op": "act", "src": src, "dst": out,
                                            "c1": round_exact(t[i]["c1"] * s),
                                            "c0": round_exact(t[i]["c0"] * s2)})
                node_t[i] = self._maybe_rescale(out)
            elif op == "pool":
                src = node_t[nd["src"]]
                info = self.prog.tensors[src]
                L = info.layout
                k = nd["k"]
                steps = [L.st * (1 << m) for m in range(int(math.log2(k)))] + \
                        [L.st * L.Wp * (1 << m) for m in range(int(math.log2(k)))]
                Lp = Layout(L.n_ct, L.rep, L.H // k, L.W // k, L.st * k, L.Wp, L.B)
                out = self.prog.new(TensorInfo(Lp, info.level, info.scale))
                self.prog.steps.append({"op": "rotsum", "src": src, "dst": out, "steps": steps})
                self.prog.rot_steps.update(steps)
                node_t[i] = out
            elif op == "add":
                a, b = nd["src"]
                ta = node_t[a]
                ia = self.prog.tensors[ta]
                if net[b]["op"] == "conv":
                    tb = self._conv(node_t[net[b]["src"]], net[b], [x[b] for x in ts], ia)
                else:
                    tb = self._shortcut_const(node_t[b], t[i]["shortcut_const"], ia)
                out = self.prog.new(TensorInfo(ia.layout, ia.level, ia.scale))
                self.prog.steps.append({"op": "add", "src": [ta, tb], "dst": out})
                node_t[i] = out
            elif op == "dense":
                node_t[i] = self._dense(node_t[nd["src"]], nd, [x[i] for x in ts], i == len(net) - 1)
        self.prog.output_tensor = node_t[len(net) - 1]
        return self.prog

    def _target_scale(self, info: TensorInfo, target: TensorInfo) -> Tuple[float, bool]:
        """Scale for the shortcut's multiplier so that, after the tower-reuse
        rule, it lands on the main branch's scale: with one rescale by
        q_level the multiplier is target*q/s, else target/s."""
        q = self.prm.q[info.level]
        w_scale = target.scale * q / info.scale
        lam_p = lam_of(info.scale * w_scale, self.log_delta)
        if info.level >= 1 and lam_p > lam_of(q, self.log_delta):
            return w_scale, True
        return target.scale / info.scale, False

    def _shortcut_const(self, src: int, value: float, target: TensorInfo) -> int:
        info = self.prog.tensors[src]
        w_scale, _ = self._target_scale(info, target)
        out = self.prog.new(TensorInfo(info.layout, info.level, info.scale * w_scale))
        self.prog.steps.append({"op": "cmul", "src": src, "dst": out,
                                "value": round_exact(value * w_scale)})
        out = self._maybe_rescale(out)
        return self._align(out, target)

    def _align(self, t: int, target: TensorInfo) -> int:
        info = self.prog.tensors[t]
        assert info.level >= target.level
        if info.level > target.level:
            out = self.prog.new(TensorInfo(info.layout, target.level, target.scale))
            self.prog.steps.append({"op": "drop", "src": t, "dst": out, "level": target.level})
            return out
        info.scale = target.scale
        return t

    def _conv(self, src: int, nd: Dict, tps: List[Dict], target: Optional[TensorInfo]) -> int:
        """tps: the layer's parameters of every member (one entry unless the
        layout is hw_ens, where output replica k uses member k)"""
        info = self.prog.tensors[src]
        Lin = info.layout
        Ho = (Lin.H + 2 * nd["pad"] - nd["k"]) // nd["stride"] + 1
        Wo = (Lin.W + 2 * nd["pad"] - nd["k"]) // nd["stride"] + 1
        st = Lin.st * nd["stride"]
        if self.kind in ("hw", "hw_ens"):
            Lout = Layout(nd["cout"], [[(o, base) for (_, base) in Lin.rep[0]] for o in range(nd["cout"])],
                          Ho, Wo, st, Lin.Wp, Lin.B)
            G = self.n
        else:
            Lout = packed_layout(nd["cout"], Ho, Wo, st, Lin.Wp, Lin.B, self.n)
            G = Lin.B
        if self.kind == "hw_ens":
            w_in, b_in = [tp["w"] for tp in tps], [tp["bias"] for tp in tps]
        else:
            w_in, b_in = tps[0]["w"], tps[0]["bias"]
        diags = _lower_conv(w_in, nd["stride"], nd["pad"], Lin, Lout, self.n)
        w_scale = self.prm.scale if target is None else self._target_scale(info, target)[0]
        bias = _bias_vector(b_in, Lout, self.n)
        out = self._linear(src, diags, G, Lout, w_scale, bias)
        out = self._maybe_rescale(out)
        if target is not None:
            out = self._align(out, target)
        return out

    def _dense(self, src: int, nd: Dict, tps: List[Dict], classifier: bool = False) -> int:
        info = self.prog.tensors[src]
        Lin = info.layout
        cout = nd["cout"]
        tp = tps[0]
        w = tp["w"]
        w_scale = self.prm.scale * (2.0 ** CLASSIFIER_SCALE_BITS if classifier else 1.0)
        if self.kind == "hw_ens":
            return self._dense_ensemble(src, nd, tps, w_scale)
        if self.kind == "hw":
            # per-output partial products in block k, then a sum over the block
            cin = len(Lin.rep)
            Lpart = Layout(1, [[(0, k * Lin.B)] for k in range(cout)], Lin.H, Lin.W, Lin.st, Lin.Wp, Lin.B)
            diags: Dict[Tuple[int, int, int], np.ndarray] = {}
            for c in range(cin):
                for k in range(cout):
                    ict, ibase = min(Lin.rep[c], key=lambda cb: ((cb[1] - k * Lin.B) % self.n, cb[0]))
                    assert ibase == k * Lin.B
                    v = diags.setdefault((0, ict, 0), np.zeros(self.n))
                    for h in range(Lin.H):
                        for x in range(Lin.W):
                            v[Lin.slot(ibase, h, x)] = w[k, (c * Lin.H + h) * Lin.W + x]
            bias = np.zeros(self.n)
            for k in range(cout):
                bias[k * Lin.B] = tp["bias"][k]
            out = self._linear(src, diags, self.n, Lpart, w_scale, {0: bias})
            out = self._maybe_rescale(out)
            oi = self.prog.tensors[out]
            steps = [Lin.st * (1 << m) for m in range(int(math.log2(Lin.W)))] + \
                    [Lin.st * Lin.Wp * (1 << m) for m in range(int(math.log2(Lin.H)))]
            Lo = single_layout(cout, Lin.B, self.n)
            res = self.prog.new(TensorInfo(Lo, oi.level, oi.scale))
            self.prog.steps.append({"op": "rotsum", "src": out, "dst": res, "steps": steps})
            self.prog.rot_steps.update(steps)
            return res
        # packed: features sit at block bases; generic diagonals with giant
        # steps of 8 blocks
        assert Lin.H == 1 and Lin.W == 1
        Lo = single_layout(cout, Lin.B, self.n)
        diags = _lower_conv(w[:, :, None, None], 1, 0, Lin, Lo, self.n)
        bias = _bias_vector(tp["bias"], Lo, self.n)
        out = self._linear(src, diags, 8 * Lin.B, Lo, w_scale, bias)
        return self._maybe_rescale(out)


    def _dense_ensemble(self, src: int, nd: Dict, tps: List[Dict], w_scale: float) -> int:
        """Ensemble dense layer and average (Sec. 5.3) in the HW layout: the
        pooled feature of channel c, member m, sits in ciphertext c at slot
        m*B; logit k of member m is accumulated at slot m*B + k from the
        diagonal r = -k with weight w_m[k, c] / M (the 1/M of the average
        folded into the weights and bias); every diagonal is a giant step
        (G = 1).  Then, before the rescale (at the product's larger scale,
        where rotation noise is negligible), the blocks are summed with
        rotations by B, 2B, .., so the average of logit k lands in slot k."""
        info = self.prog.tensors[src]
        Lin = info.layout
        cout, M, B = nd["cout"], self.members, Lin.B
        assert Lin.H == 1 and Lin.W == 1 and cout <= B
        diags: Dict[Tuple[int, int, int], np.ndarray] = {}
        for c in range(len(Lin.rep)):
            ict = Lin.rep[c][0][0]
            for k in range(cout):
                v = diags.setdefault((0, ict, (-k) % self.n), np.zeros(self.n))
                for m in range(M):
                    assert Lin.rep[c][m][1] == m * B
                    v[m * B + k] = tps[m]["w"][k, c] / float(M)
        Lpart = Layout(1, [[(0, m * B + k) for m in range(M)] for k in range(cout)], 1, 1, 1, 1, B)
        bias = np.zeros(self.n)
        for k in range(cout):
            for m in range(M):
                bias[m * B + k] = tps[m]["bias"][k] / float(M)
        out = self._linear(src, diags, 1, Lpart, w_scale, {0: bias})
        oi = self.prog.tensors[out]
        steps = []
        span = 1
        while span < M:
            steps.append(span * B)
            span *= 2
        res = self.prog.new(TensorInfo(Layout(1, [[(0, k)] for k in range(cout)], 1, 1, 1, 1, B), oi.level,
                                       oi.scale))
        self.prog.steps.append({"op": "rotsum", "src": out, "dst": res, "steps": steps})
        self.prog.rot_steps.update(steps)
        return self._maybe_rescale(res)


def compile_he(net: List[Dict], t, prm: C.Params, layout_kind: str,
               giants: Optional[List[int]] = None, members: int = 1, input_lambda: int = 1,
               hoists: Optional[List[int]] = None) -> Program:
    return Compiler(prm, layout_kind, giants, members, input_lambda, hoists).compile(net, t)


# =================================================================== running

def input_vectors(prog: Program, img: np.ndarray, n_slots: int) -> List[np.ndarray]:
    L = prog.tensors[prog.input_tensor].layout
    vecs = [np.zeros(n_slots) for _ in range(L.n_ct)]
    for c in range(len(L.rep)):
        for (ct, base) in L.rep[c]:
            for h in range(L.H):
                for w in range(L.W):
                    vecs[ct][L.slot(base, h, w)] = img[c, h, w]
    return vecs


def encrypt_input(S: C.CKKS, keys: C.Keys, prog: Program, img: np.ndarray, image_index: int,
                  enc_seed) -> List[C.Ciphertext]:
    prm = S.prm
    out = []
    scale = prog.tensors[prog.input_tensor].scale
    for k, v in enumerate(input_vectors(prog, img, prm.N // 2)):
        pt = S.encode(v, scale, prm.L)
        out.append(S.encrypt(keys, pt, enc_seed(image_index, k)))
    return out


def _const_ct(S: C.CKKS, x: C.Ciphertext, value: int) -> C.Ciphertext:
    return S.mul_const(x, value, 1.0)


def run_he(S: C.CKKS, keys: C.Keys, prog: Program, cts: List[C.Ciphertext],
           stop_after: Optional[int] = None) -> Dict[int, List[C.Ciphertext]]:
    """Evaluate the program; returns every tensor's ciphertexts."""
    prm = S.prm
    vals: Dict[int, List[C.Ciphertext]] = {prog.input_tensor: cts}
    for si, st in enumerate(prog.steps):
        op = st["op"]
        dst_info = prog.tensors[st["dst"]]
        if op == "linear":
            # baby steps: the rotations of one input share its ModUp; giant
            # steps: the rotated partial sums of one output share a ModDown
            xs = vals[st["src"]]
            level = xs[0].level
            dh = st.get("hoist", 1) == 2
            rot = {}
            for i in range(len(xs)):
                rot[(i, 0)] = xs[i]
                steps_i = [b for (ii, b) in st["baby"] if ii == i]
                if steps_i:
                    hoisted = S.rotate_hoisted_ext if dh else S.rotate_hoisted
                    for b, r in hoisted(xs[i], steps_i, keys).items():
                        rot[(i, b)] = r
            outs = []
            for o in range(st["n_out"]):
                partial = {}
                for g in sorted(st["groups"].get(o, {})):
                    acc = None
                    ext_acc = None
                    for (i, b, vec) in st["groups"][o][g]:
                        if dh and b != 0:
                            # double hoisting: the product and the sum in Q_l u P
                            term = S.mul_plain_ext(rot[(i, b)], S.encode_ext(vec, st["w_scale"], level), level)
                            ext_acc = term if ext_acc is None else S.add_ext(ext_acc, term, level)
                            continue
                        pt = S.encode(vec, st["w_scale"], level)
                        term = S.mul_plain(rot[(i, b)], pt)
                        acc = term if acc is None else S.add(acc, term)
                    if ext_acc is not None:
                        # one ModDown for the group's rotated terms
                        down = C.Ciphertext(S.moddown(ext_acc, level), level, xs[0].scale * st["w_scale"])
                        acc = down if acc is None else S.add(acc, down)
                    partial[g] = acc
                base = partial.get(0)
                if base is None:
                    base = C.Ciphertext(np.zeros((2, level + 1, prm.N), dtype=np.uint64), level, 1.0)
                if o in st["bias"]:
                    base = S.add_plain(base, S.encode(st["bias"][o], st["bias_scale"], level))
                giants = [(partial[g], g) for g in sorted(partial) if g]
                total = S.rotate_sum_lazy(giants, keys, base) if giants else base
                total.scale = dst_info.scale
                outs.append(total)
            vals[st["dst"]] = outs
        elif op == "rescale":
            vals[st["dst"]] = [S.rescale(x) for x in vals[st["src"]]]
        elif op == "act":
            outs = []
            for k, x in enumerate(vals[st["src"]]):
                y = S.relinearize(S.tensor_square(x), keys)
                if "c1_vecs" in st:
                    # per-channel coefficients: plaintext product and sum
                    y = S.add(y, S.mul_plain(x, S.encode(st["c1_vecs"][k], st["c1_scale"], x.level)))
                    y = S.add_plain(y, S.encode(st["c0_vecs"][k], st["c0_scale"], x.level))
                else:
                    y = S.add(y, S.mul_const(x, st["c1"], x.scale))
                    y = S.add_const(y, st["c0"])
                y.scale = dst_info.scale
                outs.append(y)
            vals[st["dst"]] = outs
        elif op == "rotsum":
            outs = []
            for x in vals[st["src"]]:
                for s in st["steps"]:
                    x = S.add(x, S.rotate(x, s, keys))
                outs.append(x)
            vals[st["dst"]] = outs
        elif op == "cmul":
            outs = []
            for x in vals[st["src"]]:
                y = S.mul_const(x, st["value"], 1.0)
                y.scale = dst_info.scale
                outs.append(y)
            vals[st["dst"]] = outs
        elif op == "drop":
            vals[st["dst"]] = [S.drop_to(x, st["level"]) for x in vals[st["src"]]]
        elif op == "add":
            a, b = st["src"]
            vals[st["dst"]] = [S.add(x, y) for x, y in zip(vals[a], vals[b])]
        for x in vals[st["dst"]]:
            assert x.level == dst_info.level, (si, op, x.level, dst_info.level)
            x.scale = dst_info.scale
        if stop_after is not None and si >= stop_after:
            break
    return vals


def decrypt_logits(S: C.CKKS, keys: C.Keys, prog: Program, cts: List[C.Ciphertext]) -> np.ndarray:
    L = prog.tensors[prog.output_tensor].layout
    slots = [S.decrypt_decode(keys, ct).real for ct in cts]
    return np.array([slots[L.rep[k][0][0]][L.rep[k][0][1]] for k in range(len(L.rep))])
