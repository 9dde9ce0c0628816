"""Seeded synthetic workloads: network shapes, raw parameters and images.

This module is shared by the oracle, the tests and the benchmark.  It holds
no arithmetic of the method itself: it only draws random numbers with fixed
seeds and describes network shapes.  Batch-norm folding, weight
redistribution, slot layouts and everything homomorphic live elsewhere.

Value distributions (synthetic stand-ins for the paper's CIFAR/Tiny-ImageNet
workloads; no dataset items are reproduced):
  images                  float64 uniform[0,1], numpy default_rng(1000 + i)
  conv / dense weights    normal, variance 1/fan_in (std fan_in^-1/2), seed 1
  batch-norm parameters   gamma ~ U[0.5,1.5], beta ~ N(0,0.1), mu ~ N(0,0.1),
                          sigma ~ U[0.5,1.5] per output channel, seed 2
  dense bias              N(0, 0.01), seed 2 (after the batch-norm draws)
  activation coefficients a ~ N(0.1,0.02), b ~ N(0.5,0.05), c ~ N(0,0.01),
                          one triple per activation layer, seed 3
  ensemble member m       weights and batch norm from seeds 1 + 100 m and
                          2 + 100 m; the activation polynomial of a layer
                          (seed 3) is shared by the members
  clustered weights       per layer, joint k-means in R^M over the members'
                          weight draws (k centroids fitted on at most 10^5
                          positions, ``cluster_joint``); every weight is
                          replaced by its nearest centroid's entry
"""
from __future__ import annotations

from typing import Dict, List

import numpy as np

SEED_WEIGHTS = 1
SEED_BN = 2
SEED_ACT = 3
SEED_ENCRYPT = 7
SEED_KEYS = 11


def image(i: int, c: int, h: int, w: int) -> np.ndarray:
    """Image number i: float64 uniform[0,1] of shape [c, h, w]."""
    return np.random.default_rng(1000 + i).uniform(0.0, 1.0, size=(c, h, w))


# ----------------------------------------------------------------- shapes

def _conv(src, cin, cout, k, stride, pad, name, bn=True):
    return {"op": "conv", "src": src, "cin": cin, "cout": cout, "k": k,
            "stride": stride, "pad": pad, "bn": bn, "name": name}


def tiny() -> List[Dict]:
    """16x16x3 input, conv 3x3 3->8 (+BN), activation, 2x2 average pool,
    dense 512->10."""
    net = [{"op": "input", "c": 3, "h": 16, "w": 16}]
    net.append(_conv(0, 3, 8, 3, 1, 1, "conv1"))
    net.append({"op": "act", "src": 1})
    net.append({"op": "pool", "src": 2, "k": 2})
    net.append({"op": "dense", "src": 3, "cin": 8 * 8 * 8, "cout": 10, "name": "fc"})
    return net


def resnet(widths=(16, 32, 64), blocks=3, in_hw=32, num_classes=10, bn=True) -> List[Dict]:
    """CIFAR-style ResNet: conv 3->widths[0], len(widths) stages of `blocks`
    basic blocks (the first block of every later stage has stride 2 and a
    1x1 stride-2 convolution on the shortcut, the others identity
    shortcuts), global average pool, dense -> num_classes.  Every
    convolution is followed by batch norm; every block ends with add then
    activation."""
    net = [{"op": "input", "c": 3, "h": in_hw, "w": in_hw}]

    def add(node):
        net.append(node)
        return len(net) - 1

    x = add(_conv(0, 3, widths[0], 3, 1, 1, "conv1", bn))
    x = add({"op": "act", "src": x})
    cin = widths[0]
    hw = in_hw
    for s, cout in enumerate(widths):
        for b in range(blocks):
            stride = 2 if (s > 0 and b == 0) else 1
            hw //= stride
            a = add(_conv(x, cin, cout, 3, stride, 1, "s%db%da" % (s + 1, b + 1), bn))
            a = add({"op": "act", "src": a})
            m = add(_conv(a, cout, cout, 3, 1, 1, "s%db%db" % (s + 1, b + 1), bn))
            if stride != 1 or cin != cout:
                sc = add(_conv(x, cin, cout, 1, stride, 0, "s%db%dsc" % (s + 1, b + 1), bn))
            else:
                sc = x
            y = add({"op": "add", "src": [m, sc]})
            x = add({"op": "act", "src": y})
            cin = cout
    p = add({"op": "pool", "src": x, "k": hw})
    add({"op": "dense", "src": p, "cin": cin, "cout": num_classes, "name": "fc"})
    return net


def resnet20(num_classes: int = 10) -> List[Dict]:
    """ResNet-20 for 32x32x3: three stages of three basic blocks with
    16/32/64 channels, global 8x8 average pool, dense 64->num_classes."""
    return resnet((16, 32, 64), 3, 32, num_classes)


def resnet32(num_classes: int = 10) -> List[Dict]:
    """ResNet-32 for 32x32x3: three stages of five basic blocks with
    16/32/64 channels (the paper's N = 2^16 workload, Table 4)."""
    return resnet((16, 32, 64), 5, 32, num_classes)


def resnet_mini() -> List[Dict]:
    """A ResNet with the same structure at a small size (8x8x3 input,
    4/8/16 channels, one block per stage) for full-network parity tests."""
    return resnet((4, 8, 16), 1, 8, 10)


def resnet18(num_classes: int = 200) -> List[Dict]:
    """ResNet-18 for 64x64x3 (Tiny-ImageNet shape): 3x3 stem, four stages of
    two basic blocks with 64/128/256/512 channels (stride 2 and a 1x1
    shortcut convolution at each later stage), global 8x8 average pool,
    dense 512->num_classes.  No batch norm: the weights are clustered after
    folding, so the synthetic model is drawn already folded (see
    ``cluster_joint``)."""
    return resnet((64, 128, 256, 512), 2, 64, num_classes, bn=False)


def resnet18_mini() -> List[Dict]:
    """ResNet-18's structure (four stages of two basic blocks, 18 levels) at
    a small size: 16x16x3, 2/2/4/4 channels, global 2x2 pool, 10 classes."""
    return resnet((2, 2, 4, 4), 2, 16, 10, bn=False)


def vgg(cfg=(64, "M", 128, "M", 256, 256, "M", 512, 512, "M", 512, 512, "M"), in_hw=32,
        fc=(512, 512), num_classes=10) -> List[Dict]:
    """VGG-style network: 3x3 convolutions (+BN, activation) with 2x2 average
    pools ("M"), then dense layers with activations, then the classifier."""
    net = [{"op": "input", "c": 3, "h": in_hw, "w": in_hw}]

    def add(node):
        net.append(node)
        return len(net) - 1

    x, cin, hw = 0, 3, in_hw
    for i, v in enumerate(cfg):
        if v == "M":
            x = add({"op": "pool", "src": x, "k": 2})
            hw //= 2
        else:
            x = add(_conv(x, cin, v, 3, 1, 1, "conv%d" % (i + 1)))
            x = add({"op": "act", "src": x})
            cin = v
    feat = cin * hw * hw
    for j, f in enumerate(fc):
        x = add({"op": "dense", "src": x, "cin": feat, "cout": f, "name": "fc%d" % (j + 1)})
        x = add({"op": "act", "src": x})
        feat = f
    add({"op": "dense", "src": x, "cin": feat, "cout": num_classes, "name": "fc%d" % (len(fc) + 1)})
    return net


def vgg11(num_classes: int = 10) -> List[Dict]:
    """VGG-11 (configuration A: 8 convolutions 64-128-256-256-512-512-512-512,
    5 average pools, dense 512-512-num_classes) for 32x32x3."""
    return vgg()


def vgg_mini() -> List[Dict]:
    """A VGG with the same structure at a small size (8x8x3, 4/8 channels,
    3 pools, dense 8-8-10) for full-network parity tests."""
    return vgg(cfg=(4, "M", 8, "M", "M"), in_hw=8, fc=(8,), num_classes=10)


def preact_mini() -> List[Dict]:
    """A pre-activation residual network at a small size (8x8x3, 4 channels,
    10 classes): 3x3 stem convolution and activation, two blocks x -> BN ->
    act -> conv -> act -> conv, + x, then BN -> act -> 8x8 average pool ->
    dense.  Each
    block's batch norm follows an addition, not a convolution: it is a node
    of its own, and the activation after it takes the fused per-channel
    polynomial of Sec. 4.1 Case 1.  The inner convolutions carry their own
    batch norm (folded, Case 2); the second has none (pre-activation)."""
    net = [{"op": "input", "c": 3, "h": 8, "w": 8}]

    def add(node):
        net.append(node)
        return len(net) - 1

    x = add(_conv(0, 3, 4, 3, 1, 1, "stem"))
    x = add({"op": "act", "src": x})
    for b in range(2):
        n = add({"op": "bn", "src": x, "c": 4})
        a = add({"op": "act", "src": n})
        c1 = add(_conv(a, 4, 4, 3, 1, 1, "b%d_conv1" % b))
        a2 = add({"op": "act", "src": c1})
        c2 = add(_conv(a2, 4, 4, 3, 1, 1, "b%d_conv2" % b, bn=False))
        x = add({"op": "add", "src": [c2, x]})
    n = add({"op": "bn", "src": x, "c": 4})
    a = add({"op": "act", "src": n})
    p = add({"op": "pool", "src": a, "k": 8})
    add({"op": "dense", "src": p, "cin": 4, "cout": 10, "name": "fc"})
    return net


ARCHS = {"tiny": tiny, "resnet20": resnet20, "resnet32": resnet32, "resnet_mini": resnet_mini, "vgg11": vgg11,
         "vgg_mini": vgg_mini, "resnet18": resnet18, "resnet18_mini": resnet18_mini, "preact_mini": preact_mini}


# ------------------------------------------------------------- parameters

def params(net: List[Dict], model: int = 0) -> Dict[int, Dict[str, np.ndarray]]:
    """Raw (unfolded) parameters keyed by node index, drawn in node order;
    `model` selects an ensemble member (its own weight and batch-norm draws,
    the shared activation polynomials).  A convolution without batch norm
    gets the identity (gamma 1, beta 0, mu 0, sigma 1)."""
    rw = np.random.default_rng(SEED_WEIGHTS + 100 * model)
    rb = np.random.default_rng(SEED_BN + 100 * model)
    ra = np.random.default_rng(SEED_ACT)
    out: Dict[int, Dict[str, np.ndarray]] = {}
    for i, nd in enumerate(net):
        if nd["op"] == "conv":
            fan_in = nd["cin"] * nd["k"] * nd["k"]
            w = rw.normal(0.0, fan_in ** -0.5, size=(nd["cout"], nd["cin"], nd["k"], nd["k"]))
            c = nd["cout"]
            if nd.get("bn", True):
                bn = {"gamma": rb.uniform(0.5, 1.5, c), "beta": rb.normal(0.0, 0.1, c),
                      "mu": rb.normal(0.0, 0.1, c), "sigma": rb.uniform(0.5, 1.5, c)}
            else:
                bn = {"gamma": np.ones(c), "beta": np.zeros(c), "mu": np.zeros(c), "sigma": np.ones(c)}
            out[i] = dict(w=w, bias=np.zeros(c), **bn)
        elif nd["op"] == "dense":
            w = rw.normal(0.0, nd["cin"] ** -0.5, size=(nd["cout"], nd["cin"]))
            out[i] = {"w": w, "bias": rb.normal(0.0, 0.01, nd["cout"])}
        elif nd["op"] == "act":
            out[i] = {"a": ra.normal(0.1, 0.02), "b": ra.normal(0.5, 0.05),
                      "c": ra.normal(0.0, 0.01)}
        elif nd["op"] == "bn":
            c = nd["c"]
            out[i] = {"gamma": rb.uniform(0.5, 1.5, c), "beta": rb.normal(0.0, 0.1, c),
                      "mu": rb.normal(0.0, 0.1, c), "sigma": rb.uniform(0.5, 1.5, c)}
    return out


def kmeans(points: np.ndarray, k: int, iters: int = 100):
    """Lloyd's k-means on points [n, d] (float64), deterministic: the initial
    centroids are the points at ranks floor((j + 1/2) n / k) of the order by
    (first coordinate, index); an assignment goes to the nearest centroid
    (squared Euclidean distance as |c|^2 - 2 p.c, ties to the lower index);
    a centroid is the mean of its points (an empty cluster keeps its
    centroid); stops when no
    assignment changes or after `iters` rounds.  Returns (centroids [k, d],
    assignment [n])."""
    n = len(points)
    order = np.lexsort((np.arange(n), points[:, 0]))
    k = min(k, n)
    cent = points[order[((np.arange(k) + 0.5) * n / k).astype(np.int64)]].copy()
    assign = None
    for _ in range(iters):
        # |p - c|^2 = |c|^2 - 2 p.c + |p|^2; |p|^2 is the same for every c
        d2 = (cent * cent).sum(axis=1)[None, :] - 2.0 * (points @ cent.T)
        new = np.argmin(d2, axis=1)
        if assign is not None and np.array_equal(new, assign):
            break
        assign = new
        cnt = np.bincount(assign, minlength=k)
        for dim in range(points.shape[1]):
            tot = np.bincount(assign, weights=points[:, dim], minlength=k)
            cent[cnt > 0, dim] = tot[cnt > 0] / cnt[cnt > 0]
    return cent, assign


def cluster_joint(raws: List[Dict[int, Dict[str, np.ndarray]]], net: List[Dict], k: int = 16,
                  fit_max: int = 100000):
    """Joint weight clustering of an ensemble: for every convolution and
    dense layer, the M members' weights at one position form a point of R^M;
    k-means (``kmeans``) gives k centroid vectors -- fitted on every
    ceil(n / fit_max)-th position when a layer has more than fit_max -- and
    every position takes its nearest centroid (squared distance, ties to the
    lower index): member m's weight becomes entry m of that centroid.
    Returns new parameter dicts (other entries shared)."""
    out = [{i: dict(p) for i, p in r.items()} for r in raws]
    for i, nd in enumerate(net):
        if nd["op"] not in ("conv", "dense"):
            continue
        shape = raws[0][i]["w"].shape
        pts = np.stack([r[i]["w"].reshape(-1) for r in raws], axis=1)
        stride = -(-len(pts) // fit_max)
        cent, assign = kmeans(pts[::stride], k)
        if stride > 1:
            d2 = (cent * cent).sum(axis=1)[None, :] - 2.0 * (pts @ cent.T)
            assign = np.argmin(d2, axis=1)
        for m in range(len(raws)):
            out[m][i]["w"] = cent[assign, m].reshape(shape)
    return out


def enc_seed(image_index: int, ct_index: int) -> int:
    """Encryption seed of input ciphertext ct_index of image image_index."""
    return (SEED_ENCRYPT << 40) | (image_index << 12) | ct_index


# CKKS parameter presets: ring degree 2^logn; q_1..q_L of q_bits, q_0 of
# q0_bits, alpha special primes of p_bits (alpha is also the digit width of
# hybrid key switching); default scale Delta = 2^log_scale.  The N = 2^16
# networks use dnum = 3 digits at the top level (alpha = 7 special primes of
# 58 bits for digits of seven 58-bit primes; key switches there run on
# ciphertexts at scale Delta^2 or more, where the digit/P noise term is
# negligible), and Delta = 2^29 with q ~ 2^58 keeps one prime per rescale
# (tower reuse, round(log_Delta q) = 2): measured ResNet-20 logit error
# 8.3e-4 at N = 2^16 (2.5e-3 at Delta = 2^28, 6.8e-2 at Delta = 2^25).
# scale of the client's input encoding, as a power of Delta, per preset: the
# N = 2^16 networks encrypt at Delta^2 so that the first layer's rotations,
# like all later key switches, act on a ciphertext at scale >= Delta^2
INPUT_LAMBDA = {"vgg11": 2, "resnet20": 2, "resnet18": 2}

PRESETS = {
    "tiny": dict(logn=13, L=4, q_bits=40, q0_bits=40, p_bits=40, alpha=1, log_scale=40),
    "resnet_mini": dict(logn=12, L=8, q_bits=50, q0_bits=40, p_bits=58, alpha=3, log_scale=25),
    "vgg11": dict(logn=16, L=11, q_bits=58, q0_bits=40, p_bits=58, alpha=7, log_scale=29),
    "resnet20": dict(logn=16, L=20, q_bits=58, q0_bits=40, p_bits=58, alpha=7, log_scale=29),
    "resnet18": dict(logn=16, L=18, q_bits=58, q0_bits=40, p_bits=58, alpha=7, log_scale=29),
    "resnet18_mini": dict(logn=12, L=18, q_bits=58, q0_bits=40, p_bits=58, alpha=7, log_scale=29),
}


# The paper's own parameter sets, with the prime chains its appendix on FHE
# parameters prints (q_0, the small output prime printed last there, first
# here; then q_1..q_L in printed order; then P).  One special prime, so one
# prime per key-switching digit.
PAPER_PARAMS = {
    "resnet32": dict(
        logn=16, L=32, alpha=1, log_scale=26,
        q=[
          0x8020001, 0x10000000060001, 0xffffffff00001, 0x10000000180001, 0xfffffffe40001,
          0x10000000200001, 0xfffffffe20001, 0x100000003e0001, 0xfffffffbe0001, 0x10000000500001,
          0xfffffffa60001, 0x100000006e0001, 0xfffffff820001, 0x100000007e0001, 0xfffffff480001,
          0x10000000960001, 0xfffffff280001, 0x10000000c80001, 0x10000000d80001, 0xffffffed60001,
          0x10000000ec0001, 0xffffffec40001, 0x10000000fc0001, 0xffffffeb00001, 0x100000010e0001,
          0xffffffe9e0001, 0x10000001380001, 0xffffffe9a0001, 0x100000016a0001, 0xffffffe940001,
          0x10000001bc0001, 0xffffffe6a0001, 0x10000001be0001,
        ],
        p=[0x3fffffffd60001]),
}
