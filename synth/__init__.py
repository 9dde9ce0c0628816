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

def _conv(src, cin, cout, k, stride, pad, name):
    return {"op": "conv", "src": src, "cin": cin, "cout": cout, "k": k,
            "stride": stride, "pad": pad, "bn": True, "name": name}


def tiny() -> List[Dict]:
    """16x16x3 input, conv 3x3 3->8 (+BN), activation, 2x2 average pool,
    dense 512->10."""
    net = [{"op": "input", "c": 3, "h": 16, "w": 16}]
    net.append(_conv(0, 3, 8, 3, 1, 1, "conv1"))
    net.append({"op": "act", "src": 1})
    net.append({"op": "pool", "src": 2, "k": 2})
    net.append({"op": "dense", "src": 3, "cin": 8 * 8 * 8, "cout": 10, "name": "fc"})
    return net


def resnet(widths=(16, 32, 64), blocks=3, in_hw=32, num_classes=10) -> List[Dict]:
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

    x = add(_conv(0, 3, widths[0], 3, 1, 1, "conv1"))
    x = add({"op": "act", "src": x})
    cin = widths[0]
    hw = in_hw
    for s, cout in enumerate(widths):
        for b in range(blocks):
            stride = 2 if (s > 0 and b == 0) else 1
            hw //= stride
            a = add(_conv(x, cin, cout, 3, stride, 1, "s%db%da" % (s + 1, b + 1)))
            a = add({"op": "act", "src": a})
            m = add(_conv(a, cout, cout, 3, 1, 1, "s%db%db" % (s + 1, b + 1)))
            if stride != 1 or cin != cout:
                sc = add(_conv(x, cin, cout, 1, stride, 0, "s%db%dsc" % (s + 1, b + 1)))
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


def resnet_mini() -> List[Dict]:
    """A ResNet with the same structure at a small size (8x8x3 input,
    4/8/16 channels, one block per stage) for full-network parity tests."""
    return resnet((4, 8, 16), 1, 8, 10)


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


ARCHS = {"tiny": tiny, "resnet20": resnet20, "resnet_mini": resnet_mini, "vgg11": vgg11, "vgg_mini": vgg_mini}


# ------------------------------------------------------------- parameters

def params(net: List[Dict]) -> Dict[int, Dict[str, np.ndarray]]:
    """Raw (unfolded) parameters keyed by node index, drawn in node order."""
    rw = np.random.default_rng(SEED_WEIGHTS)
    rb = np.random.default_rng(SEED_BN)
    ra = np.random.default_rng(SEED_ACT)
    out: Dict[int, Dict[str, np.ndarray]] = {}
    for i, nd in enumerate(net):
        if nd["op"] == "conv":
            fan_in = nd["cin"] * nd["k"] * nd["k"]
            w = rw.normal(0.0, fan_in ** -0.5, size=(nd["cout"], nd["cin"], nd["k"], nd["k"]))
            c = nd["cout"]
            out[i] = {
                "w": w,
                "bias": np.zeros(c),
                "gamma": rb.uniform(0.5, 1.5, c),
                "beta": rb.normal(0.0, 0.1, c),
                "mu": rb.normal(0.0, 0.1, c),
                "sigma": rb.uniform(0.5, 1.5, c),
            }
        elif nd["op"] == "dense":
            w = rw.normal(0.0, nd["cin"] ** -0.5, size=(nd["cout"], nd["cin"]))
            out[i] = {"w": w, "bias": rb.normal(0.0, 0.01, nd["cout"])}
        elif nd["op"] == "act":
            out[i] = {"a": ra.normal(0.1, 0.02), "b": ra.normal(0.5, 0.05),
                      "c": ra.normal(0.0, 0.01)}
    return out


def enc_seed(image_index: int, ct_index: int) -> int:
    """Encryption seed of input ciphertext ct_index of image image_index."""
    return (SEED_ENCRYPT << 40) | (image_index << 12) | ct_index


# CKKS parameter presets: ring degree 2^logn; q_1..q_L of q_bits, q_0 of
# q0_bits, alpha special primes of p_bits (alpha is also the digit width of
# hybrid key switching); default scale Delta = 2^log_scale.
PRESETS = {
    "tiny": dict(logn=13, L=4, q_bits=40, q0_bits=40, p_bits=40, alpha=1, log_scale=40),
    "resnet_mini": dict(logn=12, L=8, q_bits=50, q0_bits=40, p_bits=58, alpha=3, log_scale=25),
    "vgg11": dict(logn=16, L=11, q_bits=50, q0_bits=40, p_bits=58, alpha=3, log_scale=25),
    "resnet20": dict(logn=16, L=20, q_bits=50, q0_bits=40, p_bits=58, alpha=3, log_scale=25),
}
