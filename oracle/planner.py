"""Level accounting and the tower-reuse rule (test infrastructure only).

* ``table1_levels`` counts the multiplicative levels of a network along its
  longest path for the six variants of Table 1 (Sec. 4.4): per-operation level
  costs are conv 1, batch norm 1, activation 3 (degree 4, P4) or 2 (degree 2),
  average pool 1, dense 1; node fusing (F) folds batch norm into the
  convolution (cost 0); weight redistribution (R) makes batch norm x + b0
  (cost 0), the activation monic x^2 + c1 x + c0 (cost 1) and the pool a plain
  sum (cost 0); tower reuse (T) halves the count, rounding up.
* ``tower_reuse`` applies the rule of Sec. 4.3 -- rescale when
  lambda(x) > lambda(q_i), with lambda(x) = round(log_Delta Delta_x) -- to a
  sequence of multiplicative steps and reports where the rescales fall.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

VARIANTS = ("P4", "P2", "P2F", "P2R", "P2FR", "P2FRT")


def table1_levels(n_conv: int, n_bn: int, n_act: int, n_pool: int, n_fc: int,
                  variant: str) -> int:
    if variant == "P2FRT":
        return math.ceil(table1_levels(n_conv, n_bn, n_act, n_pool, n_fc, "P2FR") / 2)
    fused = "F" in variant
    redistributed = "R" in variant
    act = 3 if variant == "P4" else (1 if redistributed else 2)
    bn = 0 if (fused or redistributed) else 1
    pool = 0 if redistributed else 1
    return n_conv * 1 + n_bn * bn + n_act * act + n_pool * pool + n_fc * 1


def lam(scale_log_delta: float) -> int:
    """lambda(x) = round(log_Delta Delta_x), given log_Delta Delta_x."""
    return int(math.floor(scale_log_delta + 0.5))


def tower_reuse(steps: Sequence[Tuple[str, int]], lam_q: int, lam_in: int = 1) -> Tuple[int, List[int]]:
    """Track sublevels through `steps` = [(kind, lambda of the multiplier)],
    kind in {"mul", "square"}; "square" doubles lambda, "mul" adds the
    multiplier's lambda.  After each step, rescale if lambda > lam_q (which
    subtracts lam_q).  Returns (number of rescales, lambda after each step)."""
    lam_x = lam_in
    n = 0
    trace = []
    for kind, lam_w in steps:
        lam_x = 2 * lam_x if kind == "square" else lam_x + lam_w
        if lam_x > lam_q:
            lam_x -= lam_q
            n += 1
        trace.append(lam_x)
    return n, trace


def alternating_path(n_linear: int, n_act: int) -> List[Tuple[str, int]]:
    """Longest multiplicative path of a VGG/ResNet after fusing and
    redistribution: linear, act, linear, act, ..., linear (weights at
    lambda 1); pools and batch norms contribute no step."""
    steps: List[Tuple[str, int]] = []
    for k in range(n_linear):
        steps.append(("mul", 1))
        if k < n_act:
            steps.append(("square", 0))
    return steps


# layer counts along the longest path (Sec. 4.4; ResNet-18 is spelled out
# there, the others follow the same architecture definitions)
PROFILES: Dict[str, Dict[str, int]] = {
    "VGG-16": dict(n_conv=13, n_bn=13, n_act=15, n_pool=5, n_fc=3),
    "ResNet-18": dict(n_conv=17, n_bn=17, n_act=17, n_pool=1, n_fc=1),
    "ResNet-20": dict(n_conv=19, n_bn=19, n_act=19, n_pool=1, n_fc=1),
    "ResNet-32": dict(n_conv=31, n_bn=31, n_act=31, n_pool=1, n_fc=1),
}
