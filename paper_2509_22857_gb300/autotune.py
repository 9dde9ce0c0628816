"""Autotuner for the launch parameters the kernels leave open.

Two knobs are measured on the device through the C ABI rather than fixed by
hand, and the results are cached per device name and parameter set:

* **Digit width** alpha of hybrid key switching: alpha special primes, and
  dnum = ceil((l+1)/alpha) digits at level l.  The width changes the key's
  shape and so the ciphertexts' bits: it is a parameter of the scheme, not a
  free launch choice.  The tuner therefore only ranks the *admissible* widths
  by measured key-switch time, weighted over the levels a network switches
  at.  The chosen width goes into the parameter preset, and the parity
  checks compute both sides with that same width.  A width is admissible when
  the special modulus P (alpha primes of p_bits) is at least every digit's
  modulus, so that the key-switching noise, about digit * e / P per digit
  (Sec. 2.2, hybrid key switching with a special modulus), stays at the
  level of a fresh encryption error; and when the key has no more digits
  than the library admits, min(2^(62 - b), 64) for the largest prime of b
  bits (the inner product sums one product below 2^(2b) per digit, and
  Barrett reduction takes sums below 2^(b+62)).
* **Linear-step chunk size** (MAC sources per pass, `fhe_ctx_set_linear_chunk`):
  bit-neutral.  The tuner checks that every candidate gives identical
  ciphertexts and keeps the fastest.
* **Images per MAC block** (`fhe_ctx_set_mac_images`: 1, 2, 4 or 8; a
  block covers 512 / images coefficients of one limb for that many images,
  its plaintext loads shared by them) and **key-switch batch** (items per
  launch of a step's whole key switches, `fhe_ctx_set_keyswitch_batch`):
  bit-neutral, same protocol as the chunk size.
* **Pipeline group size** (images entering the mixed-level pipeline per
  tick): bit-neutral; measured as images leaving per second, one pipeline
  alive at a time.

The NTT split (two passes of 2^ceil(logN/2) x 2^floor(logN/2)) and one limb
per CTA row are compile-time choices of the kernels' templates and are not
tuned here.
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

MAX_LIMBS = 64


def max_digits(max_bits: int) -> int:
    """most key-switching digits the library admits with primes of at most max_bits"""
    return min(1 << (62 - max_bits), MAX_LIMBS)


def digit_bits(L: int, q_bits: int, q0_bits: int, alpha: int) -> List[int]:
    """Bit size of each digit's modulus at the top level: digit j holds
    primes q_{j alpha} .. q_{(j+1) alpha - 1} of q_0 (q0_bits), q_1..q_L (q_bits)."""
    sizes = [q0_bits] + [q_bits] * L
    return [sum(sizes[j:j + alpha]) for j in range(0, L + 1, alpha)]


def admissible(L: int, q_bits: int, q0_bits: int, p_bits: int, alpha: int) -> bool:
    """P = alpha primes of p_bits covers every digit, and the library admits
    the digit count."""
    if alpha < 1:
        return False
    d = digit_bits(L, q_bits, q0_bits, alpha)
    return len(d) <= max_digits(max(q_bits, q0_bits, p_bits)) and alpha * p_bits >= max(d)


def admissible_widths(L: int, q_bits: int, q0_bits: int, p_bits: int,
                      candidates: Iterable[int] = range(1, 9)) -> List[int]:
    return [a for a in candidates if admissible(L, q_bits, q0_bits, p_bits, a)]


def device_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


@dataclass
class Tuner:
    """Result cache: key -> record, optionally persisted as JSON at `path`."""
    path: Optional[str] = None
    records: Dict[str, dict] = field(default_factory=dict)

    def __post_init__(self):
        if self.path and os.path.exists(self.path):
            with open(self.path) as f:
                self.records = json.load(f)

    def lookup(self, key: str) -> Optional[dict]:
        return self.records.get(key)

    def record(self, key: str, rec: dict) -> dict:
        self.records[key] = rec
        if self.path:
            d = os.path.dirname(os.path.abspath(self.path))
            os.makedirs(d, exist_ok=True)
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.records, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        return rec


def _key(op: str, device: str, **kw) -> str:
    return "|".join([op, device] + ["%s=%s" % (k, kw[k]) for k in sorted(kw)])


def tune_digit_width(tuner: Tuner, logn: int, L: int, q_bits: int, q0_bits: int, p_bits: int,
                     log_scale: float, candidates: Iterable[int] = range(1, 9),
                     levels: Optional[Sequence[Tuple[int, float]]] = None, items: int = 4, iters: int = 5,
                     F=None, device: Optional[str] = None, seed: int = 11) -> dict:
    """Rank the admissible digit widths by measured key-switch time.

    levels: (level, weight) pairs, e.g. the number of key switches a network
    performs at each level; default: the top level alone.  The cost of a
    width is sum(weight * microseconds per switched polynomial at level).
    Returns {"best": alpha, "cost_us": {alpha: cost}, "us": {alpha: {level: us}}}.
    """
    if F is None:
        from . import _lib as F
    dev = device if device is not None else device_name()
    levels = list(levels) if levels else [(L, 1.0)]
    widths = admissible_widths(L, q_bits, q0_bits, p_bits, candidates)
    if not widths:
        raise ValueError("no admissible digit width among the candidates")
    key = _key("digit_width", dev, logn=logn, L=L, q=q_bits, q0=q0_bits, p=p_bits, items=items,
               levels=",".join("%d:%g" % lw for lw in levels), widths=",".join(map(str, widths)))
    hit = tuner.lookup(key)
    if hit is not None:
        return hit
    us: Dict[int, Dict[int, float]] = {}
    for a in widths:
        ctx = F.fhe_ctx_create(logn, L, q_bits, q0_bits, p_bits, a, log_scale)
        try:
            sk, evk = F.fhe_keygen(ctx, seed, [])
            try:
                us[a] = {}
                for lv, _ in levels:
                    ms = F.fhe_profile_keyswitch(ctx, evk, lv, items, iters)
                    us[a][lv] = sum(ms) / items * 1e3
            finally:
                F.fhe_evk_free(evk)
                F.fhe_sk_free(sk)
        finally:
            F.fhe_ctx_destroy(ctx)
    cost = {a: sum(w * us[a][lv] for lv, w in levels) for a in widths}
    best = min(widths, key=lambda a: (cost[a], a))
    rec = {"best": best, "cost_us": {str(a): round(c, 3) for a, c in cost.items()},
           "us": {str(a): {str(lv): round(t, 3) for lv, t in v.items()} for a, v in us.items()}}
    return tuner.record(key, rec)


def keyswitch_levels(prog) -> List[Tuple[int, float]]:
    """(level, number of key switches of one image) of a compiled network
    program, top level first: the weights for tune_digit_width."""
    from . import model as M
    return sorted(((lv, float(k)) for lv, k in M.keyswitch_census(prog).items()), reverse=True)


def _tune_infer_knob(tuner: Tuner, op: str, label: str, setter: Callable, candidates: Sequence[int], ctx, model,
                     evk, cts, n_img: int, n_out: int, N: int, reps: int, F, device: Optional[str], model_key: str,
                     sync: Optional[Callable]) -> dict:
    """Time fhe_infer with each value of one bit-neutral context knob, check
    that every value gives identical ciphertexts, leave the fastest set in
    ctx.  Returns {"best": v, "ms": {v: ms}}."""
    if sync is None:
        import torch
        sync = torch.cuda.synchronize
    dev = device if device is not None else device_name()
    key = _key(op, dev, model=model_key, n_img=n_img, cands=",".join(map(str, candidates)))
    hit = tuner.lookup(key)
    if hit is not None:
        setter(ctx, hit["best"])
        return hit
    ref = None
    ms: Dict[int, float] = {}
    for c in candidates:
        setter(ctx, c)
        best_t = None
        for r in range(reps + 1):          # first run warms up
            sync()
            t0 = time.perf_counter()
            outs = F.fhe_infer(ctx, model, evk, cts, n_img, n_out)
            sync()
            t = (time.perf_counter() - t0) * 1e3
            if r == 0:
                got = [F.fhe_ct_export(h, N)[0] for h in outs]
                if ref is None:
                    ref = got
                elif not all((a == b).all() for a, b in zip(ref, got)):
                    for h in outs:
                        F.fhe_ct_free(h)
                    raise RuntimeError("%s %d changed the output ciphertexts" % (label, c))
            else:
                best_t = t if best_t is None else min(best_t, t)
            for h in outs:
                F.fhe_ct_free(h)
        ms[c] = best_t
    best = min(candidates, key=lambda c: (ms[c], c))
    setter(ctx, best)
    return tuner.record(key, {"best": best, "ms": {str(c): round(t, 3) for c, t in ms.items()}})


def tune_linear_chunk(tuner: Tuner, ctx, model, evk, cts, n_img: int, n_out: int, N: int,
                      candidates: Sequence[int] = (40, 80, 160, 320), reps: int = 2, F=None,
                      device: Optional[str] = None, model_key: str = "", sync: Optional[Callable] = None) -> dict:
    """Time fhe_infer with each chunk size (MAC sources per pass), check that
    all candidates give identical ciphertexts, leave the fastest set in ctx.
    Returns {"best": c, "ms": {c: ms}}."""
    if F is None:
        from . import _lib as F
    return _tune_infer_knob(tuner, "linear_chunk", "chunk size", F.fhe_ctx_set_linear_chunk, candidates, ctx,
                            model, evk, cts, n_img, n_out, N, reps, F, device, model_key, sync)


def tune_mac_images(tuner: Tuner, ctx, model, evk, cts, n_img: int, n_out: int, N: int,
                    candidates: Sequence[int] = (1, 2, 4, 8), reps: int = 2, F=None,
                    device: Optional[str] = None, model_key: str = "", sync: Optional[Callable] = None) -> dict:
    """Images per block of the plaintext MAC (fhe_ctx_set_mac_images): a
    block's plaintext loads serve that many images, and the block covers
    512 / images coefficients of a limb.  Same protocol as tune_linear_chunk."""
    if F is None:
        from . import _lib as F
    return _tune_infer_knob(tuner, "mac_images", "images per MAC block", F.fhe_ctx_set_mac_images, candidates,
                            ctx, model, evk, cts, n_img, n_out, N, reps, F, device, model_key, sync)


def tune_keyswitch_batch(tuner: Tuner, ctx, model, evk, cts, n_img: int, n_out: int, N: int,
                         candidates: Sequence[int] = (0, 2, 4), reps: int = 2, F=None,
                         device: Optional[str] = None, model_key: str = "",
                         sync: Optional[Callable] = None) -> dict:
    """Items per launch of the whole key switches of a step
    (fhe_ctx_set_keyswitch_batch; 0: all of the batch at once): fewer items
    per launch shrink the workspace the passes stream, more share each key
    read.  Same protocol as tune_linear_chunk."""
    if F is None:
        from . import _lib as F
    return _tune_infer_knob(tuner, "keyswitch_batch", "key-switch batch", F.fhe_ctx_set_keyswitch_batch,
                            candidates, ctx, model, evk, cts, n_img, n_out, N, reps, F, device, model_key, sync)


def tune_pipeline_group(tuner: Tuner, ctx, model, evk, image_cts: Sequence[Sequence[int]], n_out: int, N: int,
                        candidates: Sequence[int] = (2, 4, 8), steps: int = 1, F=None,
                        device: Optional[str] = None, model_key: str = "",
                        sync: Optional[Callable] = None) -> dict:
    """Images per tick of the mixed-level pipeline (fhe_pipeline_*): for each
    candidate group g, one pipeline (only one alive at a time) is filled,
    then `steps` x S ticks of g images each are timed; throughput is the
    images that leave per second.  Bit-neutral: the first image's outputs
    must be identical for every candidate.  image_cts: the input ciphertext
    handles of each image (reused cyclically).  Returns {"best": g,
    "img_s": {g: img/s}}."""
    if F is None:
        from . import _lib as F
    if sync is None:
        import torch
        sync = torch.cuda.synchronize
    dev = device if device is not None else device_name()
    key = _key("pipeline_group", dev, model=model_key, cands=",".join(map(str, candidates)), steps=steps)
    hit = tuner.lookup(key)
    if hit is not None:
        return hit
    n_img = len(image_cts)
    ref = None
    rate: Dict[int, float] = {}
    refused: Dict[int, str] = {}
    for g in candidates:
        try:
            pipe = F.fhe_pipeline_create(ctx, model, evk, g, True)
        except F.FheError as e:
            if e.code != F.FHE_E_OOM:
                raise
            refused[g] = str(e)       # does not fit in device memory
            continue
        try:
            S = F.fhe_pipeline_info(pipe)[0]
            state = {"next": 0, "first": None}

            def tick():
                i0 = state["next"]
                grp = [h for i in range(g) for h in image_cts[(i0 + i) % n_img]]
                state["next"] += g
                outs, n_done, tag = F.fhe_pipeline_tick(pipe, grp, g, g * n_out)
                if n_done and tag == 0 and state["first"] is None:
                    state["first"] = [F.fhe_ct_export(h, N)[0] for h in outs[:n_out]]
                for h in outs:
                    F.fhe_ct_free(h)

            try:
                for _ in range(S):      # fill: the first group leaves at the last of these ticks
                    tick()
            except F.FheError as e:
                if e.code != F.FHE_E_OOM:
                    raise
                refused[g] = str(e)
                continue
            sync()
            t0 = time.perf_counter()
            for _ in range(steps * S):
                tick()
            sync()
            rate[g] = steps * S * g / (time.perf_counter() - t0)
        finally:
            F.fhe_pipeline_free(pipe)
        if ref is None:
            ref = state["first"]
        elif state["first"] is None or not all((a == b).all() for a, b in zip(ref, state["first"])):
            raise RuntimeError("group size %d changed the output ciphertexts" % g)
    if not rate:
        raise RuntimeError("no pipeline group size fits in device memory: %s" % refused)
    best = max(rate, key=lambda c: (rate[c], -c))
    return tuner.record(key, {"best": best, "img_s": {str(g): round(r, 4) for g, r in rate.items()},
                              "refused": {str(g): m for g, m in refused.items()}})
