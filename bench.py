"""Benchmark: encrypted ResNet-20 inference under leveled RNS-CKKS on GB300.

One step = one batched homomorphic inference of a batch of encrypted
32x32x3 images through the whole ResNet-20-shaped network (every
convolution, activation, rescale, shortcut, pool and dense layer: all the
hot-path operations), N = 2^16, 21 moduli of the ciphertext chain + 7
special primes (digit width 7).  Inputs are seeded synthetic images and
random weights.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B]
  python bench.py --impl reference ...   (the CPU oracle on a bounded sample)

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs an
independent replica on its own GPU; the work shards by image and needs no
exchange between ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "batched vs single encrypted img/s (ResNet-20 shape, N=2^16, bit-exact); % HBM"
PRESET = "resnet20"
KS_KERNELS = ["modup_intt_rows", "modup_intt_cols", "modup_conv_ntt_cols", "modup_ntt_rows_key_ip",
              "moddown_intt_rows", "moddown_intt_cols", "moddown_conv_ntt_cols", "moddown_ntt_rows_out"]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, device):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms: float, world: int, device: str = "cuda") -> float:
    """slowest rank's time: every rank contributes its own, all get the max"""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank: int, world: int, ms_max: float) -> float:
    """whole-job throughput: the units all ranks processed over the slowest
    rank's time (replicas, weak scaling)"""
    return units_per_rank * world / (ms_max / 1e3)


# Integer roofline.  The key switch and the plaintext MAC are bound by the
# 64-bit modular arithmetic on the integer pipes, not by HBM.  Algorithmic
# work is counted in modular multiplications (one per NTT butterfly, per
# basis-conversion term, per key inner-product term, per output scaling; one
# per plaintext-ciphertext product).  Peak: SMs x 64 32-bit integer
# multiply-adds per clock per SM (the integer multiply rate of the CUDA
# arithmetic-throughput table for compute capability 10.x: 4 sub-partitions x
# 16 lanes) x the SM clock sampled during the timed region, divided by the
# 10 multiply-adds of one 64-bit Shoup product (4 for the high 64 bits, 3 + 3
# for the two low products).
IMAD_PER_CLK_SM = 64
IMAD_PER_MODMUL = 10


def alu_peak_modmul(n_sm: int, sm_mhz: float) -> float:
    return n_sm * IMAD_PER_CLK_SM * sm_mhz * 1e6 / IMAD_PER_MODMUL


# DRAM bytes (read + write) of one top-level key switch of 4 polynomials,
# summed over its kernels from one ncu capture of the kernels as they are
# now (taken 2026-12-04, digit width 7, level 20); reported only for that
# configuration and only while those kernels are unchanged.
KS_TRAFFIC = {"bytes": 2719789568, "level": 20, "items": 8, "alpha": 7, "captured": "2026-12-04"}


def ks_parts(level, alpha, logn):
    """modular multiplications of the three phases of one hybrid key switch
    at `level`: (ModUp, key inner product, ModDown).  ModUp: inverse NTT of
    the level+1 limbs, basis conversion of every digit to the limbs outside
    it, their NTTs; inner product: two key polynomials per digit and
    extended limb; ModDown: inverse NTT of the special limbs of both
    polynomials, conversion to the level+1 limbs, their NTTs and the P^-1
    scaling."""
    N = 1 << logn
    bf = (N // 2) * logn
    nl = level + 1
    ext = nl + alpha
    digits = [min(alpha, nl - j) for j in range(0, nl, alpha)]
    nd = len(digits)
    modup = nl * bf + sum((ext - d) * d * N + (ext - d) * bf for d in digits)
    ip = 2 * nd * ext * N
    moddown = 2 * alpha * bf + 2 * nl * alpha * N + 2 * nl * bf + 2 * nl * N
    return modup, ip, moddown


def ks_modmuls(level, alpha, logn):
    """modular multiplications of one hybrid key switch at `level`"""
    return sum(ks_parts(level, alpha, logn))


def linear_ks_modmuls(level, alpha, logn, n_baby_inputs, n_babies, n_giants, n_giant_outputs, n_rot_groups=None):
    """key-switching work of one linear step with hoisting: the baby-step
    rotations of one input share its ModUp (each needs an inner product and
    a ModDown; with double hoisting, n_rot_groups given, the ModDowns are one
    per output group with rotated terms instead), the giant-step rotations
    of one output share its ModDown (each needs a ModUp and an inner
    product)"""
    mu, ip, md = ks_parts(level, alpha, logn)
    baby_md = n_babies * md if n_rot_groups is None else n_rot_groups * md
    return n_baby_inputs * mu + n_babies * ip + baby_md + n_giants * (mu + ip) + n_giant_outputs * md


def image_modmuls(prog, alpha, logn):
    """(key switches, their modular multiplications) of one image of a
    compiled program"""
    from paper_2509_22857_gb300 import model as M
    n_ks, mm = 0, 0
    for st in prog.steps:
        lv = prog.tensors[st["src"]].level
        if st["kind"] == 1:
            babies = {(int(i), int(b)) for i, b in zip(st["t_ct"], st["t_baby"]) if b}
            giants = {(int(o), int(g)) for o, g in zip(st["t_out"], st["t_giant"]) if g}
            rot_groups = {(int(o), int(g)) for o, g, b in zip(st["t_out"], st["t_giant"], st["t_baby"]) if b}
            mm += linear_ks_modmuls(lv, alpha, logn, len({i for i, _ in babies}), len(babies), len(giants),
                                    len({o for o, _ in giants}),
                                    len(rot_groups) if st.get("hoist", 1) == 2 else None)
            n_ks += len(babies) + len(giants)
        else:
            k = M.keyswitches_of_step(prog, st)
            n_ks += k
            mm += k * ks_modmuls(lv, alpha, logn)
    return n_ks, mm


def oracle_image_modmuls(prog, alpha, logn):
    """the same count on the oracle's program format"""
    mm = 0
    for st in prog.steps:
        src = st["src"][0] if isinstance(st["src"], list) else st["src"]
        t_in = prog.tensors[src]
        lv = t_in.level
        if st["op"] == "linear":
            babies = set(st["baby"])
            giants = {(o, g) for o, gs in st["groups"].items() for g in gs if g}
            rot_groups = {(o, g) for o, gs in st["groups"].items() for g, terms in gs.items()
                          if any(b for (_, b, _) in terms)}
            mm += linear_ks_modmuls(lv, alpha, logn, len({i for i, _ in babies}), len(babies), len(giants),
                                    len({o for o, _ in giants}),
                                    len(rot_groups) if st.get("hoist", 1) == 2 else None)
        elif st["op"] == "act":
            mm += t_in.layout.n_ct * ks_modmuls(lv, alpha, logn)
        elif st["op"] == "rotsum":
            mm += t_in.layout.n_ct * len(st["steps"]) * ks_modmuls(lv, alpha, logn)
    return mm


def _ext_limbs(prog, st, alpha):
    """limbs of a linear step's rotated terms: Q_l, or Q_l u P when the step
    is double-hoisted"""
    return prog.tensors[st["src"]].level + 1 + (alpha if st.get("hoist", 1) == 2 else 0)


def mac_products(prog, N, alpha):
    """plaintext-ciphertext products of one image (both polynomials, every
    active limb of every term; a double-hoisted step's rotated terms run over
    Q_l u P)"""
    total = 0
    for st in prog.steps:
        if st["kind"] == 1:
            nl = prog.tensors[st["src"]].level + 1
            n_rot = int(np.count_nonzero(st["t_baby"]))
            total += 2 * N * ((len(st["t_out"]) - n_rot) * nl + n_rot * _ext_limbs(prog, st, alpha))
    return total


def mac_bytes(prog, N, batch, alpha):
    """algorithmic HBM bytes of the MAC of a batch: every source ciphertext
    once per image, every distinct plaintext once per batch, every output
    ciphertext (a double-hoisted step: every group's sum over Q_l u P) once
    per image"""
    total = 0
    for st in prog.steps:
        if st["kind"] != 1:
            continue
        W = (prog.tensors[st["src"]].level + 1) * N * 8
        WX = _ext_limbs(prog, st, alpha) * N * 8
        n_in = len({int(i) for i, b in zip(st["t_ct"], st["t_baby"]) if not b})
        n_rot = len({(int(i), int(b)) for i, b in zip(st["t_ct"], st["t_baby"]) if b})
        n_out = prog.tensors[st["dst"]].layout.n_ct
        n_grp = len({(int(o), int(g)) for o, g, b in zip(st["t_out"], st["t_giant"], st["t_baby"]) if b}) \
            if st.get("hoist", 1) == 2 else 0
        total += batch * (2 * W * n_in + 2 * WX * n_rot + 2 * W * n_out + 2 * WX * n_grp) \
            + WX * len(st["vecs"]) + W * len(st["bias"])
    return total


def plaintext_bytes(prog, N, alpha):
    total = 0
    for st in prog.steps:
        if st["kind"] == 1:
            total += (len(st["vecs"]) * _ext_limbs(prog, st, alpha) + len(st["bias"]) * (
                prog.tensors[st["src"]].level + 1)) * N * 8
    return total


# ===================================================================== ours

def run_ours(args, rank, world):
    import torch
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import model as M

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    pre = synth.PRESETS[PRESET]
    N = 1 << pre["logn"]
    t0 = time.time()
    ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"],
                           pre["log_scale"], dev)
    F.fhe_ctx_set_mac_images(ctx, args.mac_images)
    net = synth.resnet20()
    raw = synth.params(net)
    prog = M.compile_network(net, raw, F.fhe_ctx_primes(ctx)[: pre["L"] + 1], pre["logn"], pre["log_scale"],
                             "packed", pre["alpha"], input_lambda=synth.INPUT_LAMBDA[PRESET])
    sk, evk = F.fhe_keygen(ctx, synth.SEED_KEYS, sorted(prog.rotations))
    desc = M.ModelDesc(prog, N // 2)
    model = F.fhe_model_load(ctx, desc.desc)
    t_setup = time.time() - t0
    n_in = prog.tensors[prog.input].layout.n_ct
    n_out = prog.tensors[prog.output].layout.n_ct
    B = args.batch

    # client side: encrypt B images (image index offset by rank: replicas see different images)
    cts = []
    for i in range(B):
        img = synth.image(rank * B + i, 3, 32, 32)
        for k, v in enumerate(M.input_slots(prog, img, N // 2)):
            pt = F.fhe_encode(ctx, v, M.input_scale(prog), pre["L"])
            cts.append(F.fhe_encrypt(ctx, sk, pt, synth.enc_seed(rank * B + i, k)))
            F.fhe_pt_free(pt)

    def infer(handles, n):
        outs = F.fhe_infer(ctx, model, evk, handles, n, n_out, stream)
        for h in outs:
            F.fhe_ct_free(h)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(fn, k):
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / k, world)

    if args.profile_uniform:
        # one uniform batch in the profiled NVTX range (same kernels as a
        # pipeline step, few enough launches for a serialised launch list)
        infer(cts, B)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("bench_timed")
        infer(cts, B)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_uniform": True, "batch": B}), flush=True)
        return None

    knob_tuning = None
    if args.tune_knobs:
        # images per MAC block and key-switch batch, timed on one pipeline
        # group's worth of images through the whole network (bit-neutral:
        # the tuner checks every value gives the same ciphertexts)
        from paper_2509_22857_gb300 import autotune as A
        tuner = A.Tuner(args.autotune_cache)
        nb = min(B, 8)
        knob_tuning = {
            "mac_images": A.tune_mac_images(tuner, ctx, model, evk, cts[:nb * n_in], nb, n_out, N,
                                            candidates=(0, 1, 2, 4, 8), reps=1, model_key=PRESET),
            "keyswitch_batch": A.tune_keyswitch_batch(tuner, ctx, model, evk, cts[:nb * n_in], nb, n_out, N,
                                                      candidates=(8, 4, 2), reps=1, model_key=PRESET)}

    # where the time goes: one uniform batch with events around every phase
    outs, phase_ms = F.fhe_infer_profiled(ctx, model, evk, cts, B, n_out, stream)
    for h in outs:
        F.fhe_ct_free(h)

    # single-image baseline (one image per launch sequence)
    for _ in range(max(1, args.warmup)):
        infer(cts[:n_in], 1)
    ms_single = timed(lambda: infer(cts[:n_in], 1), args.steps)

    # uniform batch: B images through the whole network together
    for _ in range(args.warmup):
        infer(cts, B)
    ms_uniform = timed(lambda: infer(cts, B), args.steps)

    # mixed levels: a pipeline of S segments with a group of g images entering
    # every tick, about B images in flight at S different levels; one step is
    # S ticks (as many images finish as one uniform pass of S*g images)
    probe = F.fhe_pipeline_create(ctx, model, evk, 1, False)
    S = F.fhe_pipeline_info(probe)[0]
    F.fhe_pipeline_free(probe)
    group_tuning = None
    if args.tune_group:
        from paper_2509_22857_gb300 import autotune as A
        images = [cts[i * n_in:(i + 1) * n_in] for i in range(B)]
        group_tuning = A.tune_pipeline_group(A.Tuner(args.autotune_cache), ctx, model, evk, images, n_out, N,
                                             candidates=(4, 8, 16), model_key=PRESET)
        g = group_tuning["best"]
    elif args.group:
        g = args.group
    else:
        g = max(1, -(-B // S))
    pipe = F.fhe_pipeline_create(ctx, model, evk, g, True)
    state = {"next": 0}

    def tick(handles_of):
        i0 = state["next"] % B
        grp = [h for i in range(g) for h in handles_of((i0 + i) % B)]
        state["next"] += g
        outs, n_done, _ = F.fhe_pipeline_tick(pipe, grp, g, g * n_out)
        for h in outs:
            F.fhe_ct_free(h)

    # one step = T ticks; a group of g images leaves per tick once the
    # pipeline is full (every tick runs every segment, full or not)
    T = args.ticks if args.ticks > 0 else S

    def pipe_step():
        for _ in range(T):
            tick(lambda i: cts[i * n_in:(i + 1) * n_in])

    for _ in range(max(args.warmup, -(-S // T))):     # at least one fill of the pipeline
        pipe_step()
    clk = Clocks(dev)
    clk.start()
    l0 = F.fhe_kernel_launches()
    torch.cuda.nvtx.range_push("bench_timed")
    ms_batch = timed(pipe_step, args.steps)
    torch.cuda.nvtx.range_pop()
    launches = (F.fhe_kernel_launches() - l0) // args.steps
    clocks = clk.stop()

    # end to end through the public API with host buffers: every tick imports
    # its group (H2D + NTT), runs, and exports the finished group (inverse
    # NTT + D2H)
    host_in = [F.fhe_ct_export(h, N)[0] for h in cts]
    lvl_in, sc_in = pre["L"], M.input_scale(prog)

    def e2e_step():
        for _ in range(T):
            i0 = state["next"] % B
            hs = [F.fhe_ct_import(ctx, host_in[((i0 + i) % B) * n_in + k], lvl_in, sc_in)
                  for i in range(g) for k in range(n_in)]
            state["next"] += g
            outs, n_done, _ = F.fhe_pipeline_tick(pipe, hs, g, g * n_out)
            for h in outs:
                F.fhe_ct_export(h, N)
                F.fhe_ct_free(h)
            for h in hs:
                F.fhe_ct_free(h)

    ms_e2e = timed(e2e_step, max(1, args.steps))
    F.fhe_pipeline_free(pipe)
    out_level = prog.tensors[prog.output].level
    h2d = T * g * n_in * 2 * (pre["L"] + 1) * N * 8
    d2h = T * g * n_out * 2 * (out_level + 1) * N * 8

    # key-switch roofline at the top level, batch of B (the pipeline that
    # dominates the step): algorithmic bytes per switched polynomial =
    # (l+1)W in + 2*beta*(l+1+alpha)W key / B + 2(l+1)W out, W = N*8
    lv = pre["L"]
    ks_ms = F.fhe_profile_keyswitch(ctx, evk, lv, g, 3, stream)
    alpha = pre["alpha"]
    beta = (lv + alpha) // alpha
    W = N * 8
    ks_bytes = g * ((lv + 1) * W + 2 * (lv + 1) * W) + 2 * beta * (lv + 1 + alpha) * W
    ks_total = sum(ks_ms) / 1e3
    peak, peak_kind = _peaks()
    achieved = ks_bytes / ks_total / 1e9
    ks_mm = g * ks_modmuls(lv, alpha, pre["logn"])
    alu_achieved = ks_mm / ks_total
    # the integer peak at this GPU's SM count and the clock sampled under load
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    alu_peak = alu_peak_modmul(n_sm, sm_mhz)
    traffic = KS_TRAFFIC["bytes"] if (KS_TRAFFIC["bytes"] and g == KS_TRAFFIC["items"] and lv == KS_TRAFFIC["level"]
                                      and alpha == KS_TRAFFIC["alpha"]) else None
    # the MAC of the uniform batch (its phase timed with events on the stream)
    mac_mm = B * mac_products(prog, N, pre["alpha"])
    mac_s = phase_ms["linear_mac"] / 1e3
    mac_b = mac_bytes(prog, N, B, pre["alpha"])
    img_s_batch = aggregate_throughput(T * g, world, ms_batch)
    img_s_uniform = aggregate_throughput(B, world, ms_uniform)
    img_s_single = aggregate_throughput(1, world, ms_single)
    n_ks, img_mm = image_modmuls(prog, alpha, pre["logn"])

    res = {
        "metric": METRIC,
        "value": round(img_s_batch, 4),
        "unit": "img/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_batch, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic",
        "config": {
            "workload": "ResNet-20 (16/32/64, 3x3 blocks, 1x1 stride-2 shortcuts), 32x32x3 seeded uniform "
                        "images, 10 classes; CKKS N=2^16, Delta=2^%d, q0 %d-bit + %d x %d-bit, %d x %d-bit "
                        "special primes, digit width %d (dnum %d); channel-packed layout"
                        % (pre["log_scale"], pre["q0_bits"], pre["L"], pre["q_bits"], pre["alpha"], pre["p_bits"],
                           pre["alpha"], -(-(pre["L"] + 1) // pre["alpha"])),
            "batch": T * g,
            "in_flight": S * g,
            "mixed_levels": True,
            "pipeline": "%d segments (cut after each activation), a group of %d images enters per tick, %d ticks "
                        "per step; segments run on concurrent streams, each tick replayed from a CUDA graph"
                        % (S, g, T),
            "group_tuning": group_tuning,
            "knob_tuning": knob_tuning,
            "mac_images_per_block": args.mac_images if knob_tuning is None else knob_tuning["mac_images"]["best"],
            "hoisting": "per linear step by the cost model: %d of %d double-hoisted" % (
                sum(1 for h in M.hoists(prog) if h == 2), len(M.hoists(prog))),
            "uniform_batch": B,
            "uniform_batch_img_s": round(img_s_uniform, 4),
            "single_img_s": round(img_s_single, 4),
            "single_ms_per_img": round(ms_single, 3),
            "batched_over_single": round(img_s_batch / img_s_single, 4),
            "keyswitches_per_img": n_ks,
            "l2": "inputs larger than L2: every tick streams the %.1f GB of resident weight plaintexts once "
                  "(each segment its own layers'), %.0f GB per step; L2 is 0.13 GB"
                  % (plaintext_bytes(prog, N, pre["alpha"]) / 1e9, T * plaintext_bytes(prog, N, pre["alpha"]) / 1e9),
            "setup_s": round(t_setup, 1),
            "uniform_batch_phase_ms": {k: round(v, 1) for k, v in phase_ms.items()},
            "parallelism": "replicas" if world > 1 else "single",
        },
        "clocks": clocks,
        "e2e": {"value": round(aggregate_throughput(T * g, world, ms_e2e), 4), "unit": "img/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu",
                     "kernel": "hybrid key switch (ModUp, key inner product, exact ModDown), level %d, "
                               "%d polynomials (one group of the pipeline), timed by CUDA events on its stream "
                               "right after the timed region" % (lv, g),
                     "achieved": round(alu_achieved / 1e9, 1), "peak": round(alu_peak / 1e9, 1),
                     "unit": "Gmodmul/s",
                     "peak_kind": "derived: %d SMs x %d IMAD/clk x %.0f MHz (median sampled SM clock) / %d IMAD "
                                  "per 64-bit Shoup product" % (n_sm, IMAD_PER_CLK_SM, sm_mhz, IMAD_PER_MODMUL),
                     "frac": round(alu_achieved / alu_peak, 4),
                     "traffic": traffic,
                     "traffic_from": (("ncu capture of these kernels, %s" % KS_TRAFFIC["captured"]) if traffic
                                      else "no capture of the current kernels at this configuration"),
                     "algorithmic_modmuls": int(ks_mm),
                     "hbm": {"achieved_gbs": round(achieved, 1), "peak_gbs": peak, "peak_kind": peak_kind,
                             "frac": round(achieved / peak, 4), "algorithmic_bytes": int(ks_bytes)},
                     "kernel_ms": {k: round(v, 4) for k, v in zip(KS_KERNELS, ks_ms)},
                     "mac": {"kernel": "plaintext MAC of the linear layers, uniform batch of %d (phase timed by "
                                       "CUDA events)" % B,
                             "achieved": round(mac_mm / mac_s / 1e9, 1), "peak": round(alu_peak / 1e9, 1),
                             "unit": "Gmodmul/s", "frac": round(mac_mm / mac_s / alu_peak, 4),
                             "algorithmic_products": int(mac_mm),
                             "hbm": {"achieved_gbs": round(mac_b / mac_s / 1e9, 1), "peak_gbs": peak,
                                     "frac": round(mac_b / mac_s / 1e9 / peak, 4),
                                     "algorithmic_bytes": int(mac_b)}}},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(img_mm, pre)
    F.fhe_model_free(model)
    for h in cts:
        F.fhe_ct_free(h)
    F.fhe_evk_free(evk)
    F.fhe_sk_free(sk)
    F.fhe_ctx_destroy(ctx)
    return res


# ===================================================================== oracle

def oracle_rotation_seconds(pre, level):
    """the CPU oracle, as it stands: one rotation of a fresh ciphertext at `level`"""
    from oracle import ckks as O
    prm = O.make_params(**pre)
    S = O.CKKS(prm)
    keys = S.keygen(synth.SEED_KEYS, [1])
    z = np.random.default_rng(0).uniform(-1, 1, prm.N // 2)
    ct = S.encrypt(keys, S.encode(z, prm.scale, level), 5)
    t0 = time.perf_counter()
    S.rotate(ct, 1, keys)
    return time.perf_counter() - t0, S, keys, ct


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_worker(pre, level, barrier, q):
    """one process of the throughput sample: set up, wait for the others,
    then time one rotation (wall-clock start and end)"""
    _, S, keys, ct = oracle_rotation_seconds(pre, level)
    barrier.wait()
    t0 = time.time()
    S.rotate(ct, 1, keys)
    q.put((t0, time.time()))


def oracle_rotation_throughput(pre, level, procs):
    """rotations per second of `procs` oracle processes running at once (one
    rotation each, started together)"""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    q = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(pre, level, barrier, q)) for _ in range(procs)]
    for p in ps:
        p.start()
    spans = [q.get(timeout=600) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    return procs / (max(e for _, e in spans) - min(t for t, _ in spans))


def cpu_baseline(img_mm, pre):
    """The CPU oracle as it stands on this host: one top-level rotation on one
    core, and the rotations per second of one process per core running at
    once; both scaled to images by the image's key-switching work (modular
    multiplications of the hoisted program, in units of one top-level
    rotation)."""
    unit = ks_modmuls(pre["L"], pre["alpha"], pre["logn"])
    rot_per_img = img_mm / unit
    secs = oracle_rotation_seconds(pre, pre["L"])[0]
    nproc = os.cpu_count() or 1
    procs = max(1, min(nproc, 32))
    rps = oracle_rotation_throughput(pre, pre["L"], procs)
    return {"value": round(rps / rot_per_img, 8), "unit": "img/s", "cores": procs, "kind": "oracle",
            "nproc": nproc, "cpu_model": _cpu_model(),
            "single_core_img_s": round(1.0 / (secs * rot_per_img), 8),
            "sample": "hybrid-key-switch rotations at the top level (N=2^16, 21 + %d primes) on the CPU oracle: "
                      "one on one core (%.1f s), then one per process in %d processes at once (%.3f rotations/s); "
                      "scaled to images by the image's key-switching work with hoisting (%.0f top-level "
                      "rotation equivalents); plaintext products and additions not counted" %
                      (pre["alpha"], secs, procs, rps, rot_per_img)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from oracle import ckks as O
    from oracle import cnn
    pre = synth.PRESETS[PRESET]
    prm = O.make_params(**dict(pre, logn=12))      # the plan depends on the primes' sizes only
    net = synth.resnet20()
    raw = synth.params(net)
    # the same baby-step / giant-step schedule as the GPU arm (host planning only)
    from paper_2509_22857_gb300 import model as M
    lam = synth.INPUT_LAMBDA[PRESET]
    plan = M.compile_network(net, raw, prm.q, pre["logn"], pre["log_scale"], "packed", pre["alpha"],
                             input_lambda=lam)
    comp = cnn.Compiler(prm, "packed", M.giant_steps(plan), 1, lam, M.hoists(plan))
    comp.n = 1 << (pre["logn"] - 1)
    prog = comp.compile(net, cnn.transform(net, raw))
    unit = oracle_image_modmuls(prog, pre["alpha"], pre["logn"]) / ks_modmuls(pre["L"], pre["alpha"], pre["logn"])
    _, S, keys, ct = oracle_rotation_seconds(pre, pre["L"])
    for _ in range(args.warmup):
        S.rotate(ct, 1, keys)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S.rotate(ct, 1, keys)
    secs = (time.perf_counter() - t0) / args.steps
    v = 1.0 / (secs * unit)
    return {"impl": "reference", "metric": METRIC, "value": round(v, 8), "unit": "img/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": "ResNet-20, N=2^16 (as the GPU arm); each step one top-level rotation of the "
                                   "CPU oracle, scaled to img/s by the image's weighted key-switch count"},
            "cpu_baseline": {"value": round(v, 8), "unit": "img/s", "cores": 1, "kind": "oracle",
                             "sample": "one top-level rotation per step"},
            "e2e": {"value": round(v, 8), "unit": "img/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_resnet18(args):
    """ResNet-18 for 64x64x3 / 200 classes, an ensemble of 3 members in the
    HW layout (member m in block m), weights clustered jointly to 16 values
    per layer: one uniform batch of `batch` images through the whole network
    (fhe_infer); its logits are checked against the float64 ensemble in
    tests/test_gpu_fullsize.py."""
    import torch
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import model as M
    pre = synth.PRESETS["resnet18"]
    N = 1 << pre["logn"]
    B = args.batch
    t0 = time.time()
    ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"],
                           pre["log_scale"], 0)
    net = synth.resnet18()
    M_members = args.members
    raws = synth.cluster_joint([synth.params(net, m) for m in range(M_members)], net, 16)
    prog = M.compile_network(net, raws, F.fhe_ctx_primes(ctx)[: pre["L"] + 1], pre["logn"], pre["log_scale"],
                             "hw_ens", pre["alpha"], input_lambda=synth.INPUT_LAMBDA["resnet18"])
    sk, evk = F.fhe_keygen(ctx, synth.SEED_KEYS, sorted(prog.rotations))
    desc = M.ModelDesc(prog, N // 2)
    model = F.fhe_model_load(ctx, desc.desc)
    if args.chunk:
        F.fhe_ctx_set_linear_chunk(ctx, args.chunk)
    # whole key switches of a step (an activation of B x 64 channel
    # ciphertexts) in launches of 64 items: the workspace stays 6.4 GB
    F.fhe_ctx_set_keyswitch_batch(ctx, 64)
    t_setup = time.time() - t0
    n_out = prog.tensors[prog.output].layout.n_ct
    cts = []
    for i in range(B):
        img = synth.image(i, 3, 64, 64)
        for k, v in enumerate(M.input_slots(prog, img, N // 2)):
            pt = F.fhe_encode(ctx, v, M.input_scale(prog), pre["L"])
            cts.append(F.fhe_encrypt(ctx, sk, pt, synth.enc_seed(i, k)))
            F.fhe_pt_free(pt)
    stream = torch.cuda.current_stream()
    # one batch, timed by events on the stream (the phase split comes from
    # events around each phase of the same run)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    outs, phase_ms = F.fhe_infer_profiled(ctx, model, evk, cts, B, n_out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n_ks, _ = image_modmuls(prog, pre["alpha"], pre["logn"])
    res = {"workload": "ResNet-18 ensemble of %d (64x64x3, 200 classes), HW layout, 16 joint clusters per layer; "
                       "CKKS N=2^16, 19 + %d primes" % (M_members, pre["alpha"]),
           "members": M_members,
           "batch": B, "img_s": round(B / (ms / 1e3), 4), "ms_per_batch": round(ms, 1),
           "phase_ms": {k: round(v, 1) for k, v in phase_ms.items()}, "setup_s": round(t_setup, 1),
           "linear_chunk_sources": args.chunk or 160,
           "keyswitches_per_img": n_ks, "distinct_plaintexts": sum(len(st["vecs"]) for st in prog.steps
                                                                  if st["kind"] == 1)}
    print(json.dumps(res), flush=True)
    for h in outs + cts:
        F.fhe_ct_free(h)
    F.fhe_model_free(model)
    F.fhe_evk_free(evk)
    F.fhe_sk_free(sk)
    F.fhe_ctx_destroy(ctx)


def run_vgg11(args):
    """VGG-11 (configuration A: 8 convolutions, 5 average pools, 3 dense
    layers) on 32x32x3 images, channel-packed, N = 2^16: the packed
    convolutions' plaintexts (239K rows, about 0.86 TB if encoded at once)
    are encoded on the device each time their layer runs; the dense layers'
    plaintexts stay resident.  One uniform batch through the whole network
    (fhe_infer) and its phase split (its logits are checked against the
    float64 network in tests/test_gpu_fullsize.py)."""
    import torch
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import model as M
    pre = synth.PRESETS["vgg11"]
    N = 1 << pre["logn"]
    B = args.batch
    t0 = time.time()
    ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"],
                           pre["log_scale"], 0)
    net = synth.vgg11()
    raw = synth.params(net)
    prog = M.compile_network(net, raw, F.fhe_ctx_primes(ctx)[: pre["L"] + 1], pre["logn"], pre["log_scale"],
                             "packed", pre["alpha"], input_lambda=synth.INPUT_LAMBDA["vgg11"], on_demand=True)
    t_compile = time.time() - t0
    sk, evk = F.fhe_keygen(ctx, synth.SEED_KEYS, sorted(prog.rotations))
    desc = M.ModelDesc(prog, N // 2)
    model = F.fhe_model_load(ctx, desc.desc)
    t_setup = time.time() - t0
    n_out = prog.tensors[prog.output].layout.n_ct
    cts = []
    for i in range(B):
        img = synth.image(i, 3, 32, 32)
        for k, v in enumerate(M.input_slots(prog, img, N // 2)):
            pt = F.fhe_encode(ctx, v, M.input_scale(prog), pre["L"])
            cts.append(F.fhe_encrypt(ctx, sk, pt, synth.enc_seed(i, k)))
            F.fhe_pt_free(pt)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    outs, phase_ms = F.fhe_infer_profiled(ctx, model, evk, cts, B, n_out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n_ks, _ = image_modmuls(prog, pre["alpha"], pre["logn"])
    rows = sum(len(st["vecs"]) for st in prog.steps if st["kind"] == 1 and st["vecs"]
               and isinstance(st["vecs"][0], M.SparseVec))
    res = {"workload": "VGG-11 (config A, 8 conv + 3 dense, 32x32x3, 10 classes), channel-packed; CKKS N=2^16, "
                       "%d + %d primes; packed convolutions' plaintexts encoded on demand" % (pre["L"] + 1,
                                                                                            pre["alpha"]),
           "batch": B, "img_s": round(B / (ms / 1e3), 4), "ms_per_batch": round(ms, 1),
           "phase_ms": {k: round(v, 1) for k, v in phase_ms.items()}, "compile_s": round(t_compile, 1),
           "setup_s": round(t_setup, 1), "keyswitches_per_img": n_ks, "rows_encoded_on_demand": rows,
           "resident_plaintext_gb": round(plaintext_bytes(prog, N, pre["alpha"]) / 1e9 - sum(
               len(st["vecs"]) * _ext_limbs(prog, st, pre["alpha"]) * N * 8 for st in prog.steps
               if st["kind"] == 1 and st["vecs"] and isinstance(st["vecs"][0], M.SparseVec)) / 1e9, 2)}
    print(json.dumps(res), flush=True)
    for h in outs + cts:
        F.fhe_ct_free(h)
    F.fhe_model_free(model)
    F.fhe_evk_free(evk)
    F.fhe_sk_free(sk)
    F.fhe_ctx_destroy(ctx)


def run_resnet32(args):
    """ResNet-32 (3 stages x 5 basic blocks) on 32x32x3 images on the
    paper's own parameter set for it (appendix "Details on FHE Parameters",
    Table 4: N = 2^16, Delta = 2^26, a 27-bit q_0 and 32 primes of ~52 bits,
    one 54-bit special prime, so every prime is its own key-switching digit:
    33 digits at the top level), channel-packed: one uniform batch through the
    whole network (fhe_infer) and its phase split."""
    import torch
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import model as M
    pp = synth.PAPER_PARAMS["resnet32"]
    N = 1 << pp["logn"]
    B = args.batch
    t0 = time.time()
    ctx = F.fhe_ctx_create(pp["logn"], pp["L"], 0, 0, 0, pp["alpha"], pp["log_scale"], 0, primes=pp["q"] + pp["p"])
    net = synth.resnet32()
    raw = synth.params(net)
    prog = M.compile_network(net, raw, pp["q"], pp["logn"], pp["log_scale"], "packed", pp["alpha"], input_lambda=2)
    sk, evk = F.fhe_keygen(ctx, synth.SEED_KEYS, sorted(prog.rotations))
    desc = M.ModelDesc(prog, N // 2)
    model = F.fhe_model_load(ctx, desc.desc)
    t_setup = time.time() - t0
    n_out = prog.tensors[prog.output].layout.n_ct
    cts = []
    for i in range(B):
        img = synth.image(i, 3, 32, 32)
        for k, v in enumerate(M.input_slots(prog, img, N // 2)):
            pt = F.fhe_encode(ctx, v, M.input_scale(prog), pp["L"])
            cts.append(F.fhe_encrypt(ctx, sk, pt, synth.enc_seed(i, k)))
            F.fhe_pt_free(pt)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    outs, phase_ms = F.fhe_infer_profiled(ctx, model, evk, cts, B, n_out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n_ks, _ = image_modmuls(prog, pp["alpha"], pp["logn"])
    res = {"workload": "ResNet-32 (16/32/64, 3x5 blocks), 32x32x3, 10 classes, channel-packed, on the paper's "
                       "ResNet-32 parameter set: N=2^16, Delta=2^26, 27-bit q0 + 32 x ~52-bit, one 54-bit P "
                       "(33 digits)",
           "batch": B, "img_s": round(B / (ms / 1e3), 5), "s_per_img": round(ms / 1e3 / B, 3),
           "ms_per_batch": round(ms, 1), "phase_ms": {k: round(v, 1) for k, v in phase_ms.items()},
           "setup_s": round(t_setup, 1), "keyswitches_per_img": n_ks,
           "plaintext_gb": round(plaintext_bytes(prog, N, pp["alpha"]) / 1e9, 1),
           "paper_cpu_s_per_img": {"value": 1833, "note": "ResNet-32 / CIFAR-10, slice clustering k=64, "
                                                          "2x AMD EPYC 64-core, SEAL 4.1 (context only)"}}
    print(json.dumps(res), flush=True)
    for h in outs + cts:
        F.fhe_ct_free(h)
    F.fhe_model_free(model)
    F.fhe_evk_free(evk)
    F.fhe_sk_free(sk)
    F.fhe_ctx_destroy(ctx)


def run_serving(args):
    """Serving stream: Poisson arrivals (rate args.rate) of single-image
    requests drawn 50/30/20 from VGG-, ResNet-20- and ResNet-18-ensemble-
    shaped models, submitted to the continuous-batching server at their
    arrival times; reports p50 / p99 latency and the images per second
    completed.  --serving-size small: their small forms (one ring N = 2^12);
    full: the full-size models at N = 2^16 in one context (ResNet-20's
    21-prime chain; VGG-11 and the ResNet-18 ensemble are compiled on its
    first 12 and 19 primes, VGG-11 with its convolutions' plaintexts encoded
    on demand)."""
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import model as M
    full = args.serving_size == "full"
    pre = synth.PRESETS["resnet20" if full else "resnet18_mini"]
    N = 1 << pre["logn"]
    ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"],
                           pre["log_scale"], 0)
    chain = F.fhe_ctx_primes(ctx)
    if full:
        # every pipeline segment keeps its own encode scratch (1 GiB each)
        # and its rotated copies (chunks of 40 sources; bit-neutral)
        F.fhe_ctx_set_encode_scratch(ctx, 1 << 30)
        F.fhe_ctx_set_linear_chunk(ctx, 40)
        # and its key-switch workspace (8 items per launch)
        F.fhe_ctx_set_keyswitch_batch(ctx, 8)
        # (arch, layout, members, levels, on demand, clusters)
        specs = [("vgg11", "packed", None, synth.PRESETS["vgg11"]["L"], True, 0),
                 ("resnet20", "packed", None, pre["L"], False, 0),
                 ("resnet18", "hw_ens", 3, synth.PRESETS["resnet18"]["L"], False, 16)]
    else:
        specs = [("vgg_mini", "packed", None, pre["L"], False, 0), ("resnet_mini", "packed", None, pre["L"], False, 0),
                 ("resnet18_mini", "hw_ens", 3, pre["L"], False, 4)]
    progs, rots = [], set()
    for arch, layout, members, lv, od, k in specs:
        net = synth.ARCHS[arch]()
        raw = synth.cluster_joint([synth.params(net, m) for m in range(members)], net, k) if members else \
            synth.params(net)
        progs.append((net, M.compile_network(net, raw, chain[: lv + 1], pre["logn"], pre["log_scale"], layout,
                                             pre["alpha"], input_lambda=2 if full else 1, on_demand=od)))
        rots |= progs[-1][1].rotations
    sk, evk = F.fhe_keygen(ctx, synth.SEED_KEYS, sorted(rots))
    descs = [M.ModelDesc(p, N // 2) for _, p in progs]
    models = [F.fhe_model_load(ctx, d.desc) for d in descs]
    server = F.fhe_server_create(ctx, evk)
    # admission by device memory: a model whose pipeline does not fit is
    # refused (FHE_E_OOM) and the stream is served by the admitted ones
    mids, refused = [], []
    for k, m in enumerate(models):
        try:
            mids.append(F.fhe_server_add_model(server, m, 1 if full else 4))
        except F.FheError as e:
            if e.code != F.FHE_E_OOM:
                raise
            mids.append(None)
            refused.append({"model": specs[k][0], "error": str(e)})
    mix = np.array([0.5, 0.3, 0.2]) * np.array([mid is not None for mid in mids])
    rng = np.random.default_rng(5)
    n_req = args.requests
    which = rng.choice(3, size=n_req, p=mix / mix.sum())
    gaps = rng.exponential(1.0 / args.rate, size=n_req)
    # client side: every request's image encrypted before the stream starts
    reqs = []
    for r in range(n_req):
        net, prog = progs[which[r]]
        inp = net[0]
        img = synth.image(r, inp["c"], inp["h"], inp["w"])
        cts = []
        for k, v in enumerate(M.input_slots(prog, img, N // 2)):
            pt = F.fhe_encode(ctx, v, M.input_scale(prog), prog.tensors[prog.input].level)
            cts.append(F.fhe_encrypt(ctx, sk, pt, synth.enc_seed(r, k)))
            F.fhe_pt_free(pt)
        reqs.append(cts)
    t0 = time.perf_counter()
    t_next = t0
    tickets = []
    for r in range(n_req):
        t_next += gaps[r]
        d = t_next - time.perf_counter()
        if d > 0:
            time.sleep(d)
        tickets.append(F.fhe_server_submit(server, mids[which[r]], reqs[r]))
    lat = []
    for r, t in enumerate(tickets):
        n_out = progs[which[r]][1].tensors[progs[which[r]][1].output].layout.n_ct
        outs, ms = F.fhe_server_poll(server, t, True, n_out)
        lat.append(ms)
        for h in outs:
            F.fhe_ct_free(h)
    t_end = time.perf_counter()
    done, p50, p99 = F.fhe_server_stats(server)
    def pct(k, q):
        v = [l for l, w in zip(lat, which) if w == k]
        return round(float(np.percentile(v, q)), 2) if v else None

    per_model = {specs[k][0]: {"requests": int((which == k).sum()), "p50_ms": pct(k, 50), "p99_ms": pct(k, 99)}
                 for k in range(3)}
    print(json.dumps({"workload": "serving: Poisson %.2f req/s, %d single-image requests, 50/30/20 VGG / ResNet-20 / "
                                  "ResNet-18-ensemble shapes (%s, N=2^%d, %d primes)"
                                  % (args.rate, n_req, "full size" if full else "small forms", pre["logn"],
                                     pre["L"] + 1 + pre["alpha"]),
                      "refused_models": refused,
                      "completed": done, "p50_ms": round(p50, 2), "p99_ms": round(p99, 2),
                      "img_s": round(done / (t_end - t0), 3), "per_model": per_model}), flush=True)
    F.fhe_server_destroy(server)
    for m in models:
        F.fhe_model_free(m)
    F.fhe_evk_free(evk)
    F.fhe_sk_free(sk)
    F.fhe_ctx_destroy(ctx)


def run_ks_only(args):
    """Only the hybrid key switch at the top level for `batch` items (small
    device footprint: the relinearisation key and the workspace); used for
    detailed profiles of the key-switching kernels."""
    import torch
    from paper_2509_22857_gb300 import _lib as F
    pre = dict(synth.PRESETS[PRESET])
    if args.alpha is not None:
        pre["alpha"] = args.alpha
    ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"],
                           pre["log_scale"], 0)
    sk, evk = F.fhe_keygen(ctx, synth.SEED_KEYS, [])
    level = pre["L"] if args.ks_level is None else args.ks_level
    ms = F.fhe_profile_keyswitch(ctx, evk, level, args.batch, max(1, args.steps), torch.cuda.current_stream())
    print(json.dumps({"level": level, "alpha": pre["alpha"], "items": args.batch,
                      "kernel_ms": dict(zip(KS_KERNELS, ms)),
                      "total_ms": sum(ms), "us_per_item": sum(ms) / args.batch * 1e3}))
    F.fhe_evk_free(evk)
    F.fhe_sk_free(sk)
    F.fhe_ctx_destroy(ctx)


def run_autotune(args):
    """Rank the admissible digit widths (dnum) for the ResNet-20 parameters by
    measured key-switch time, weighted by how many key switches one image
    performs at each level; print the table as one JSON line."""
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import autotune as A
    from paper_2509_22857_gb300 import model as M
    pre = dict(synth.PRESETS[PRESET])
    ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"],
                           pre["log_scale"], 0)
    primes = F.fhe_ctx_primes(ctx)[: pre["L"] + 1]
    F.fhe_ctx_destroy(ctx)
    net = synth.ARCHS[PRESET]()
    prog = M.compile_network(net, synth.params(net), primes, pre["logn"], pre["log_scale"], "packed",
                             pre["alpha"], input_lambda=synth.INPUT_LAMBDA[PRESET])
    levels = A.keyswitch_levels(prog)
    tuner = A.Tuner(args.autotune_cache)
    t0 = time.time()
    rec = A.tune_digit_width(tuner, pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"],
                             pre["log_scale"], candidates=range(1, 9), levels=levels, items=4, iters=5)
    top = {a: v[str(pre["L"])] for a, v in rec["us"].items()}
    print(json.dumps({"autotune": "digit_width", "preset": PRESET, "preset_alpha": pre["alpha"],
                      "device": A.device_name(), "keyswitch_levels": levels, "best": rec["best"],
                      "cost_us_per_img": rec["cost_us"], "top_level_us": top,
                      "top_level_best": int(min(top, key=lambda a: top[a])), "tune_s": round(time.time() - t0, 1)}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ks-only", action="store_true", help="time only the top-level key switch")
    ap.add_argument("--ks-level", type=int, default=None)
    ap.add_argument("--alpha", type=int, default=None, help="--ks-only: digit width (special primes)")
    ap.add_argument("--workload", default="resnet20", choices=["resnet20", "resnet18_ensemble", "vgg11", "resnet32", "serving"],
                    help="resnet18_ensemble: one batch of the clustered ResNet-18 ensemble; serving: a Poisson "
                         "request stream through the server (neither is the bench line)")
    ap.add_argument("--profile-uniform", action="store_true",
                    help="run one uniform batch inside the NVTX range bench_timed and exit (for ncu launch lists)")
    ap.add_argument("--members", type=int, default=3, help="resnet18_ensemble: ensemble members (1..8)")
    ap.add_argument("--chunk", type=int, default=0,
                    help="resnet18_ensemble: MAC sources per linear chunk (0: the library's default, 160)")
    ap.add_argument("--requests", type=int, default=1000, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=20.0, help="serving: mean arrivals per second")
    ap.add_argument("--serving-size", default="small", choices=["small", "full"],
                    help="serving: the models' small forms (N=2^12) or full size (N=2^16)")
    ap.add_argument("--autotune", action="store_true",
                    help="rank the admissible digit widths by measured, census-weighted key-switch time and exit")
    ap.add_argument("--autotune-cache", default=None, help="--autotune: JSON cache file of the tuner")
    ap.add_argument("--group", type=int, default=8,
                    help="images per pipeline tick (8: the best of 4, 8, 16 measured by --tune-group on GB300; "
                         "0: the uniform batch spread over the segments)")
    ap.add_argument("--ticks", type=int, default=5,
                    help="pipeline ticks per timed step (every tick runs every segment, i.e. the whole network, "
                         "for the group at each level; a group of images leaves per tick)")
    ap.add_argument("--mac-images", type=int, default=1,
                    help="images per plaintext-MAC block (1: the best of 0, 1, 2, 4, 8 measured by --tune-knobs on "
                         "GB300 for ResNet-20, 8 images; bit-neutral)")
    ap.add_argument("--tune-knobs", action="store_true",
                    help="measure images per MAC block and the key-switch batch on the device first (reported)")
    ap.add_argument("--tune-group", action="store_true",
                    help="pick the pipeline's images per tick by measurement (2, 4, 8) before the timed run")
    args = ap.parse_args()
    if args.autotune:
        run_autotune(args)
        return
    if args.ks_only:
        run_ks_only(args)
        return
    if args.workload == "resnet18_ensemble":
        run_resnet18(args)
        return
    if args.workload == "vgg11":
        run_vgg11(args)
        return
    if args.workload == "resnet32":
        run_resnet32(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
