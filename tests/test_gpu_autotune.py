"""The autotuner on the device: every admissible digit width timed and
ranked, the cache answering a second tuner; the linear chunk size and the
pipeline's group size tuned on a small network with identical outputs across
candidates."""
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_digit_width_tuning_on_device(tmp_path):
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import autotune as A
    path = str(tmp_path / "tune.json")
    kw = dict(logn=12, L=6, q_bits=50, q0_bits=40, p_bits=58, log_scale=25, candidates=(1, 2, 3),
              levels=[(6, 1.0), (2, 3.0)], items=2, iters=2)
    rec = A.tune_digit_width(A.Tuner(path), **kw)
    # width 1 has 7 digits at L = 6 and P = 58 bits covers a 50-bit digit: all three admissible
    assert set(rec["us"]) == {"1", "2", "3"} and rec["best"] in (1, 2, 3)
    assert all(v > 0 for per in rec["us"].values() for v in per.values())
    assert rec["cost_us"][str(rec["best"])] == min(rec["cost_us"].values())

    class NoTiming:
        def __getattr__(self, name):
            if name == "fhe_profile_keyswitch":
                raise AssertionError("the cache should have answered")
            return getattr(F, name)

    assert A.tune_digit_width(A.Tuner(path), F=NoTiming(), **kw) == rec


def test_linear_chunk_tuning_keeps_outputs():
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import autotune as A
    from paper_2509_22857_gb300 import model as M
    pre = synth.PRESETS["resnet_mini"]
    N = 1 << pre["logn"]
    ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"],
                           pre["log_scale"])
    net = synth.resnet_mini()
    prog = M.compile_network(net, synth.params(net), F.fhe_ctx_primes(ctx)[: pre["L"] + 1], pre["logn"],
                             pre["log_scale"], "packed", pre["alpha"])
    sk, evk = F.fhe_keygen(ctx, synth.SEED_KEYS, sorted(prog.rotations))
    desc = M.ModelDesc(prog, N // 2)
    model = F.fhe_model_load(ctx, desc.desc)
    cts = []
    try:
        for i in range(2):
            img = synth.image(i, 3, 8, 8)
            for k, v in enumerate(M.input_slots(prog, img, N // 2)):
                pt = F.fhe_encode(ctx, v, M.input_scale(prog), pre["L"])
                cts.append(F.fhe_encrypt(ctx, sk, pt, synth.enc_seed(i, k)))
                F.fhe_pt_free(pt)
        n_out = prog.tensors[prog.output].layout.n_ct
        # raises if a chunk size changes any output ciphertext
        rec = A.tune_linear_chunk(A.Tuner(), ctx, model, evk, cts, 2, n_out, N, candidates=(4, 160), reps=1,
                                  model_key="resnet_mini")
        assert rec["best"] in (4, 160) and all(t > 0 for t in rec["ms"].values())
        # images per MAC block and key-switch batch: raise if a value changes any output
        rec = A.tune_mac_images(A.Tuner(), ctx, model, evk, cts, 2, n_out, N, candidates=(0, 1, 2, 4, 8), reps=1,
                                model_key="resnet_mini")
        assert rec["best"] in (0, 1, 2, 4, 8)
        rec = A.tune_keyswitch_batch(A.Tuner(), ctx, model, evk, cts, 2, n_out, N, candidates=(0, 1), reps=1,
                                     model_key="resnet_mini")
        assert rec["best"] in (0, 1)
        with pytest.raises(F.FheError):
            F.fhe_ctx_set_mac_images(ctx, 3)
        # the pipeline's group size: raises if a group size changes image 0's outputs
        n_in = len(cts) // 2
        images = [cts[i * n_in:(i + 1) * n_in] for i in range(2)]
        rec = A.tune_pipeline_group(A.Tuner(), ctx, model, evk, images, n_out, N, candidates=(1, 2, 4),
                                    model_key="resnet_mini")
        assert rec["best"] in (1, 2, 4) and all(r > 0 for r in rec["img_s"].values())
    finally:
        for h in cts:
            F.fhe_ct_free(h)
        F.fhe_model_free(model)
        F.fhe_evk_free(evk)
        F.fhe_sk_free(sk)
        F.fhe_ctx_destroy(ctx)
