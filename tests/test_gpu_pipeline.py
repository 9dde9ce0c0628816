"""Continuous batching with images at mixed levels: groups entering a
pipeline tick by tick (some ticks empty, partial groups) leave with exactly
the ciphertexts that one-image fhe_infer produces; with and without CUDA
graph replay."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mini():
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import model as M
    pre = synth.PRESETS["resnet_mini"]
    N = 1 << pre["logn"]
    ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"],
                           pre["log_scale"])
    net = synth.resnet_mini()
    prog = M.compile_network(net, synth.params(net), F.fhe_ctx_primes(ctx)[: pre["L"] + 1], pre["logn"],
                             pre["log_scale"], "packed",
                             pre["alpha"])
    sk, evk = F.fhe_keygen(ctx, synth.SEED_KEYS, sorted(prog.rotations))
    desc = M.ModelDesc(prog, N // 2)
    model = F.fhe_model_load(ctx, desc.desc)

    def encrypt(i):
        img = synth.image(i, 3, 8, 8)
        cts = []
        for k, v in enumerate(M.input_slots(prog, img, N // 2)):
            pt = F.fhe_encode(ctx, v, 2.0 ** pre["log_scale"], pre["L"])
            cts.append(F.fhe_encrypt(ctx, sk, pt, synth.enc_seed(i, k)))
            F.fhe_pt_free(pt)
        return cts

    yield F, ctx, model, evk, encrypt, N
    F.fhe_model_free(model)
    F.fhe_evk_free(evk)
    F.fhe_sk_free(sk)
    F.fhe_ctx_destroy(ctx)


@pytest.mark.parametrize("graphs", [True, False])
def test_pipeline_equals_alone(mini, graphs):
    F, ctx, model, evk, encrypt, N = mini
    group = 2
    pipe = F.fhe_pipeline_create(ctx, model, evk, group, graphs)
    S, g, n_in_ct, n_out_ct = F.fhe_pipeline_info(pipe)
    assert S >= 3 and g == group
    # arrival pattern: full, partial, empty, full, then drain
    pattern = [2, 1, 0, 2] + [0] * S
    next_img = 0
    entries = {}
    got = {}
    for tick, cnt in enumerate(pattern):
        imgs = list(range(next_img, next_img + cnt))
        next_img += cnt
        cts = [h for i in imgs for h in encrypt(i)]
        entries[tick] = imgs
        outs, n_out, tag = F.fhe_pipeline_tick(pipe, cts, cnt, group * n_out_ct)
        if n_out:
            assert tag >= 0 and len(entries[tag]) == n_out
            for j, i in enumerate(entries[tag]):
                got[i] = [F.fhe_ct_export(h, N)[0] for h in outs[j * n_out_ct:(j + 1) * n_out_ct]]
        for h in outs + cts:
            F.fhe_ct_free(h)
    assert sorted(got) == list(range(next_img))
    for i in range(next_img):
        cts = encrypt(i)
        alone = F.fhe_infer(ctx, model, evk, cts, 1, n_out_ct)
        for a, b in zip(alone, got[i]):
            assert np.array_equal(F.fhe_ct_export(a, N)[0], b), i
            F.fhe_ct_free(a)
        for h in cts:
            F.fhe_ct_free(h)
    F.fhe_pipeline_free(pipe)


def test_refused_output_allocation_keeps_the_groups_aligned(mini):
    """A tick whose output ciphertexts cannot be allocated is refused before
    launch: nothing enters, the tick is not counted, and the group due to
    leave leaves at the next call with the ciphertexts it gets alone."""
    F, ctx, model, evk, encrypt, N = mini
    pipe = F.fhe_pipeline_create(ctx, model, evk, 1, True)
    S, g, n_in_ct, n_out_ct = F.fhe_pipeline_info(pipe)
    entries, got = {}, {}

    def tick(imgs, cts):
        t = F.fhe_pipeline_ticks(pipe)
        outs, n_out, tag = F.fhe_pipeline_tick(pipe, cts, len(imgs), n_out_ct)
        entries[t] = imgs
        if n_out:
            assert entries[tag] and len(entries[tag]) == n_out
            got[entries[tag][0]] = [F.fhe_ct_export(h, N)[0] for h in outs]
        for h in outs:
            F.fhe_ct_free(h)

    for i in range(S - 1):
        cts = encrypt(i)
        tick([i], cts)
        for h in cts:
            F.fhe_ct_free(h)
    assert not got
    cts = encrypt(S - 1)
    before = F.fhe_pipeline_ticks(pipe)
    F.fhe_ctx_inject_alloc_failure(ctx, 0)    # the leaving image's output ciphertext
    with pytest.raises(F.FheError) as e:
        F.fhe_pipeline_tick(pipe, cts, 1, n_out_ct)
    assert e.value.code == F.FHE_E_OOM
    assert F.fhe_pipeline_ticks(pipe) == before
    tick([S - 1], cts)
    assert sorted(got) == [0]
    for h in cts:
        F.fhe_ct_free(h)
    for _ in range(S):
        tick([], [])
    assert sorted(got) == list(range(S))
    for i in range(S):
        cts = encrypt(i)
        alone = F.fhe_infer(ctx, model, evk, cts, 1, n_out_ct)
        for a, b in zip(alone, got[i]):
            assert np.array_equal(F.fhe_ct_export(a, N)[0], b), i
            F.fhe_ct_free(a)
        for h in cts:
            F.fhe_ct_free(h)
    F.fhe_pipeline_free(pipe)
