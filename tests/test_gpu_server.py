"""Serving with continuous batching: requests for two models, submitted
while earlier ones are on the GPU, come back with exactly the ciphertexts each
image gets alone; latency statistics are reported."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_stalled_worker_times_out_then_completes():
    """A paused server (its host worker stalled) leaves a request pending:
    a bounded poll returns FHE_E_TIMEOUT and the request stays queued; after
    resuming, it completes with the ciphertexts the image gets alone."""
    from paper_2509_22857_gb300 import _lib as F
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
    n_out = prog.tensors[prog.output].layout.n_ct

    def encrypt():
        cts = []
        for k, v in enumerate(M.input_slots(prog, synth.image(0, 3, 8, 8), N // 2)):
            pt = F.fhe_encode(ctx, v, M.input_scale(prog), pre["L"])
            cts.append(F.fhe_encrypt(ctx, sk, pt, synth.enc_seed(0, k)))
            F.fhe_pt_free(pt)
        return cts

    server = F.fhe_server_create(ctx, evk)
    try:
        mid = F.fhe_server_add_model(server, model, 2)
        F.fhe_server_pause(server, True)
        t = F.fhe_server_submit(server, mid, encrypt())
        with pytest.raises(F.FheError) as e:
            F.fhe_server_poll(server, t, 100, n_out)
        assert e.value.code == F.FHE_E_TIMEOUT
        assert F.fhe_server_poll(server, t, False, n_out)[0] == []
        F.fhe_server_pause(server, False)
        outs, lat = F.fhe_server_poll(server, t, True, n_out)
        assert len(outs) == n_out and lat >= 100
        cts = encrypt()
        alone = F.fhe_infer(ctx, model, evk, cts, 1, n_out)
        for a, b in zip(alone, outs):
            assert np.array_equal(F.fhe_ct_export(a, N)[0], F.fhe_ct_export(b, N)[0])
        for h in alone + outs + cts:
            F.fhe_ct_free(h)
        assert F.fhe_server_stats(server)[0] == 1
    finally:
        F.fhe_server_destroy(server)
        F.fhe_model_free(model)
        F.fhe_evk_free(evk)
        F.fhe_sk_free(sk)
        F.fhe_ctx_destroy(ctx)


def test_server_results_equal_alone():
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import model as M
    pre = synth.PRESETS["resnet_mini"]
    N = 1 << pre["logn"]
    ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"],
                           pre["log_scale"])
    primes = F.fhe_ctx_primes(ctx)[: pre["L"] + 1]
    models, progs, descs = [], [], []
    rots = set()
    for arch in ("resnet_mini", "vgg_mini"):
        net = synth.ARCHS[arch]()
        prog = M.compile_network(net, synth.params(net), primes, pre["logn"], pre["log_scale"], "packed",
                                 pre["alpha"])
        progs.append(prog)
        rots |= prog.rotations
    sk, evk = F.fhe_keygen(ctx, synth.SEED_KEYS, sorted(rots))
    for prog in progs:
        descs.append(M.ModelDesc(prog, N // 2))
        models.append(F.fhe_model_load(ctx, descs[-1].desc))

    def encrypt(prog, i):
        img = synth.image(i, 3, 8, 8)
        cts = []
        for k, v in enumerate(M.input_slots(prog, img, N // 2)):
            pt = F.fhe_encode(ctx, v, 2.0 ** pre["log_scale"], pre["L"])
            cts.append(F.fhe_encrypt(ctx, sk, pt, synth.enc_seed(i, k)))
            F.fhe_pt_free(pt)
        return cts

    server = F.fhe_server_create(ctx, evk)
    try:
        _serve(F, ctx, evk, server, models, progs, encrypt, N)
    finally:
        F.fhe_server_destroy(server)
        for m in models:
            F.fhe_model_free(m)
        F.fhe_evk_free(evk)
        F.fhe_sk_free(sk)
        F.fhe_ctx_destroy(ctx)


def _serve(F, ctx, evk, server, models, progs, encrypt, N):
    mids = [F.fhe_server_add_model(server, m, 2) for m in models]
    # a stream of requests: model picked round robin with a 2:1 mix, small
    # random gaps so later requests arrive while earlier ones are in flight
    rng = np.random.default_rng(5)
    plan = [(0 if k % 3 != 2 else 1, k) for k in range(9)]
    tickets = []
    for mi, img in plan:
        tickets.append((mi, img, F.fhe_server_submit(server, mids[mi], encrypt(progs[mi], img))))
        time.sleep(float(rng.exponential(0.01)))
    for mi, img, t in tickets:
        n_out = progs[mi].tensors[progs[mi].output].layout.n_ct
        outs, lat = F.fhe_server_poll(server, t, True, n_out)
        assert len(outs) == n_out and lat > 0
        cts = encrypt(progs[mi], img)
        alone = F.fhe_infer(ctx, models[mi], evk, cts, 1, n_out)
        for a, b in zip(alone, outs):
            assert np.array_equal(F.fhe_ct_export(a, N)[0], F.fhe_ct_export(b, N)[0]), (mi, img)
        for h in alone + outs + cts:
            F.fhe_ct_free(h)
    done, p50, p99 = F.fhe_server_stats(server)
    assert done == len(plan) and 0 < p50 <= p99
    # an unknown ticket is an error, not a hang
    with pytest.raises(F.FheError):
        F.fhe_server_poll(server, 10 ** 9, False, 1)
