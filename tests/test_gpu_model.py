"""Whole networks on the GPU through the C ABI: output ciphertexts bit-equal
to the oracle's, decrypted logits within 1e-3 of the float64 network with
the same argmax, batching and per-layer entry points consistent."""
import numpy as np
import pytest

import synth
from oracle import ckks as O
from oracle import cnn

pytestmark = pytest.mark.gpu

# (arch, preset, layout[, input scale as a power of Delta[, hoisting mode]]);
# the planner's default mode ("auto") picks double hoisting for most linear
# steps of these networks, "mini_single" keeps every step single-hoisted
CASES = {"tiny": ("tiny", "tiny", "hw"), "mini": ("resnet_mini", "resnet_mini", "packed", 2),
         "mini_single": ("resnet_mini", "resnet_mini", "packed", 2, 1),
         "vgg_mini": ("vgg_mini", "resnet_mini", "packed"),
         # pre-activation blocks: batch norm fused into the activation after
         # it, per-channel quadratic coefficients (node fusing Case 1)
         "preact": ("preact_mini", "resnet_mini", "packed"),
         # ResNet-18's structure, an ensemble of 3 in the HW layout, weights
         # clustered jointly to 4 values per layer
         "ens": ("resnet18_mini", "resnet18_mini", "hw_ens")}
ENSEMBLE = 3


class Setup:
    def __init__(self, case):
        from paper_2509_22857_gb300 import _lib as F
        from paper_2509_22857_gb300 import model as M
        arch, preset, layout = CASES[case][:3]
        lam = CASES[case][3] if len(CASES[case]) > 3 else 1
        hoist = CASES[case][4] if len(CASES[case]) > 4 else "auto"
        self.F, self.M = F, M
        self.net = synth.ARCHS[arch]()
        if layout == "hw_ens":
            self.raws = synth.cluster_joint([synth.params(self.net, m) for m in range(ENSEMBLE)], self.net, 4)
            self.raw = self.raws
            t = [cnn.transform(self.net, r) for r in self.raws]
        else:
            self.raws = None
            self.raw = synth.params(self.net)
            t = cnn.transform(self.net, self.raw)
        pre = synth.PRESETS[preset]
        self.pre = pre
        self.prm = O.make_params(**pre)
        self.S = O.CKKS(self.prm)
        self.ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"],
                                    pre["alpha"], pre["log_scale"])
        self.pm = M.compile_network(self.net, self.raw, F.fhe_ctx_primes(self.ctx)[: pre["L"] + 1], pre["logn"],
                                    pre["log_scale"], layout, pre["alpha"], input_lambda=lam, hoist=hoist)
        # the oracle evaluates the same diagonals with the package's baby-step
        # / giant-step split and hoisting modes
        self.po = cnn.compile_he(self.net, t, self.prm, layout, M.giant_steps(self.pm),
                                 ENSEMBLE if layout == "hw_ens" else 1, lam, M.hoists(self.pm))
        self._oracle_cache = {}
        self.keys = self.S.keygen(synth.SEED_KEYS, sorted(self.po.rot_steps))
        self.sk, self.evk = F.fhe_keygen(self.ctx, synth.SEED_KEYS, sorted(self.pm.rotations))
        self.desc = M.ModelDesc(self.pm, self.prm.N // 2)
        self.model = F.fhe_model_load(self.ctx, self.desc.desc)
        self.inp = self.net[0]

    def encrypt(self, i):
        F, M = self.F, self.M
        img = synth.image(i, self.inp["c"], self.inp["h"], self.inp["w"])
        out = []
        for k, v in enumerate(M.input_slots(self.pm, img, self.prm.N // 2)):
            pt = F.fhe_encode(self.ctx, v, M.input_scale(self.pm), self.prm.L)
            out.append(F.fhe_encrypt(self.ctx, self.sk, pt, synth.enc_seed(i, k)))
            F.fhe_pt_free(pt)
        return img, out

    def oracle_outputs(self, i):
        if i not in self._oracle_cache:
            img = synth.image(i, self.inp["c"], self.inp["h"], self.inp["w"])
            cts = cnn.encrypt_input(self.S, self.keys, self.po, img, i, synth.enc_seed)
            self._oracle_cache[i] = cnn.run_he(self.S, self.keys, self.po, cts)
        return self._oracle_cache[i]

    def reference_logits(self, img):
        if self.raws is not None:
            return cnn.forward_ensemble(self.net, self.raws, img)
        return cnn.forward_plain(self.net, self.raw, img)

    def coef(self, ct):
        prm = self.prm
        return np.stack([np.stack([O.intt(ct.c[r, t], prm.primes[t], prm.psi[t]) for t in range(ct.level + 1)])
                         for r in range(ct.c.shape[0])])

    def logits(self, handles):
        F = self.F
        vals = []
        for ct, slot in self.M.logit_slots(self.pm):
            pt = F.fhe_decrypt(self.ctx, self.sk, handles[ct])
            z = F.fhe_decode(self.ctx, pt, self.prm.N // 2)
            F.fhe_pt_free(pt)
            vals.append(z[slot].real)
        return np.array(vals)

    def close(self):
        F = self.F
        F.fhe_model_free(self.model)
        F.fhe_evk_free(self.evk)
        F.fhe_sk_free(self.sk)
        F.fhe_ctx_destroy(self.ctx)


@pytest.fixture(scope="module", params=list(CASES))
def setup(request):
    s = Setup(request.param)
    yield s
    s.close()


def test_network_bit_exact_and_logits(setup):
    s = setup
    F = s.F
    img, cts = s.encrypt(0)
    n_out = s.pm.tensors[s.pm.output].layout.n_ct
    outs = F.fhe_infer(s.ctx, s.model, s.evk, cts, 1, n_out)
    ref = s.oracle_outputs(0)[s.po.output_tensor]
    for h, r in zip(outs, ref):
        buf, lv, sc = F.fhe_ct_export(h, s.prm.N)
        assert lv == r.level and sc == r.scale
        assert np.array_equal(buf, s.coef(r))
    y = s.logits(outs)
    want = s.reference_logits(img)
    assert np.max(np.abs(y - want)) < 1e-3
    assert np.argmax(y) == np.argmax(want)
    for h in outs + cts:
        F.fhe_ct_free(h)


def test_batched_equals_one_at_a_time(setup):
    s = setup
    F = s.F
    n_out = s.pm.tensors[s.pm.output].layout.n_ct
    imgs = [s.encrypt(i)[1] for i in range(3)]
    flat = [h for cts in imgs for h in cts]
    batched = F.fhe_infer(s.ctx, s.model, s.evk, flat, 3, n_out)
    for i in range(3):
        single = F.fhe_infer(s.ctx, s.model, s.evk, imgs[i], 1, n_out)
        for a, b in zip(single, batched[i * n_out:(i + 1) * n_out]):
            assert np.array_equal(F.fhe_ct_export(a, s.prm.N)[0], F.fhe_ct_export(b, s.prm.N)[0])
            F.fhe_ct_free(a)
    for h in batched + flat:
        F.fhe_ct_free(h)


def test_per_layer_entry_points(setup):
    """fhe_eval_conv / fhe_eval_quad_act / fhe_eval_pool_dense on one image
    reproduce the oracle's tensors of those steps."""
    s = setup
    F = s.F
    ref = s.oracle_outputs(0)
    kinds = [st["kind"] for st in s.pm.steps]
    # first linear step (a convolution), the first activation (the first
    # with per-channel coefficients where the network has one), the first rotsum
    vec_act = [i for i, st in enumerate(s.pm.steps) if st["kind"] == 3 and "c1_vecs" in st]
    for kind, call in ((1, "conv"), (3, "act"), (4, "pool")):
        i = vec_act[0] if kind == 3 and vec_act else kinds.index(kind)
        st = s.pm.steps[i]
        so = s.po.steps[i]
        ins = ref[so["src"]]
        handles = []
        for ct in ins:
            handles.append(F.fhe_ct_import(s.ctx, s.coef(ct), ct.level, ct.scale))
        n_out = s.pm.tensors[st["dst"]].layout.n_ct
        if call == "conv":
            outs = F.fhe_eval_conv(s.ctx, s.model, s.evk, i, handles, n_out)
        elif call == "pool":
            outs = F.fhe_eval_pool_dense(s.ctx, s.model, s.evk, i, handles, n_out)
        else:
            F.fhe_eval_quad_act(s.ctx, s.model, s.evk, i, handles)
            outs, handles = handles, []
        for h, r in zip(outs, ref[so["dst"]]):
            assert np.array_equal(F.fhe_ct_export(h, s.prm.N)[0], s.coef(r)), (call, i)
            F.fhe_ct_free(h)
        for h in handles:
            F.fhe_ct_free(h)


def test_keyswitch_item_cap_changes_nothing(setup):
    """Whole key switches of a step (activations, rotate-and-sum) split into
    launches of at most 2 items give the ciphertexts of one launch."""
    s = setup
    F = s.F
    n_out = s.pm.tensors[s.pm.output].layout.n_ct
    imgs = [s.encrypt(i)[1] for i in range(3)]
    flat = [h for cts in imgs for h in cts]
    whole = F.fhe_infer(s.ctx, s.model, s.evk, flat, 3, n_out)
    F.fhe_ctx_set_keyswitch_batch(s.ctx, 2)
    try:
        parts = F.fhe_infer(s.ctx, s.model, s.evk, flat, 3, n_out)
    finally:
        F.fhe_ctx_set_keyswitch_batch(s.ctx, 0)
    for a, b in zip(whole, parts):
        assert np.array_equal(F.fhe_ct_export(a, s.prm.N)[0], F.fhe_ct_export(b, s.prm.N)[0])
    for h in whole + parts + flat:
        F.fhe_ct_free(h)


def test_chunked_linear_steps_change_nothing(setup):
    """Linear steps split into chunks of few sources (rotated copies made and
    consumed a chunk at a time, MAC outputs accumulated over chunks) give
    the same ciphertexts as one chunk."""
    s = setup
    F = s.F
    n_out = s.pm.tensors[s.pm.output].layout.n_ct
    img, cts = s.encrypt(0)
    whole = F.fhe_infer(s.ctx, s.model, s.evk, cts, 1, n_out)
    F.fhe_ctx_set_linear_chunk(s.ctx, 5)
    try:
        parts = F.fhe_infer(s.ctx, s.model, s.evk, cts, 1, n_out)
    finally:
        F.fhe_ctx_set_linear_chunk(s.ctx, 160)
    for a, b in zip(whole, parts):
        assert np.array_equal(F.fhe_ct_export(a, s.prm.N)[0], F.fhe_ct_export(b, s.prm.N)[0])
    for h in whole + parts + cts:
        F.fhe_ct_free(h)
    with pytest.raises(F.FheError):
        F.fhe_ctx_set_linear_chunk(s.ctx, 1)


def test_batch_of_nine_equals_one_at_a_time(setup):
    """Nine images: the MAC runs 8 images per CTA (the shape of the bench's
    uniform batch and of the ResNet-18 batch of 32) plus a ragged CTA of one
    image; every image equals its one-image run (image 0 equals the oracle
    in test_network_bit_exact_and_logits)."""
    s = setup
    F = s.F
    n_out = s.pm.tensors[s.pm.output].layout.n_ct
    B = 9
    imgs = [s.encrypt(i)[1] for i in range(B)]
    flat = [h for cts in imgs for h in cts]
    batched = F.fhe_infer(s.ctx, s.model, s.evk, flat, B, n_out)
    for i in range(B):
        single = F.fhe_infer(s.ctx, s.model, s.evk, imgs[i], 1, n_out)
        for a, b in zip(single, batched[i * n_out:(i + 1) * n_out]):
            assert np.array_equal(F.fhe_ct_export(a, s.prm.N)[0], F.fhe_ct_export(b, s.prm.N)[0]), i
            F.fhe_ct_free(a)
    for h in batched + flat:
        F.fhe_ct_free(h)


@pytest.mark.parametrize("case", ["mini", "vgg_mini"])
def test_oracle_chosen_schedule_bit_exact(case):
    """The oracle compiles the network with a baby-step / giant-step split it
    chooses itself (its default: one block per convolution, eight for the
    packed dense layer), the GPU program is compiled with that split in
    place of its planner's, and the output ciphertexts are equal: the GPU
    path is checked on a schedule its own planner did not produce."""
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import model as M
    arch, preset, layout = CASES[case][:3]
    lam = CASES[case][3] if len(CASES[case]) > 3 else 1
    net = synth.ARCHS[arch]()
    raw = synth.params(net)
    pre = synth.PRESETS[preset]
    prm = O.make_params(**pre)
    S = O.CKKS(prm)
    po = cnn.compile_he(net, cnn.transform(net, raw), prm, layout, None, 1, lam)
    own = [st["giant"] for st in po.steps if st["op"] == "linear"]
    ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"],
                           pre["log_scale"])
    try:
        planned = M.giant_steps(M.compile_network(net, raw, F.fhe_ctx_primes(ctx)[: pre["L"] + 1], pre["logn"],
                                                  pre["log_scale"], layout, pre["alpha"], input_lambda=lam))
        # the oracle's own default split, single-hoisted like the oracle's default
        pm = M.compile_network(net, raw, F.fhe_ctx_primes(ctx)[: pre["L"] + 1], pre["logn"], pre["log_scale"],
                               layout, pre["alpha"], input_lambda=lam, giants=own, hoist=1)
        assert M.giant_steps(pm) == own
        if case == "mini":
            assert own != planned     # the planner would have split differently
        assert pm.rotations == po.rot_steps
        keys = S.keygen(synth.SEED_KEYS, sorted(po.rot_steps))
        sk, evk = F.fhe_keygen(ctx, synth.SEED_KEYS, sorted(pm.rotations))
        desc = M.ModelDesc(pm, prm.N // 2)
        model = F.fhe_model_load(ctx, desc.desc)
        inp = net[0]
        img = synth.image(2, inp["c"], inp["h"], inp["w"])
        cts = []
        for k, v in enumerate(M.input_slots(pm, img, prm.N // 2)):
            pt = F.fhe_encode(ctx, v, M.input_scale(pm), pre["L"])
            cts.append(F.fhe_encrypt(ctx, sk, pt, synth.enc_seed(2, k)))
            F.fhe_pt_free(pt)
        n_out = pm.tensors[pm.output].layout.n_ct
        outs = F.fhe_infer(ctx, model, evk, cts, 1, n_out)
        ref = cnn.run_he(S, keys, po, cnn.encrypt_input(S, keys, po, img, 2, synth.enc_seed))[po.output_tensor]
        for h, r in zip(outs, ref):
            buf, lv, sc = F.fhe_ct_export(h, prm.N)
            assert lv == r.level and sc == r.scale
            want = np.stack([np.stack([O.intt(r.c[p, t], prm.primes[t], prm.psi[t]) for t in range(r.level + 1)])
                             for p in range(2)])
            assert np.array_equal(buf, want)
        for h in outs + cts:
            F.fhe_ct_free(h)
        F.fhe_model_free(model)
        F.fhe_evk_free(evk)
        F.fhe_sk_free(sk)
    finally:
        F.fhe_ctx_destroy(ctx)


@pytest.mark.parametrize("case", ["mini", "mini_single", "vgg_mini", "preact"])
def test_on_demand_encoding_equals_resident(case):
    """The same network with its packed convolutions' plaintexts encoded on
    the device each time a step runs (sparse rows, host encoder's operation
    order) gives the ciphertexts of the resident program, with a scratch so
    small that every step runs its output groups in several batches, and
    through the graph-replayed pipeline as well."""
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import model as M
    arch, preset, layout = CASES[case][:3]
    lam = CASES[case][3] if len(CASES[case]) > 3 else 1
    hoist = CASES[case][4] if len(CASES[case]) > 4 else "auto"
    net = synth.ARCHS[arch]()
    raw = synth.params(net)
    pre = synth.PRESETS[preset]
    N = 1 << pre["logn"]
    ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"],
                           pre["log_scale"])
    try:
        primes = F.fhe_ctx_primes(ctx)[: pre["L"] + 1]
        pm = M.compile_network(net, raw, primes, pre["logn"], pre["log_scale"], layout, pre["alpha"],
                               input_lambda=lam, hoist=hoist)
        po = M.compile_network(net, raw, primes, pre["logn"], pre["log_scale"], layout, pre["alpha"],
                               input_lambda=lam, on_demand=True, hoist=hoist)
        assert M.hoists(po) == M.hoists(pm)
        assert any(st["kind"] == 1 and isinstance(st["vecs"][0], M.SparseVec) for st in po.steps)
        sk, evk = F.fhe_keygen(ctx, synth.SEED_KEYS, sorted(pm.rotations))
        dm, do = M.ModelDesc(pm, N // 2), M.ModelDesc(po, N // 2)
        m_res, m_od = F.fhe_model_load(ctx, dm.desc), F.fhe_model_load(ctx, do.desc)
        inp = net[0]
        cts = []
        for i in range(2):
            img = synth.image(i, inp["c"], inp["h"], inp["w"])
            for k, v in enumerate(M.input_slots(pm, img, N // 2)):
                pt = F.fhe_encode(ctx, v, M.input_scale(pm), pre["L"])
                cts.append(F.fhe_encrypt(ctx, sk, pt, synth.enc_seed(i, k)))
                F.fhe_pt_free(pt)
        n_out = pm.tensors[pm.output].layout.n_ct
        n_in = len(cts) // 2
        want_h = F.fhe_infer(ctx, m_res, evk, cts, 2, n_out)
        want = [F.fhe_ct_export(h, N)[0] for h in want_h]
        # a few rows per batch: (lv + 2) N words of scratch per row
        F.fhe_ctx_set_encode_scratch(ctx, 5 * (pre["L"] + 2) * N * 8)
        got_h = F.fhe_infer(ctx, m_od, evk, cts, 2, n_out)
        got = [F.fhe_ct_export(h, N)[0] for h in got_h]
        assert all(np.array_equal(a, b) for a, b in zip(want, got))
        pipe = F.fhe_pipeline_create(ctx, m_od, evk, 1, True)
        S = F.fhe_pipeline_info(pipe)[0]
        outs = []
        for t in range(S + 1):
            grp = cts[:n_in] if t == 0 else []
            o, n_done, tag = F.fhe_pipeline_tick(pipe, grp, len(grp) // n_in, n_out)
            if n_done:
                assert tag == 0
                outs = [F.fhe_ct_export(h, N)[0] for h in o]
            for h in o:
                F.fhe_ct_free(h)
        F.fhe_pipeline_free(pipe)
        assert outs and all(np.array_equal(a, b) for a, b in zip(want[:n_out], outs))
        for h in got_h + want_h + cts:
            F.fhe_ct_free(h)
        F.fhe_model_free(m_res)
        F.fhe_model_free(m_od)
        F.fhe_evk_free(evk)
        F.fhe_sk_free(sk)
    finally:
        F.fhe_ctx_destroy(ctx)
