"""The paper's own parameter set for ResNet-32 (its printed chain: q_0 of 28
bits, 32 primes of ~52 bits, one 54-bit special prime, so 33 key-switching
digits) on the device, at N = 2^12 (the primes are = 1 mod 2^17): rotation,
relinearised square, rescales and a double-hoisted convolution bit-equal to
the oracle's; chains the library must refuse."""
import numpy as np
import pytest

import paper_chains
from oracle import ckks as O

pytestmark = pytest.mark.gpu

LOGN = 12


@pytest.fixture(scope="module")
def paper():
    from paper_2509_22857_gb300 import _lib as F
    _, d, q, p = paper_chains.chain("ResNet-32")
    prm = O.Params(LOGN, q, p, 1, 2.0 ** d)
    ctx = F.fhe_ctx_create(LOGN, prm.L, 0, 0, 0, 1, d, primes=q + p)
    S = O.CKKS(prm)
    steps = [1, -1, 5]
    keys = S.keygen(11, steps)
    sk, evk = F.fhe_keygen(ctx, 11, steps)
    yield F, ctx, prm, S, keys, sk, evk
    F.fhe_evk_free(evk)
    F.fhe_sk_free(sk)
    F.fhe_ctx_destroy(ctx)


def _same(F, S, ct_o, ct_g):
    prm = S.prm
    buf, lv, sc = F.fhe_ct_export(ct_g, prm.N)
    ref = np.stack([np.stack([O.intt(ct_o.c[r, t], prm.primes[t], prm.psi[t]) for t in range(ct_o.level + 1)])
                    for r in range(ct_o.c.shape[0])])
    assert lv == ct_o.level and sc == ct_o.scale and np.array_equal(buf, ref)


def test_chain_is_taken_as_given(paper):
    F, ctx, prm, S, keys, sk, evk = paper
    assert F.fhe_ctx_primes(ctx) == prm.primes
    assert len(prm.digits(prm.L)) == 33


def test_keyswitching_with_33_digits_bit_exact(paper):
    F, ctx, prm, S, keys, sk, evk = paper
    z = np.random.default_rng(2).uniform(-1, 1, prm.N // 2)
    scale = prm.scale ** 3
    ct_o = S.encrypt(keys, S.encode(z, scale, prm.L), 21)
    pt = F.fhe_encode(ctx, z, scale, prm.L)
    ct_g = F.fhe_encrypt(ctx, sk, pt, 21)
    F.fhe_pt_free(pt)
    _same(F, S, ct_o, ct_g)
    for step in (1, -1, 5):
        r = F.fhe_rotate(ctx, evk, ct_g, step)
        _same(F, S, S.rotate(ct_o, step, keys), r)
        F.fhe_ct_free(r)
    sq_o = S.relinearize(S.tensor_square(ct_o), keys)
    sq_g = F.fhe_square(ctx, evk, ct_g)
    _same(F, S, sq_o, sq_g)
    # rescales down the chain, the last onto the 28-bit q_0
    for _ in range(prm.L):
        sq_o = S.rescale(sq_o)
        F.fhe_rescale(ctx, sq_g)
    _same(F, S, sq_o, sq_g)
    for h in (sq_g, ct_g):
        F.fhe_ct_free(h)


def test_bad_explicit_chains_are_refused():
    from paper_2509_22857_gb300 import _lib as F
    _, d, q, p = paper_chains.chain("ResNet-32")
    composite = q[3] + 2 * 8192
    assert composite % 8192 == 1 and not O.is_prime(composite)
    bad = [q[:3] + [q[1]] + p,                 # a repeated prime
           q[:3] + [composite] + p,            # = 1 mod 2N, not prime
           q[:3] + [2 ** 31 - 1] + p]          # prime, not = 1 mod 2N
    for chain in bad:
        with pytest.raises(F.FheError) as e:
            F.fhe_ctx_create(LOGN, 3, 0, 0, 0, 1, d, primes=chain)
        assert e.value.code == F.FHE_E_INVAL
    # more digits than Barrett's bound allows for 58-bit primes: 17 > 2^(62-58)
    with pytest.raises(F.FheError) as e:
        F.fhe_ctx_create(LOGN, 16, 58, 40, 58, 1, 29)
    assert e.value.code == F.FHE_E_INVAL


def test_batch_beyond_one_launch_of_33_digit_modup(paper):
    """64 ciphertexts key-switched together at the top of the 33-digit chain:
    33 digits x 34 extended limbs per item put at most 58 items on one
    launch's grid, so the batch is launched in two parts.  Each image's
    relinearised square equals the one-image fhe_square."""
    from types import SimpleNamespace
    from paper_2509_22857_gb300 import model as M
    F, ctx, prm, S, keys, sk, evk = paper
    lay = SimpleNamespace(n_ct=1)
    scale = prm.scale ** 3
    prog = M.Program(tensors=[M.TInfo(lay, prm.L, scale), M.TInfo(lay, prm.L, scale * scale)],
                     steps=[{"kind": F.STEP_ACT, "src": 0, "dst": 1, "c1": 0.0, "c0": 0.0}], input=0, output=1)
    desc = M.ModelDesc(prog, prm.N // 2)
    model = F.fhe_model_load(ctx, desc.desc)
    B = 64
    cts = []
    for i in range(B):
        z = np.random.default_rng(100 + i).uniform(-1, 1, prm.N // 2)
        pt = F.fhe_encode(ctx, z, scale, prm.L)
        cts.append(F.fhe_encrypt(ctx, sk, pt, 300 + i))
        F.fhe_pt_free(pt)
    outs = F.fhe_infer(ctx, model, evk, cts, B, 1)
    for i in (0, 57, 58, 63):
        one = F.fhe_square(ctx, evk, cts[i])
        assert np.array_equal(F.fhe_ct_export(outs[i], prm.N)[0], F.fhe_ct_export(one, prm.N)[0]), i
        F.fhe_ct_free(one)
    for h in outs + cts:
        F.fhe_ct_free(h)
    F.fhe_model_free(model)


def test_rescale_batch_beyond_one_launch(paper):
    """1100 ciphertexts rescaled together at level 32 (2 polynomials x 32
    limbs per item: one launch's grid takes 1023 items, so the batch runs in
    two parts); each equals its one-ciphertext fhe_rescale."""
    from types import SimpleNamespace
    from paper_2509_22857_gb300 import model as M
    F, ctx, prm, S, keys, sk, evk = paper
    lay = SimpleNamespace(n_ct=1)
    scale = prm.scale ** 3
    prog = M.Program(tensors=[M.TInfo(lay, prm.L, scale), M.TInfo(lay, prm.L - 1, scale / prm.q[prm.L])],
                     steps=[{"kind": F.STEP_RESCALE, "src": 0, "dst": 1}], input=0, output=1)
    desc = M.ModelDesc(prog, prm.N // 2)
    model = F.fhe_model_load(ctx, desc.desc)
    z = np.random.default_rng(5).uniform(-1, 1, prm.N // 2)
    pt = F.fhe_encode(ctx, z, scale, prm.L)
    B = 1100
    cts = [F.fhe_encrypt(ctx, sk, pt, 500 + i) for i in range(B)]
    F.fhe_pt_free(pt)
    outs = F.fhe_infer(ctx, model, evk, cts, B, 1)
    for i in (0, 1022, 1023, 1099):
        one = F.fhe_ct_import(ctx, F.fhe_ct_export(cts[i], prm.N)[0], prm.L, scale)
        F.fhe_rescale(ctx, one)
        assert np.array_equal(F.fhe_ct_export(outs[i], prm.N)[0], F.fhe_ct_export(one, prm.N)[0]), i
        F.fhe_ct_free(one)
    for h in outs + cts:
        F.fhe_ct_free(h)
    F.fhe_model_free(model)


def test_double_hoisted_convolution_on_the_papers_chain_bit_exact(paper):
    """A 3x3 convolution (2 -> 4 channels, HW layout) at the top of the
    33-digit chain, double-hoisted: its baby rotations stay in Q u P
    through the many-digit inner product (the form that folds P sigma(c0)
    in), the products run over Q u P and each output takes one ModDown
    from the single special prime.  fhe_eval_conv's ciphertexts equal the
    oracle's limb for limb."""
    import synth
    from oracle import cnn
    from paper_2509_22857_gb300 import model as M
    F, ctx, prm, S, _, _, _ = paper
    net = [{"op": "input", "c": 2, "h": 8, "w": 8}, synth._conv(0, 2, 4, 3, 1, 1, "c1"), {"op": "act", "src": 1},
           {"op": "pool", "src": 2, "k": 2}, {"op": "dense", "src": 3, "cin": 4 * 4 * 4, "cout": 10, "name": "fc"}]
    raw = synth.params(net)
    log_scale = int(round(np.log2(prm.scale)))
    pm = M.compile_network(net, raw, prm.q, LOGN, log_scale, "hw", 1, hoist=2)
    assert M.hoists(pm)[0] == 2 and pm.steps[0]["kind"] == F.STEP_LINEAR
    po = cnn.compile_he(net, cnn.transform(net, raw), prm, "hw", M.giant_steps(pm), 1, 1, M.hoists(pm))
    assert po.rot_steps == pm.rotations
    keys = S.keygen(synth.SEED_KEYS, sorted(po.rot_steps))
    sk, evk = F.fhe_keygen(ctx, synth.SEED_KEYS, sorted(pm.rotations))
    desc = M.ModelDesc(pm, prm.N // 2)
    model = F.fhe_model_load(ctx, desc.desc)
    img = synth.image(0, 2, 8, 8)
    ref = cnn.run_he(S, keys, po, cnn.encrypt_input(S, keys, po, img, 0, synth.enc_seed), stop_after=0)
    ins = []
    for k, v in enumerate(M.input_slots(pm, img, prm.N // 2)):
        pt = F.fhe_encode(ctx, v, M.input_scale(pm), prm.L)
        ins.append(F.fhe_encrypt(ctx, sk, pt, synth.enc_seed(0, k)))
        F.fhe_pt_free(pt)
    st = pm.steps[0]
    outs = F.fhe_eval_conv(ctx, model, evk, 0, ins, pm.tensors[st["dst"]].layout.n_ct)
    want = ref[po.steps[0]["dst"]]
    assert len(outs) == len(want)
    for h, r in zip(outs, want):
        _same(F, S, r, h)
    for h in outs + ins:
        F.fhe_ct_free(h)
    F.fhe_model_free(model)
    F.fhe_evk_free(evk)
    F.fhe_sk_free(sk)
