"""Pins of the oracle's CNN layers: float64 network, transforms, layouts and
the homomorphic evaluation of the small network."""
import numpy as np
import pytest

import synth
from oracle import ckks as C
from oracle import cnn


def test_conv2d_matches_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 9, 9))
    w = rng.normal(size=(4, 3, 3, 3))
    got = cnn.conv2d(x, w, 1, 1)
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    for o in range(4):
        ref = sum(signal.correlate2d(xp[i], w[o, i], mode="valid") for i in range(3))
        assert np.allclose(got[o], ref)
    got2 = cnn.conv2d(x, w, 2, 1)
    assert np.allclose(got2, got[:, ::2, ::2])


def test_avgpool_by_hand():
    x = np.arange(32, dtype=float).reshape(2, 4, 4)
    p = cnn.avgpool(x, 2)
    assert p[0, 0, 0] == (0 + 1 + 4 + 5) / 4 and p[1, 1, 1] == (26 + 27 + 30 + 31) / 4


@pytest.mark.parametrize("arch", ["tiny", "resnet20", "preact_mini"])
def test_transforms_preserve_the_function(arch):
    """Batch-norm folding (Case 2), batch norm fused into the activation that
    follows it (Case 1, the pre-activation network) and forward weight
    redistribution give the same network output (Sec. 4.1-4.2: functional
    equivalence)."""
    net = synth.ARCHS[arch]()
    raw = synth.params(net)
    t = cnn.transform(net, raw)
    hwc = net[0]
    for i in range(2):
        img = synth.image(i, hwc["c"], hwc["h"], hwc["w"])
        y0 = cnn.forward_plain(net, raw, img)
        y1 = cnn.forward_transformed(net, t, img)
        assert np.allclose(y0, y1, rtol=1e-9, atol=1e-12)


def _poly(c2, c1, c0, x):
    return c2 * x * x + c1 * x + c0


def _bivariate(d, x, y):
    dx2, dy2, dxy, dx, dy, d0 = d
    return dx2 * x * x + dy2 * y * y + dxy * x * y + dx * x + dy * y + d0


def test_node_fusing_closed_forms_equal_the_composition():
    """Sec. 4.1 Cases 1, 3 and 4: each closed form evaluated at random points
    equals the composition it replaces, P(B(x)), P(B_X(x) + B_Y(y)) and
    P(B_X(x) + y), written out as separate affine and quadratic steps.
    Every coefficient is exercised: a dropped term, a wrong sign or a swapped
    operand changes the value at some of the points."""
    rng = np.random.default_rng(7)
    k = 64
    bx1, bx0, by1, by0 = (rng.normal(size=k) for _ in range(4))
    c2, c1, c0 = rng.normal(size=3)
    x, y = rng.normal(size=k), rng.normal(size=k)
    p = cnn.fuse_bn_act(bx1, bx0, c2, c1, c0)
    assert np.allclose(_poly(*p, x), _poly(c2, c1, c0, bx1 * x + bx0), rtol=1e-12, atol=1e-12)
    d3 = cnn.fuse_bn_bn_add_act(bx1, bx0, by1, by0, c2, c1, c0)
    ref3 = _poly(c2, c1, c0, (bx1 * x + bx0) + (by1 * y + by0))
    assert np.allclose(_bivariate(d3, x, y), ref3, rtol=1e-12, atol=1e-12)
    d4 = cnn.fuse_bn_add_act(bx1, bx0, c2, c1, c0)
    ref4 = _poly(c2, c1, c0, (bx1 * x + bx0) + y)
    assert np.allclose(_bivariate(d4, x, y), ref4, rtol=1e-12, atol=1e-12)
    # Case 4 is Case 3 with the shortcut's batch norm the identity
    d3i = cnn.fuse_bn_bn_add_act(bx1, bx0, np.ones(k), np.zeros(k), c2, c1, c0)
    for a, b in zip(d3i, d4):
        assert np.allclose(a, b, rtol=1e-14, atol=1e-14)
    # Case 1 with the identity batch norm is the activation itself
    q = cnn.fuse_bn_act(np.ones(k), np.zeros(k), c2, c1, c0)
    assert np.allclose(q[0], c2) and np.allclose(q[1], c1) and np.allclose(q[2], c0)
    # the batch norm's affine form (b1, b0) reproduces (x - mu) gamma / sigma + beta
    prm = {k2: rng.uniform(0.5, 1.5, size=k) for k2 in ("gamma", "sigma")}
    prm.update(mu=rng.normal(size=k), beta=rng.normal(size=k))
    b1, b0 = cnn.bn_linear(prm)
    assert np.allclose(b1 * x + b0, (x - prm["mu"]) * prm["gamma"] / prm["sigma"] + prm["beta"])


def test_case1_fusion_changes_function_if_coefficient_dropped():
    """Sanity of the fused-activation check on a whole network: zeroing the
    linear term of one fused activation changes the pre-activation network's
    output."""
    net = synth.preact_mini()
    raw = synth.params(net)
    t = cnn.transform(net, raw)
    acts = [i for i, nd in enumerate(net) if nd["op"] == "act" and np.ndim(t[i]["c1"]) > 0]
    assert len(acts) == 3
    img = synth.image(0, net[0]["c"], net[0]["h"], net[0]["w"])
    y0 = cnn.forward_plain(net, raw, img)
    assert np.allclose(y0, cnn.forward_transformed(net, t, img), rtol=1e-9, atol=1e-12)
    i = acts[1]
    t[i] = dict(t[i], c1=np.zeros_like(t[i]["c1"]))
    assert not np.allclose(y0, cnn.forward_transformed(net, t, img), rtol=1e-6)


def test_transform_changes_function_if_receiver_not_updated():
    """Sanity of the previous test: dropping the receiver update breaks it."""
    net = synth.tiny()
    raw = synth.params(net)
    t = cnn.transform(net, raw)
    t[4] = dict(t[4], w=raw[4]["w"])  # dense without upsilon
    img = synth.image(0, 3, 16, 16)
    assert not np.allclose(cnn.forward_plain(net, raw, img), cnn.forward_transformed(net, t, img))


def test_layout_lowering_reproduces_conv_on_plain_vectors():
    """The diagonal lowering of a strided conv between channel-packed layouts,
    applied to plain slot vectors with numpy rolls, equals conv2d."""
    rng = np.random.default_rng(1)
    n = 2048
    Lin = cnn.packed_layout(4, 8, 8, 1, 8, 64, n)        # 32 blocks, 4 ch x 8 replicas
    x = rng.normal(size=(4, 8, 8))
    w = rng.normal(size=(8, 4, 3, 3))
    Lout = cnn.packed_layout(8, 4, 4, 2, 8, 64, n)
    diags = cnn._lower_conv(w, 2, 1, Lin, Lout, n)
    vin = np.zeros(n)
    for c in range(4):
        for (ct, base) in Lin.rep[c]:
            for h in range(8):
                for ww in range(8):
                    vin[Lin.slot(base, h, ww)] = x[c, h, ww]
    out = np.zeros(n)
    baby, groups = cnn._bsgs(diags, 64, n)
    for o, gs in groups.items():
        for g, terms in gs.items():
            acc = sum(v * np.roll(vin, -b) for (_, b, v) in terms)
            out += np.roll(acc, -g)
    ref = cnn.conv2d(x, w, 2, 1)
    for c in range(8):
        for (ct, base) in Lout.rep[c]:
            got = np.array([[out[Lout.slot(base, h, ww)] for ww in range(4)] for h in range(4)])
            assert np.allclose(got, ref[c])


@pytest.mark.slow
def test_tiny_network_under_ckks_matches_float64():
    """The whole small network homomorphically: decrypted logits within 1e-3
    of the float64 network and the same argmax."""
    net = synth.tiny()
    raw = synth.params(net)
    t = cnn.transform(net, raw)
    prm = C.make_params(**synth.PRESETS["tiny"])
    prog = cnn.compile_he(net, t, prm, "hw")
    S = C.CKKS(prm)
    keys = S.keygen(synth.SEED_KEYS, sorted(prog.rot_steps))
    img = synth.image(0, 3, 16, 16)
    cts = cnn.encrypt_input(S, keys, prog, img, 0, synth.enc_seed)
    vals = cnn.run_he(S, keys, prog, cts)
    y = cnn.decrypt_logits(S, keys, prog, vals[prog.output_tensor])
    ref = cnn.forward_plain(net, raw, img)
    assert np.max(np.abs(y - ref)) < 1e-3
    assert np.argmax(y) == np.argmax(ref)
    # three rescales (conv, activation, dense): output on q_0, q_1
    assert prog.tensors[prog.output_tensor].level == 1


@pytest.mark.slow
def test_preact_network_under_ckks_matches_float64():
    """The pre-activation network homomorphically, its three batch norms
    fused into per-channel activations (Case 1): decrypted logits within 1e-3
    of the float64 network with separate batch norms, and the same argmax."""
    net = synth.preact_mini()
    raw = synth.params(net)
    t = cnn.transform(net, raw)
    prm = C.make_params(**synth.PRESETS["resnet_mini"])
    prog = cnn.compile_he(net, t, prm, "packed")
    assert sum(1 for s in prog.steps if s["op"] == "act" and "c1_vecs" in s) == 3
    S = C.CKKS(prm)
    keys = S.keygen(synth.SEED_KEYS, sorted(prog.rot_steps))
    hwc = net[0]
    img = synth.image(0, hwc["c"], hwc["h"], hwc["w"])
    cts = cnn.encrypt_input(S, keys, prog, img, 0, synth.enc_seed)
    vals = cnn.run_he(S, keys, prog, cts)
    y = cnn.decrypt_logits(S, keys, prog, vals[prog.output_tensor])
    ref = cnn.forward_plain(net, raw, img)
    assert np.max(np.abs(y - ref)) < 1e-3
    assert np.argmax(y) == np.argmax(ref)


def test_resnet20_program_levels_follow_tower_reuse():
    """ResNet-20 compiled with Delta = 2^25, q ~ 2^50: 20 rescales along the
    network, output at level 0 (Table 1, P2FRT = 20)."""
    net = synth.resnet20()
    raw = synth.params(net)
    t = cnn.transform(net, raw)
    pre = synth.PRESETS["resnet20"]
    # small ring for speed; the level/scale plan depends only on the primes' sizes
    prm = C.make_params(**dict(pre, logn=12))
    c = cnn.Compiler(prm, "packed")
    c.n = 1 << 15                      # slot count of N = 2^16
    prog = c.compile(net, t)
    n_rescale = sum(1 for s in prog.steps if s["op"] == "rescale")
    main_path = [s for s in prog.steps if s["op"] == "rescale"]
    assert prog.tensors[prog.output_tensor].level == 0
    assert n_rescale >= 20
    assert prm.L == 20


@pytest.mark.slow
def test_double_hoisted_network_under_ckks_matches_float64():
    """The mini ResNet with every linear step double-hoisted (baby rotations
    left in Q_l u P, one ModDown per output group): decrypted logits within
    1e-3 of the float64 network, same argmax."""
    net = synth.resnet_mini()
    raw = synth.params(net)
    t = cnn.transform(net, raw)
    prm = C.make_params(**synth.PRESETS["resnet_mini"])
    n_lin = sum(1 for s in cnn.compile_he(net, t, prm, "packed").steps if s["op"] == "linear")
    prog = cnn.compile_he(net, t, prm, "packed", input_lambda=2, hoists=[2] * n_lin)
    assert all(s["hoist"] == 2 for s in prog.steps if s["op"] == "linear")
    S = C.CKKS(prm)
    keys = S.keygen(synth.SEED_KEYS, sorted(prog.rot_steps))
    img = synth.image(0, 3, 8, 8)
    cts = cnn.encrypt_input(S, keys, prog, img, 0, synth.enc_seed)
    vals = cnn.run_he(S, keys, prog, cts)
    y = cnn.decrypt_logits(S, keys, prog, vals[prog.output_tensor])
    ref = cnn.forward_plain(net, raw, img)
    assert np.max(np.abs(y - ref)) < 1e-3
    assert np.argmax(y) == np.argmax(ref)


@pytest.mark.slow
def test_giant_step_choice_keeps_the_layer_function():
    """The first convolution of the mini ResNet under CKKS with giant steps of
    one block and of four blocks (more baby steps, fewer giant steps): both
    decrypt to the float64 convolution (the split is a schedule choice)."""
    net = synth.resnet_mini()
    raw = synth.params(net)
    t = cnn.transform(net, raw)
    pre = synth.PRESETS["resnet_mini"]
    prm = C.make_params(**pre)
    S = C.CKKS(prm)
    img = synth.image(0, 3, 8, 8)
    ref = cnn.conv2d(img, t[1]["w"], 1, 1) + t[1]["bias"][:, None, None]
    n_lin = sum(1 for s in cnn.compile_he(net, t, prm, "packed").steps if s["op"] == "linear")
    got = []
    for k in (1, 4):
        prog = cnn.compile_he(net, t, prm, "packed", [64 * k] * n_lin)
        st = prog.steps[0]
        assert st["op"] == "linear" and st["giant"] == 64 * k
        keys = S.keygen(synth.SEED_KEYS, sorted(prog.rot_steps))
        cts = cnn.encrypt_input(S, keys, prog, img, 0, synth.enc_seed)
        vals = cnn.run_he(S, keys, prog, cts, stop_after=0)
        out = vals[st["dst"]]
        L = prog.tensors[st["dst"]].layout
        z = [S.decrypt_decode(keys, ct).real for ct in out]
        got.append(np.array([[[z[L.rep[c][0][0]][L.slot(L.rep[c][0][1], h, w)] for w in range(8)]
                              for h in range(8)] for c in range(len(L.rep))]))
        # fewer giant rotations with the wider baby steps
        n_giant = sum(1 for gs in st["groups"].values() for g in gs if g)
        n_baby = len(st["baby"])
        if k == 1:
            g1, b1 = n_giant, n_baby
        else:
            assert n_giant < g1 and n_baby > b1
    # key-switching noise at Delta = 2^25, N = 2^12 is about 1e-4 on these values
    for y in got:
        assert np.max(np.abs(y - ref)) < 2e-3
