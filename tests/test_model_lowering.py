"""The package's host-side model lowering (parameter transforms, slot layouts,
diagonals, levels, scales, constants) produces exactly the oracle's program:
same steps, same rotation set, bit-identical diagonal and bias vectors."""
import os

import numpy as np
import pytest

import synth
from oracle import ckks as O
from oracle import cnn
from paper_2509_22857_gb300 import model as M

NAMES = {1: "linear", 2: "rescale", 3: "act", 4: "rotsum", 5: "cmul", 6: "drop", 7: "add"}


def _both(arch, preset, layout, hoist="auto"):
    net = synth.ARCHS[arch]()
    raw = synth.params(net)
    pre = synth.PRESETS[preset]
    prm = O.make_params(**dict(pre, logn=min(pre["logn"], 12)))   # primes' sizes fix the plan
    pm = M.compile_network(net, raw, prm.q, pre["logn"], pre["log_scale"], layout, pre["alpha"], hoist=hoist)
    # the baby-step / giant-step split and the hoisting mode are schedule
    # choices of the package's cost model; the oracle evaluates the same
    # diagonals with the same split and mode
    c = cnn.Compiler(prm, layout, M.giant_steps(pm), hoists=M.hoists(pm))
    c.n = 1 << (pre["logn"] - 1)
    po = c.compile(net, cnn.transform(net, raw))
    return po, pm


def _check(po, pm):
    assert sorted(po.rot_steps) == sorted(pm.rotations)
    ko = [(s["op"], po.tensors[s["dst"]].level, po.tensors[s["dst"]].scale) for s in po.steps]
    km = [(NAMES[s["kind"]], pm.tensors[s["dst"]].level, pm.tensors[s["dst"]].scale) for s in pm.steps]
    assert ko == km
    lo = [s for s in po.steps if s["op"] == "linear"]
    lm = [s for s in pm.steps if s["kind"] == 1]
    assert [s["hoist"] for s in lo] == M.hoists(pm)
    for a, b in zip(lo, lm):
        ga = {(o, g): sorted((i, bb, v.tobytes()) for (i, bb, v) in terms)
              for o, gs in a["groups"].items() for g, terms in gs.items()}
        gb = {k: sorted((i, bb, v.tobytes()) for (i, bb, v) in terms) for k, terms in M.groups_of(b).items()}
        assert ga == gb
        assert a["w_scale"] == b["w_scale"] and a["bias_scale"] == b["bias_scale"]
        assert {k: v.tobytes() for k, v in a["bias"].items()} == {k: v.tobytes() for k, v in b["bias"].items()}
    co = [float(s[k]) for s in po.steps if s["op"] in ("act", "cmul") and "c1_vecs" not in s
          for k in ("c1", "c0", "value") if k in s]
    cm = [s[k] for s in pm.steps if s["kind"] in (3, 5) and "c1_vecs" not in s
          for k in ("c1", "c0", "value") if k in s]
    assert co == cm
    # per-channel activations (node fusing Case 1): the same slot vectors and scales
    vo = [(np.stack(s["c1_vecs"]).tobytes(), np.stack(s["c0_vecs"]).tobytes(), s["c1_scale"], s["c0_scale"])
          for s in po.steps if s["op"] == "act" and "c1_vecs" in s]
    vm = [(np.stack(s["c1_vecs"]).tobytes(), np.stack(s["c0_vecs"]).tobytes(), s["c1_scale"], s["c0_scale"])
          for s in pm.steps if s["kind"] == 3 and "c1_vecs" in s]
    assert vo == vm
    assert [s["steps"] for s in po.steps if s["op"] == "rotsum"] == \
        [s["steps"] for s in pm.steps if s["kind"] == 4]


def test_tiny_hw_program_matches_oracle():
    _check(*_both("tiny", "tiny", "hw"))


def test_mini_resnet_program_matches_oracle():
    _check(*_both("resnet_mini", "resnet_mini", "packed"))


@pytest.mark.parametrize("hoist", [1, 2])
def test_forced_hoisting_mode_reaches_both_compilers(hoist):
    po, pm = _both("resnet_mini", "resnet_mini", "packed", hoist=hoist)
    assert set(M.hoists(pm)) == {hoist}
    _check(po, pm)


def test_mini_vgg_program_matches_oracle():
    _check(*_both("vgg_mini", "resnet_mini", "packed"))


def test_mini_preact_program_matches_oracle():
    """Pre-activation blocks: each block's batch norm fused into its
    activation (Case 1), per-channel coefficients, per-channel upsilon taken
    up by the next convolution and the dense layer."""
    po, pm = _both("preact_mini", "resnet_mini", "packed")
    assert sum(1 for s in pm.steps if s["kind"] == 3 and "c1_vecs" in s) == 3
    _check(po, pm)


@pytest.mark.slow
def test_resnet20_program_matches_oracle():
    po, pm = _both("resnet20", "resnet20", "packed")
    _check(po, pm)
    # 20 levels consumed along the main path: output at level 0 (Table 1, P2FRT)
    assert pm.tensors[pm.output].level == 0


def test_input_slots_match_oracle():
    po, pm = _both("resnet_mini", "resnet_mini", "packed")
    img = synth.image(3, 3, 8, 8)
    a = cnn.input_vectors(po, img, 2048)
    b = M.input_slots(pm, img, 2048)
    assert len(a) == len(b) and all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("hoist", [1, "auto"])
def test_cost_model_prefers_wider_baby_steps_for_wide_layers(hoist):
    """A 16-channel packed convolution: giant steps of one block need 15 giant
    rotations per output; the cost model moves part of them to hoisted baby
    steps, and never picks a split (and hoisting mode) that costs more than
    one block with either mode."""
    po, pm = _both("resnet_mini", "resnet_mini", "packed", hoist=hoist)
    lin = [s for s in pm.steps if s["kind"] == 1]
    blk = pm.tensors[pm.input].layout.block
    assert any(s["giant"] > blk for s in lin)
    modes = (1,) if hoist == 1 else (1, 2)
    for s in lin:
        terms = M.Terms(s["t_out"], s["t_ct"], s["t_giant"] + s["t_baby"], s["t_vid"], s["vecs"])
        lv = pm.tensors[s["src"]].level
        chosen = M.split_cost(terms, s["giant"], lv, 3, s["hoist"])
        assert chosen <= min(M.split_cost(terms, blk, lv, 3, h) for h in modes) + 1e-9
        if hoist == 1:
            assert M.bsgs_cost(terms, s["giant"], lv, 3) <= M.bsgs_cost(terms, blk, lv, 3)


def test_double_hoisting_cost_counts_one_moddown_per_rotated_group():
    """split_cost with double hoisting against a count by hand on a toy term
    set: two inputs, baby steps {1, 2}, giant steps {0, 4}, one output."""
    r = np.array([0, 1, 2, 4, 5, 6, 1])
    ct = np.array([0, 0, 0, 0, 0, 0, 1])
    terms = M.Terms(np.zeros(7, dtype=np.int64), ct, r, np.arange(7), [None] * 7)
    mu, ip, md = M.ks_cost(5, 3)
    nl, alpha = 6, 3
    # babies (0,1) (0,2) (1,1); giants (0,4); rotated groups (0,0) (0,4)
    ks = 2 * mu + 3 * ip + 2 * md + 1 * (mu + ip) + 1 * md
    mac = (7 * 2 * nl + 5 * 2 * alpha) / 8 * M.MAC_WEIGHT
    assert M.split_cost(terms, 4, 5, alpha, 2) == pytest.approx(ks + mac)
    assert M.split_cost(terms, 4, 5, alpha, 1) == pytest.approx(M.bsgs_cost(terms, 4, 5, alpha) + 7 * 2 * nl / 8
                                                                 * M.MAC_WEIGHT)



def _ensemble_both(k=4, members=3):
    net = synth.resnet18_mini()
    raws = synth.cluster_joint([synth.params(net, m) for m in range(members)], net, k)
    pre = synth.PRESETS["resnet18_mini"]
    prm = O.make_params(**pre)
    pm = M.compile_network(net, raws, prm.q, pre["logn"], pre["log_scale"], "hw_ens", pre["alpha"])
    po = cnn.compile_he(net, [cnn.transform(net, r) for r in raws], prm, "hw_ens", M.giant_steps(pm), members,
                        hoists=M.hoists(pm))
    return po, pm


def test_clustered_ensemble_program_matches_oracle():
    """ResNet-18's structure, three members in blocks 0..2 of the HW layout,
    weights clustered jointly (4 centroids per layer): same program as the
    oracle's, and every convolution needs at most 4 x 9 distinct plaintexts."""
    po, pm = _ensemble_both()
    _check(po, pm)
    for st in pm.steps:
        if st["kind"] == 1 and len(pm.tensors[st["src"]].layout.copies[0]) == 3 \
                and pm.tensors[st["src"]].layout.H > 1:
            assert len(st["vecs"]) <= 4 * 9
    # 18 levels along the network (Table 1, ResNet-18 P2FRT = 18): output on q_0
    assert pm.tensors[pm.output].level == 0


def test_input_at_delta_squared_costs_no_level():
    """Encrypting the image at Delta^2 (first-layer rotations at scale
    Delta^2) leaves ResNet-20's plan at the same depth: output at level 0
    after the same number of rescales, in both compilers."""
    net = synth.resnet20()
    raw = synth.params(net)
    pre = synth.PRESETS["resnet20"]
    prm = O.make_params(**dict(pre, logn=12))
    plans = {}
    for lam in (1, 2):
        pm = M.compile_network(net, raw, prm.q, pre["logn"], pre["log_scale"], "packed", pre["alpha"],
                               input_lambda=lam)
        c = cnn.Compiler(prm, "packed", M.giant_steps(pm), 1, lam, M.hoists(pm))
        c.n = 1 << (pre["logn"] - 1)
        po = c.compile(net, cnn.transform(net, raw))
        _check(po, pm)
        assert M.input_scale(pm) == po.tensors[po.input_tensor].scale == prm.scale ** lam
        plans[lam] = (pm.tensors[pm.output].level, sum(1 for s in pm.steps if s["kind"] == 2))
    assert plans[1] == plans[2] == (0, plans[1][1])


@pytest.mark.slow
def test_resnet32_on_the_papers_chain_uses_table1_levels():
    """ResNet-32 compiled on the paper's own chain (Delta = 2^26, 52-bit
    primes, tower reuse) enters at level L = 32 and leaves at level 0: the
    32 levels of Table 1's P2FRT column for ResNet-32."""
    pp = synth.PAPER_PARAMS["resnet32"]
    levels = {r.split()[0]: int(r.split()[-1]) for r in open(os.path.join(os.path.dirname(__file__), "golden",
                                                                          "table1_levels.txt"))
              if r.strip() and not r.startswith("#")}
    net = synth.resnet32()
    prog = M.compile_network(net, synth.params(net), pp["q"], pp["logn"], pp["log_scale"], "packed", pp["alpha"],
                             input_lambda=2)
    assert prog.tensors[prog.input].level == pp["L"] == levels["ResNet-32"]
    assert prog.tensors[prog.output].level == 0


def test_ensemble_work_is_flat_in_members():
    """Sec. 5.3 (ensembles share ciphertexts): with the members in the blocks
    of one HW layout, the homomorphic work of an image does not grow with M
    -- the same input ciphertexts, levels and plaintext-MAC terms for
    M = 1..4 -- except ceil(log2 M) rotations that sum the members' blocks
    before the output (the structural reason the paper's ensemble time is
    flat in M)."""
    pre = synth.PRESETS["resnet18_mini"]
    prm = O.make_params(**pre)
    net = synth.resnet18_mini()
    base = None
    for members in (1, 2, 3, 4):
        raws = synth.cluster_joint([synth.params(net, m) for m in range(members)], net, 4)
        prog = M.compile_network(net, raws, prm.q, pre["logn"], pre["log_scale"], "hw_ens", pre["alpha"])
        got = (prog.tensors[prog.input].layout.n_ct, prog.tensors[prog.input].level,
               prog.tensors[prog.output].level, sum(len(st["t_out"]) for st in prog.steps if st["kind"] == 1))
        ks = sum(M.keyswitch_census(prog).values())
        if base is None:
            base = (got, ks)
        assert got == base[0], (members, got, base[0])
        assert ks == base[1] + (members - 1).bit_length(), (members, ks, base[1])


@pytest.mark.parametrize("arch,layout", [("vgg_mini", "packed"), ("resnet_mini", "packed")])
def test_on_demand_program_describes_the_resident_one(arch, layout):
    """A program compiled for on-demand encoding keeps its convolution rows
    sparse; term for term it is the resident program (same outputs, giant
    and baby steps, inputs), and every sparse row is the resident vector."""
    pre = synth.PRESETS["resnet_mini"]
    prm = O.make_params(**pre)
    net = synth.ARCHS[arch]()
    raw = synth.params(net)
    dense = M.compile_network(net, raw, prm.q, pre["logn"], pre["log_scale"], layout, pre["alpha"])
    od = M.compile_network(net, raw, prm.q, pre["logn"], pre["log_scale"], layout, pre["alpha"], on_demand=True)
    assert len(dense.steps) == len(od.steps) and dense.rotations == od.rotations
    n = prm.N // 2
    n_sparse = 0
    for a, b in zip(dense.steps, od.steps):
        assert a["kind"] == b["kind"]
        if a["kind"] != 1:
            continue
        for k in ("t_out", "t_giant", "t_ct", "t_baby"):
            assert np.array_equal(a[k], b[k]), k
        sparse = isinstance(b["vecs"][0], M.SparseVec)
        n_sparse += sparse
        for t in range(len(a["t_out"])):
            va, vb = a["vecs"][a["t_vid"][t]], b["vecs"][b["t_vid"][t]]
            assert np.array_equal(va, vb.dense(n) if sparse else vb)
            if sparse:
                assert np.count_nonzero(va) == len(vb)
    assert n_sparse >= 2     # the packed convolutions


def test_model_descriptor_keeps_its_arrays_alive():
    """The C descriptor points into arrays its ModelDesc owns; taken on its
    own (the owner otherwise unreferenced) it still reads the program."""
    import gc
    import ctypes
    pre = synth.PRESETS["resnet_mini"]
    prm = O.make_params(**pre)
    net = synth.resnet_mini()
    pm = M.compile_network(net, synth.params(net), prm.q, pre["logn"], pre["log_scale"], "packed", pre["alpha"])
    d = M.ModelDesc(pm, prm.N // 2).desc
    gc.collect()
    big = [np.full(1 << 16, 7, dtype=np.int64) for _ in range(64)]   # reuse freed memory if any was freed
    assert d.n_steps == len(pm.steps) and d.n_tensors == len(pm.tensors)
    assert [d.tensor_level[i] for i in range(d.n_tensors)] == [t.level for t in pm.tensors]
    st = [d.steps[i] for i in range(d.n_steps)]
    lin = [s for s in st if s.kind == 1]
    assert ctypes.addressof(lin[0]) and lin[0].term_ct[0] == int(pm.steps[0]["t_ct"][0])
    del big


def test_double_hoisting_stays_within_its_memory_budget():
    """The planner admits double hoisting only where a step's group sums
    over Q_l u P fit the per-image budget: with a budget of 0 bytes every
    step with baby rotations is single-hoisted, and every double-hoisted
    step of the default plan fits the default budget."""
    pre = synth.PRESETS["resnet_mini"]
    prm = O.make_params(**pre)
    net = synth.resnet_mini()
    raw = synth.params(net)
    tight = M.compile_network(net, raw, prm.q, pre["logn"], pre["log_scale"], "packed", pre["alpha"], dh_bytes=0)
    assert set(M.hoists(tight)) == {1}
    plan = M.compile_network(net, raw, prm.q, pre["logn"], pre["log_scale"], "packed", pre["alpha"])
    for st in plan.steps:
        if st["kind"] == 1 and st["hoist"] == 2:
            terms = M.Terms(st["t_out"], st["t_ct"], st["t_giant"] + st["t_baby"], st["t_vid"], st["vecs"])
            lv = plan.tensors[st["src"]].level
            assert 0 < M.dh_group_bytes(terms, st["giant"], lv, pre["alpha"], pre["logn"]) <= 1 << 30
